"""FP64 pipe probe: throughput of FP64 fused multiply-adds (constant or
register operands), adds and multiplies on the current GPU, optionally with
only some lanes of each warp active (``python -m paper_2401_03378_gb300.probe``)."""
from __future__ import annotations

import argparse

import torch

from .hydro import fp64_probe, sm_count


FORMS = {0: "DFMA, two constant operands", 1: "DFMA, per-thread registers", 2: "DADD", 3: "DMUL",
         4: "DFMA, warp-uniform registers"}


def measure(lanes: int, iters: int = 20000, per_sm: int = 8, threads: int = 256, repeats: int = 3, form: int = 1):
    """(best milliseconds, FP64 operations per second over the active lanes)."""
    blocks = sm_count() * per_sm
    out = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    fp64_probe(blocks, threads, 100, out, lanes, form)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fp64_probe(blocks, threads, iters, out, lanes, form)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    ops = 8.0 * iters * blocks * (threads // 32) * lanes
    return best, ops / (best * 1e-3)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--lanes", default="32,16,8,4,1")
    ap.add_argument("--forms", default="1", help="comma list of 0..4 (%s)" % FORMS)
    ap.add_argument("--iters", type=int, default=20000)
    ap.add_argument("--clock-mhz", type=float, default=2070.0, help="SM clock for the per-clock figure")
    args = ap.parse_args(argv)
    sms = sm_count()
    for form in [int(x) for x in args.forms.split(",")]:
        for lanes in [int(x) for x in args.lanes.split(",")]:
            ms, ops = measure(lanes, args.iters, form=form)
            per_clk = ops / sms / (args.clock_mhz * 1e6)
            print(f"form={form} ({FORMS[form]:28s}) lanes={lanes:2d} ms={ms:9.3f} "
                  f"G ops/s(active lanes)={ops / 1e9:8.2f} lanes/clk/SM={per_clk:6.3f}")


if __name__ == "__main__":
    main()
