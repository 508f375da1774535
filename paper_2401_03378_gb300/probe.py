"""FP64 pipe probe: DFMA throughput of the current GPU, optionally with only
some lanes of each warp active (``python -m paper_2401_03378_gb300.probe``)."""
from __future__ import annotations

import argparse

import torch

from .hydro import fp64_probe, sm_count


def measure(lanes: int, iters: int = 20000, per_sm: int = 8, threads: int = 256, repeats: int = 3):
    """(best milliseconds, FP64 TFLOP/s counted over the active lanes)."""
    blocks = sm_count() * per_sm
    out = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    fp64_probe(blocks, threads, 100, out, lanes)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fp64_probe(blocks, threads, iters, out, lanes)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    flops = 16.0 * iters * blocks * (threads // 32) * lanes
    return best, flops / (best * 1e-3) / 1e12


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--lanes", default="32,16,8,4,1")
    ap.add_argument("--iters", type=int, default=20000)
    args = ap.parse_args(argv)
    for lanes in [int(x) for x in args.lanes.split(",")]:
        ms, tf = measure(lanes, args.iters)
        print(f"lanes={lanes:2d} ms={ms:9.3f} TFLOP/s(active lanes)={tf:7.3f}")


if __name__ == "__main__":
    main()
