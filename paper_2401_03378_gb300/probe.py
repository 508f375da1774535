"""FP64 pipe probe: throughput of FP64 fused multiply-adds (constant or
register operands), adds and multiplies on the current GPU, optionally with
only some lanes of each warp active (``python -m paper_2401_03378_gb300.probe``).

``--count`` launches the instruction-count probe of the stage kernel's
arithmetic building blocks instead (gbh_op_count_probe), one launch per
building block, for ncu's FP64 instruction counters; it prints the number of
calls of each launch."""
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
    # the active lanes: the first `lanes` of every warp, the last (partial) warp included
    active = (threads // 32) * lanes + min(lanes, threads % 32)
    ops = 8.0 * iters * blocks * active
    return best, ops / (best * 1e-3)


OP_COUNT = {0: "cons->prim, one cell", 1: "x/y slope item (3 cells), one variable", 2: "HLLC, one face",
            3: "3-D update, one variable", 4: "second-stage combine, one variable",
            5: "CFL epilogue, one cell", 6: "z-march slope and face states, one variable",
            7: "block-boundary face states, one variable"}


def op_count_inputs(fn: int, n: int, seed: int = 0) -> torch.Tensor:
    """Valid inputs of gbh_op_count_probe for n threads: conserved states (fn 0, 5),
    two primitive states (fn 2) or values in [0.5, 2] (the rest)."""
    g = torch.Generator().manual_seed(seed)
    x = 0.5 + 1.5 * torch.rand((n, 10), generator=g, dtype=torch.float64)
    if fn in (0, 5):
        rho, u, v, w, p = x[:, 0], x[:, 1] - 1.25, x[:, 2] - 1.25, x[:, 3] - 1.25, x[:, 4]
        x[:, 1], x[:, 2], x[:, 3] = rho * u, rho * v, rho * w
        x[:, 4] = p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)
    elif fn == 2:
        x[:, 1] -= 1.25
        x[:, 2] -= 1.25
        x[:, 3] -= 1.25
        x[:, 6] -= 1.25
        x[:, 7] -= 1.25
        x[:, 8] -= 1.25
    return x.contiguous()


def op_count(fn: int, blocks: int, threads: int, iters: int) -> torch.Tensor:
    """One launch of gbh_op_count_probe; returns the device buffer it ran on."""
    from . import _abi
    lib = _abi.load()
    io = op_count_inputs(fn, blocks * threads).cuda()
    rc = lib.gbh_op_count_probe(int(fn), int(blocks), int(threads), int(iters), io.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise _abi.GbhError(rc, lib.gbh_last_error(None).decode())
    return io


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--lanes", default="32,16,8,4,1")
    ap.add_argument("--forms", default="1", help="comma list of 0..4 (%s)" % FORMS)
    ap.add_argument("--iters", type=int, default=20000)
    ap.add_argument("--clock-mhz", type=float, default=2070.0, help="SM clock for the per-clock figure")
    ap.add_argument("--threads", default="256", help="comma list of threads per CTA")
    ap.add_argument("--per-sm", type=int, default=8, help="CTAs per SM in the grid")
    ap.add_argument("--count", action="store_true", help="launch the instruction-count probe instead")
    args = ap.parse_args(argv)
    sms = sm_count()
    if args.count:
        blocks, threads, iters = 2 * sms, 128, 64
        for fn, name in OP_COUNT.items():
            op_count(fn, blocks, threads, iters)
            torch.cuda.synchronize()
            print(f"op_count fn={fn} ({name}): calls={blocks * threads * iters}")
        return
    for threads in [int(x) for x in args.threads.split(",")]:
        for form in [int(x) for x in args.forms.split(",")]:
            for lanes in [int(x) for x in args.lanes.split(",")]:
                ms, ops = measure(lanes, args.iters, per_sm=args.per_sm, threads=threads, form=form)
                per_clk = ops / sms / (args.clock_mhz * 1e6)
                print(f"threads={threads:4d} per_sm={args.per_sm} form={form} ({FORMS[form]:28s}) lanes={lanes:2d} "
                      f"ms={ms:9.3f} G ops/s(active lanes)={ops / 1e9:8.2f} lanes/clk/SM={per_clk:6.3f}")


if __name__ == "__main__":
    main()
