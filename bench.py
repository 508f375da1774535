"""Benchmark: FP64 zone-updates/s of the block-structured Euler update.

Workload: 3-D Sedov blast at 256^3 = 4096 blocks of 16^3 interior cells + 4
guard cells, gamma 1.4, CFL 0.8, SSP-RK2 with MC-limited PLM and HLLC, dt on
the device every step.  A step = one full SSP-RK2 time step (two stage kernels
with the guard fill fused, the CFL reduction fused into the second) on the
whole domain.  The state (2.26 GB) is larger than L2 (129 MB), so no flush
is needed between steps.

One JSON line on rank 0.  Under torchrun every rank advances its own replica
(the method's only exchanges are guard cells and the dt minimum inside one
domain on one GPU), and `value` sums all ranks' zones over the slowest
rank's time.

--impl reference times the FP64 CPU oracle on the host cores instead (the
same scheme, same config and metric), rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FP64 zone-updates/s (3D Sedov 256^3, SSP-RK2 PLM-MC HLLC)"
UNIT = "zone-updates/s"
WORKLOAD = ("3D Sedov blast 256^3: 4096 blocks of 16^3 + 4 guard cells, FP64, gamma 1.4, CFL 0.8, "
            "SSP-RK2 (non-telescoping), MC-limited PLM, HLLC, CFL dt on device each step")
# Algorithmic FP64 operations per zone-update (+, -, *, /, sqrt = 1 each),
# counted on the oracle's arithmetic by oracle/opcount.cpp: stage 1 570 (its
# 13 for the conversion of its input included), stage 2 585 + 11 for the CFL
# signal speed of the new state.  calcEos runs once per stage: the primitives
# of the new state serve the CFL speed and the next step's first stage, so
# the conversion is counted once (the oracle converts the new state a second
# time for its dt, 13 more: 1179 per zone-update).
FLOPS_STAGE1 = 570
FLOPS_STAGE2 = 585 + 11
# FP64 peak derived from the nominal GB300 rate (1.25 TFLOP/s) at 152 SMs and
# 2070 MHz: 2 FP64 FMA lanes per SM per clock -> 152 * 2 * 2 * 2.07e9.
FP64_PEAK_NOMINAL = 152 * 2 * 2 * 2.07e9
# stage 1: read U^n and its primitives, write U1 and its primitives (160 B);
# stage 2: read U1, its primitives and U^n, write U^{n+1} and its primitives (200 B)
ALG_BYTES_PER_ZONE = 360


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def aggregate(local_seconds: float, local_units: float, world: int, group=None):
    """(max seconds over ranks, total units over ranks) -- the job's clock and work."""
    if world == 1:
        return local_seconds, local_units
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_seconds], dtype=torch.float64)
    u = torch.tensor([local_units], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t, u = t.cuda(), u.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampler running during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        counts = {names[i]: sum(1 for r in rows if r[5 + i].lower() == "active") for i in range(4)}
        reasons = sorted(k for k, v in counts.items() if v)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "sm_mhz_min": min(sm) if sm else None, "reasons": reasons,
                "reason_samples": {k: v for k, v in counts.items() if v}, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def source_hash():
    """Hash of what the stage kernel compiles from: its sources, the headers it
    includes and the definitions of Layout, Eos and StageArgs."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2401_03378_gb300", "csrc")
    for rel in ("gbh_stage.cu", "gbh_device.cuh", "gbh_fastmath.cuh", "gbh_gather.cuh", "gbh_check.cuh"):
        with open(os.path.join(csrc, rel), "rb") as f:
            h.update(f.read())
    with open(os.path.join(csrc, "gbh_internal.h")) as f:
        text = f.read()
    a = text.index("struct Layout {")
    b = text.index("};", text.index("struct StageArgs {")) + 2
    h.update(text[a:b].encode())
    return h.hexdigest()[:16]


def measured_traffic(zones: int):
    """DRAM bytes per stage-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != source_hash():
        return None
    per_zone = rec["dram_bytes_per_launch"] / rec["zones"]
    return per_zone * zones


def measured_fp64_inst(zones: int):
    """FP64 thread instructions per stage-kernel launch (mean of the two stages)
    from the committed ncu record, if it was taken on the current kernel source
    (else None)."""
    path = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != source_hash() or "fp64_inst_per_zone_stage1" not in rec:
        return None
    return 0.5 * (rec["fp64_inst_per_zone_stage1"] + rec["fp64_inst_per_zone_stage2"]) * zones


def fp64_issue(inst_per_launch, ms_per_launch: float, sm_mhz, sms: int):
    """FP64 lanes issued per SM clock (2 is the unit's peak) over a launch."""
    if not inst_per_launch or not ms_per_launch or not sms:
        return None
    mhz = sm_mhz if sm_mhz else 2070.0
    lanes = inst_per_launch / (ms_per_launch / 1e3 * mhz * 1e6 * sms)
    return {"fp64_inst_per_launch": inst_per_launch, "lanes_per_sm_clock": lanes, "of_peak_lanes": lanes / 2.0,
            "sm_mhz": mhz, "sm_mhz_source": "sampled median" if sm_mhz else "nominal (no clock samples)",
            "note": "FP64 thread instructions per zone from the ncu record of the same kernel source, "
                    "times zones, over the CUDA-event launch time"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def bench_config(lat):
    """The workload object both arms print (identical for the same --nb)."""
    workload = WORKLOAD if lat.nb[0] == 16 else f"{WORKLOAD} (at {lat.global_cells[0]}^3)"
    return {"workload": workload, "zones": lat.interior_cells, "blocks": lat.nblocks,
            "l2": "state %.2f GB per array > 129 MB L2: no flush needed" % (
                8 * lat.nblocks * 5 * lat.padded[0] * lat.padded[1] * lat.padded[2] / 1e9)}


def host_cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def autotuned(h, U, rings, time_default):
    """Run the library's autotuner on U and describe its choice; when that is
    not the default decomposition (whole block per work item, one item per
    CTA, unsplit tiles), time_default() is timed with the default restored
    before the choice is set back."""
    kc, ipc = h.autotune(U)
    splits = {r: h.tile_split(r) for r in rings}
    full = h.n[2] if h.ndim == 3 else 1
    choice = {"kchunk": kc, "items_per_cta": ipc, "ysplit": {str(r): s for r, s in splits.items()}}
    is_default = kc == full and ipc == 1 and all(s == 1 for s in splits.values())
    out = {"chosen": choice, "chosen_is_default": is_default, "default_ms_per_step": None}
    if not is_default:
        h.set_decomposition(0, 1)
        for r in rings:
            h.set_tile_split(r, 1)
        out["default_ms_per_step"] = time_default()
        h.set_decomposition(kc if h.ndim == 3 else 0, ipc)
        for r, sp in splits.items():
            h.set_tile_split(r, sp)
    return out


def lat_kchunk(lat):
    """z planes of one work item in the default decomposition (the whole block)."""
    return lat.n[2] if lat.ndim == 3 else 1


def make_problem(nb: int):
    import workloads as wl
    lat = wl.lattice_3d(nb, nb, nb, 16, 16, 16, 4)
    return lat, wl.sedov(lat)


def fp64_probe_tflops(gb, torch, form=1):
    """FP64 flop/s of the probe's fused multiply-add chains: form 1 with all
    operands in registers (the fastest form), form 0 with constant operands."""
    sms = gb.sm_count()
    blocks, threads, iters = sms * 8, 256, 20000
    out = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    gb.fp64_probe(blocks, threads, 100, out, 32, form)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gb.fp64_probe(blocks, threads, iters, out, 32, form)
        e1.record()
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1e3
        best = max(best, 16.0 * iters * blocks * threads / s)
    return best


def run_gpu(args):
    import numpy as np
    import torch
    import paper_2401_03378_gb300 as gb

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lat, U0 = make_problem(args.nb)
    zones = lat.interior_cells
    h = gb.Hydro.from_lattice(lat)
    U = torch.from_numpy(U0).cuda()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def ms_per_step(n=10):
        V = torch.from_numpy(U0).cuda()
        d = h.compute_dt(V)
        for _ in range(3):
            h.step_cfl(V, d)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record()
        for _ in range(n):
            h.step_cfl(V, d)
        e1.record()
        barrier()
        return e0.elapsed_time(e1) / n

    # the decomposition the library's autotuner picks on this workload (the
    # timed loop below runs with it)
    tuning = autotuned(h, U, (0,), ms_per_step) if args.autotune else None
    dt = h.compute_dt(U)
    for _ in range(args.warmup):
        h.step_cfl(U, dt)
    torch.cuda.synchronize()

    h.set_kernel_timing(True)
    h.stage_kernel_time()  # clear
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        e0.record(stream)
        h.advance(U, args.steps, dt)      # K steps of one call (CFL dt on the device each step)
        e1.record(stream)
        barrier()
    secs = e0.elapsed_time(e1) / 1e3
    stage_ms, stage_launches = h.stage_kernel_time()
    h.set_kernel_timing(False)
    clocks = clk.summary()
    tmax, units = aggregate(secs, float(zones) * args.steps, world)
    value = units / tmax
    # the same loop repeated (5 x 10 steps, CUDA events each): spread and median
    reps = []
    for _ in range(5 if args.repeats else 0):
        barrier()
        e0.record(stream)
        h.advance(U, 10, dt)
        e1.record(stream)
        barrier()
        reps.append(e0.elapsed_time(e1) / 10)
    repeats = ({"ms_per_step": reps, "median_ms_per_step": float(np.median(reps)), "steps_each": 10}
               if reps else None)
    nbad = h.check_state(U)

    # end to end through the host-buffer C-ABI call: every step copies the
    # state in from pinned host memory and the updated state back out
    e2e = None
    if args.e2e_steps > 0:
        # through hydro_step_host_interior: every step copies the interior
        # cells in from pinned host memory and the new state (and its dt) back
        # out, overlapped with the stages chunk by chunk (guard cells are not
        # inputs of a step: every stage fills them itself)
        g, gz = h.nguard, (h.nguard if h.ndim == 3 else 0)
        n = h.interior_shape
        Ui = torch.from_numpy(np.ascontiguousarray(
            U0[:, :, gz:gz + n[2], g:g + n[3], g:g + n[4]])).pin_memory()
        dth = np.zeros(1)
        for _ in range(3):    # warm: allocates the device buffers, computes the first dt
            h.step_host_interior(Ui, dth)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            h.step_host_interior(Ui, dth)
        barrier()
        esecs = time.perf_counter() - t0
        etmax, eunits = aggregate(esecs, float(zones) * args.e2e_steps, world)
        ibytes = Ui.numel() * Ui.element_size()
        # the same pipelined step on a host state in the padded layout
        # (guard cells copied too)
        Uh = torch.from_numpy(U0.copy()).pin_memory()
        dtp = np.zeros(1)
        for _ in range(3):
            h.step_host(Uh, dtp)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            h.step_host(Uh, dtp)
        barrier()
        psecs = time.perf_counter() - t0
        ptmax, punits = aggregate(psecs, float(zones) * args.e2e_steps, world)
        nbytes = h.lib.gbh_state_bytes(h.ctx)
        # the unpipelined host-buffer call, for comparison
        hist = np.zeros(1)
        h.advance_host(Uh, 1, hist)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            h.advance_host(Uh, 1, hist)
        barrier()
        usecs = time.perf_counter() - t0
        utmax, uunits = aggregate(usecs, float(zones) * args.e2e_steps, world)
        e2e = {"value": eunits / etmax, "unit": UNIT, "h2d_bytes_per_step": int(ibytes) + 8,
               "d2h_bytes_per_step": int(ibytes) + 8, "steps": args.e2e_steps,
               "call": "hydro_step_host_interior (interior cells only; copies overlapped with the stages)",
               "padded_step_host": {"value": punits / ptmax, "unit": UNIT, "h2d_bytes_per_step": int(nbytes) + 8,
                                    "d2h_bytes_per_step": int(nbytes) + 8,
                                    "call": "hydro_step_host (padded state; copies overlapped with the stages)"},
               "unpipelined_advance_host": {"value": uunits / utmax, "unit": UNIT,
                                            "h2d_bytes_per_step": int(nbytes), "d2h_bytes_per_step": int(nbytes)}}

    two_level = None
    if args.two_level_steps > 0:
        two_level = run_two_level(args, gb, torch, barrier)
    ensemble = None
    if args.ensemble_steps > 0:
        ensemble = run_ensemble(args, gb, torch, barrier)
    tl_ensemble = None
    if args.tl_ensemble_steps > 0:
        tl_ensemble = run_two_level_ensemble(args, gb, torch, barrier)
    adjoint = None
    if args.adjoint_steps > 0:
        adjoint = run_adjoint(args, gb, torch, barrier)
    variants = None
    if args.variant_steps > 0:
        variants = run_variants(args, gb, torch, barrier, 1e3 * tmax / args.steps)

    # roofline of the dominant kernel (the fused stage kernel, both stages)
    flops_per_launch = 0.5 * (FLOPS_STAGE1 + FLOPS_STAGE2) * zones
    ms_per_launch = stage_ms / max(stage_launches, 1)
    achieved = flops_per_launch / (ms_per_launch / 1e3)
    probe = fp64_probe_tflops(gb, torch, 1) if rank == 0 else None
    probe_const = fp64_probe_tflops(gb, torch, 0) if rank == 0 else None
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs")
    traffic = measured_traffic(zones)
    roof = {
        "kernel": ("gbh face_flux_kernel<16,3D> + stage_kernel<16,3D> per stage, timed together (both SSP-RK2 "
                   "stages: each block face solved once in the pre-pass, fused halo gather, dt epilogue)"
                   if h.face_prepass() else
                   "gbh stage_kernel<16,3D> (both SSP-RK2 stages, fused halo gather, dt epilogue)"),
        "bound": "alu",
        "achieved": achieved / 1e12,
        "peak": FP64_PEAK_NOMINAL / 1e12,
        "unit": "TFLOP/s",
        "frac": achieved / FP64_PEAK_NOMINAL,
        "peak_source": "derived: nominal GB300 FP64 1.25 TFLOP/s = 152 SMs x 2 FMA lanes x 2 flops x 2.07 GHz",
        "peak_probe_measured": probe / 1e12 if probe else None,
        "peak_probe_note": "DFMA chains with all operands in registers; with constant operands: %.3f TFLOP/s"
                           % (probe_const / 1e12) if probe_const else None,
        "frac_of_probe": achieved / probe if probe else None,
        "flops_per_zone_update": FLOPS_STAGE1 + FLOPS_STAGE2,
        "launches": stage_launches,
        "ms_per_launch": ms_per_launch,
        "traffic": traffic,
        "algorithmic_bytes_per_launch": ALG_BYTES_PER_ZONE / 2 * zones,
        "hbm_frac": (ALG_BYTES_PER_ZONE / 2 * zones / (ms_per_launch / 1e3)) / (hbm * 1e9) if hbm else None,
        "fp64_issue": fp64_issue(measured_fp64_inst(zones), ms_per_launch, clocks.get("sm_mhz"), gb.sm_count()),
    }
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * tmax / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded Sedov initial condition)",
        "config": bench_config(lat),
        "parallelism": f"replicas x{world}",
        "gpu_launches": (5 if h.face_prepass() else 3) * args.steps,
        "autotune": tuning,
        "clocks": clocks,
        "repeats": repeats,
        "roofline": roof,
        "e2e": e2e,
        "two_level": two_level,
        "ensemble": ensemble,
        "two_level_ensemble": tl_ensemble,
        "adjoint": adjoint,
        "variants": variants,
        "unphysical_cells": nbad,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, U0, lat)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_variants(args, gb, torch, barrier, ms_headline):
    """The headline workload in the paper's other stepper variants: the
    telescoping mode (one guard fill per step, earlier stages also update a
    ring of guard cells) with two stages, and the three-stage SSP-RK without
    and with telescoping (the latter on 6 guard cells).  Step time against
    the headline (non-telescoping, two-stage) step measured above."""
    import workloads as wl
    nb = args.nb
    out = {}
    for name, ng, stages, tele in (("telescoping_rk2", 4, 2, True), ("ssp_rk3", 4, 3, False),
                                   ("telescoping_rk3", 6, 3, True)):
        lat = wl.lattice_3d(nb, nb, nb, 16, 16, 16, ng)
        h = gb.Hydro.from_lattice(lat)
        h.set_rk_stages(stages)
        h.set_telescoping(tele)
        U0 = wl.sedov(lat)
        U = torch.from_numpy(U0).cuda()

        def ms_per_step(n=5):
            V = torch.from_numpy(U0).cuda()
            d = h.compute_dt(V)
            h.step_cfl(V, d)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            e0.record()
            for _ in range(n):
                h.step_cfl(V, d)
            e1.record()
            barrier()
            del V
            return e0.elapsed_time(e1) / n

        rings = (0,) + ((2,) if tele else ()) + ((4,) if tele and stages == 3 else ())
        tuning = autotuned(h, U, rings, ms_per_step) if args.autotune else None
        dt = h.compute_dt(U)
        for _ in range(args.warmup):
            h.step_cfl(U, dt)
        h.set_kernel_timing(True)
        h.stage_kernel_time()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(args.variant_steps):
            h.step_cfl(U, dt)
        e1.record(stream)
        barrier()
        secs = e0.elapsed_time(e1) / 1e3
        stage_ms, _ = h.stage_kernel_time()
        h.set_kernel_timing(False)
        nbad = h.check_state(U)
        pre = h.face_prepass() and not tele      # the face pre-pass runs before halo-gathering stages
        h.close()
        del U
        torch.cuda.empty_cache()
        ms = 1e3 * secs / args.variant_steps
        out[name] = {"nguard": ng, "stages": stages, "telescoping": tele,
                     "value": lat.interior_cells * args.variant_steps / secs, "unit": UNIT,
                     "steps": args.variant_steps, "ms_per_step": ms,
                     "stage_kernels_ms_per_step": stage_ms / args.variant_steps,
                     "over_headline_step": ms / ms_headline,
                     "launches_per_step": stages + 1 + (1 if tele else 0) + (stages if pre else 0),
                     "unphysical_cells": nbad,
                     "autotune": tuning}
    out["workload"] = f"{WORKLOAD} -- stepper variants (nguard as listed)"
    return out


def run_two_level(args, gb, torch, barrier):
    """The two-level variant of the workload: 4096 coarse blocks (256^3) plus 4096
    fine blocks at half the cell width over the central eighth of the volume,
    one dt for both levels; zone-updates counted over leaf cells."""
    import workloads as wl
    nb = args.nb
    tl = wl.two_level(wl.lattice_3d(nb, nb, nb, 16, 16, 16, 4), (nb // 4,) * 3, (3 * nb // 4,) * 3)
    U0 = wl.sedov_two_level(tl)
    h = gb.Hydro.from_two_level(tl)
    U = torch.from_numpy(U0).cuda()
    h.fill_guardcells(U)
    dt = h.compute_dt(U)
    for _ in range(args.warmup):
        h.step_cfl(U, dt)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    h.advance(U, args.two_level_steps, dt)
    e1.record(stream)
    barrier()
    secs = e0.elapsed_time(e1) / 1e3
    nbad = h.check_state(U)
    # the same grid in the level-by-level telescoping variant
    h.set_telescoping(True)
    U.copy_(torch.from_numpy(U0))
    h.fill_guardcells(U)
    h.compute_dt(U, dt)
    for _ in range(args.warmup):
        h.step_cfl(U, dt)
    barrier()
    e0.record(stream)
    h.advance(U, args.two_level_steps, dt)
    e1.record(stream)
    barrier()
    tsecs = e0.elapsed_time(e1) / 1e3
    tbad = h.check_state(U)
    pre = 2 if h.face_prepass() else 0     # the face pre-pass of the two all-levels stages
    h.close()
    del U
    torch.cuda.empty_cache()
    return {"workload": f"{WORKLOAD} -- two-level variant: {tl.n0} coarse + {tl.n1} fine blocks, "
                        "restriction/prolongation in the guard fill, flux correction every stage",
            "value": tl.leaf_cells * args.two_level_steps / secs, "unit": UNIT, "zones": tl.leaf_cells,
            "steps": args.two_level_steps, "ms_per_step": 1e3 * secs / args.two_level_steps,
            "launches_per_step": 10 + pre, "unphysical_cells": nbad,
            "level_by_level_telescoping": {
                "value": tl.leaf_cells * args.two_level_steps / tsecs, "unit": UNIT,
                "ms_per_step": 1e3 * tsecs / args.two_level_steps, "launches_per_step": 9,
                "unphysical_cells": tbad}}


def run_ensemble(args, gb, torch, barrier):
    """Batched ensemble: 96 independent periodic 2-D problems of sizes drawn from
    {64^2, 128^2, 256^2, 512^2} in 16^2 blocks (Sod / Kelvin-Helmholtz with
    log-normal density noise), each with its own dt, advanced together as one
    CUDA graph of batched launches -- against one launch per problem per stage."""
    import numpy as np
    import workloads as wl
    probs = wl.ensemble(count=96, seed=0)
    lats = [l for l, _ in probs]
    zones = sum(l.interior_cells for l in lats)
    n = args.ensemble_steps
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        fn()
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / 1e3

    h = gb.Hydro.from_batch(lats)
    U0 = np.concatenate([u for _, u in probs])
    U = torch.from_numpy(U0).cuda()

    def default_ms():
        V = torch.from_numpy(U0).cuda()
        d = h.compute_dt(V)
        h.advance(V, 3, d)
        ms = timed(lambda: h.advance(V, 10, d)) * 1e3 / 10
        del V
        return ms

    tuning = autotuned(h, U, (0,), default_ms) if args.autotune else None
    kc, ipc = (tuning["chosen"]["kchunk"], tuning["chosen"]["items_per_cta"]) if tuning else (lat_kchunk(lats[0]), 1)
    dt = h.compute_dt(U)
    h.advance_graph(U, n, dt)          # capture + warm-up run
    U.copy_(torch.from_numpy(U0))
    h.compute_dt(U, dt)
    batched = timed(lambda: h.advance_graph(U, n, dt))
    h.close()
    del U
    # baseline: a context per problem, one launch per problem per stage
    ctxs = [(gb.Hydro.from_lattice(l), torch.from_numpy(u).cuda()) for l, u in probs]
    dts = [c.compute_dt(u) for c, u in ctxs]
    for (c, u), d in zip(ctxs, dts):
        c.step_cfl(u, d)
    def loop():
        for _ in range(n):
            for (c, u), d in zip(ctxs, dts):
                c.step_cfl(u, d)
    separate = timed(loop)
    for c, _ in ctxs:
        c.close()
    del ctxs
    torch.cuda.empty_cache()
    return {"workload": "96 independent periodic 2-D problems, sizes drawn from {64^2,128^2,256^2,512^2} "
                        "(seed 0) in 16^2 blocks + 4 guards, Sod / Kelvin-Helmholtz with log-normal density "
                        "noise (sigma 0.1, seeds 1000+i), own CFL dt each, FP64",
            "zones": zones, "blocks": sum(l.nblocks for l in lats), "steps": n,
            "batched_graph": {"value": zones * n / batched, "unit": UNIT, "ms_per_step": 1e3 * batched / n,
                              "launches_per_step": 3, "graph_launches": 1, "kchunk": kc, "items_per_cta": ipc,
                              "autotune": tuning},
            "one_launch_per_problem": {"value": zones * n / separate, "unit": UNIT,
                                       "ms_per_step": 1e3 * separate / n, "launches_per_step": 3 * len(lats)},
            "speedup": separate / batched}


def run_two_level_ensemble(args, gb, torch, barrier):
    """Batched two-level ensemble: 12 independent 3-D two-level Sedov problems of
    uneven sizes (coarse 4^3, 6^3 or 8^3 blocks of 16^3 cells drawn with seed 0,
    the central half refined), each with its own dt, advanced together as one
    CUDA graph of batched launches over both levels of all problems -- against
    a two-level context per problem."""
    import numpy as np
    import workloads as wl
    probs = wl.two_level_ensemble(count=12, seed=0)
    tls = [t for t, _ in probs]
    zones = sum(t.leaf_cells for t in tls)
    n = args.tl_ensemble_steps
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        fn()
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / 1e3

    h = gb.Hydro.from_two_level_batch(tls)
    U0 = np.concatenate([u for _, u in probs])
    U = torch.from_numpy(U0).cuda()
    h.fill_guardcells(U)
    dt = h.compute_dt(U)
    h.advance_graph(U, n, dt)          # capture + warm-up run
    U.copy_(torch.from_numpy(U0))
    h.fill_guardcells(U)
    h.compute_dt(U, dt)
    batched = timed(lambda: h.advance_graph(U, n, dt))
    nbad = h.check_state(U)
    pre = 2 if h.face_prepass() else 0     # the face pre-pass of the two stages
    h.close()
    del U
    torch.cuda.empty_cache()
    ctxs = [(gb.Hydro.from_two_level(t), torch.from_numpy(u).cuda()) for t, u in probs]
    dts = []
    for c, u in ctxs:
        c.fill_guardcells(u)
        dts.append(c.compute_dt(u))
    for (c, u), d in zip(ctxs, dts):
        c.step_cfl(u, d)
    def loop():
        for _ in range(n):
            for (c, u), d in zip(ctxs, dts):
                c.step_cfl(u, d)
    separate = timed(loop)
    for c, _ in ctxs:
        c.close()
    del ctxs
    torch.cuda.empty_cache()
    return {"workload": "12 independent 3-D two-level Sedov problems, coarse 4^3/6^3/8^3 blocks (seed 0) of "
                        "16^3 cells + 4 guards, central half refined, own CFL dt each, FP64",
            "zones": zones, "blocks": sum(t.nblocks for t in tls), "steps": n,
            "batched_graph": {"value": zones * n / batched, "unit": UNIT, "ms_per_step": 1e3 * batched / n,
                              "launches_per_step": 10 + pre, "graph_launches": 1, "unphysical_cells": nbad},
            "one_context_per_problem": {"value": zones * n / separate, "unit": UNIT,
                                        "ms_per_step": 1e3 * separate / n,
                                        "launches_per_step": (10 + pre) * len(tls)},
            "speedup": separate / batched}


def run_adjoint(args, gb, torch, barrier):
    """Gradient workload: 2-D Sod-like 256^2 in 16^2 blocks, 50 steps, checkpoint
    every 10; forward (with checkpoints) and adjoint sweep timed separately."""
    import numpy as np
    import workloads as wl
    from paper_2401_03378_gb300.adjoint import CheckpointedRun
    lat = wl.lattice_2d(16, 16, 16, 16, 4)
    n = args.adjoint_steps
    h = gb.Hydro.from_lattice(lat)
    U0 = torch.from_numpy(wl.sod_smooth(lat)).cuda()
    rng = np.random.default_rng(7)
    lam = torch.from_numpy(rng.standard_normal(lat.shape)).cuda()
    run = CheckpointedRun(h, n, every=10)
    run.forward(U0)
    run.backward(lam)           # warm-up (allocates the adjoint buffers)
    stream = torch.cuda.current_stream()
    times = []
    for fn in (lambda: run.forward(U0), lambda: run.backward(lam)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        fn()
        e1.record(stream)
        barrier()
        times.append(e0.elapsed_time(e1))
    h.close()
    return {"workload": "2-D Sod-like (tanh-smoothed jump, smooth 2-D modulations) 256^2 in 16^2 blocks + 4 guards, "
                        f"{n} steps, checkpoint every 10, dt held fixed, FP64",
            "forward_ms": times[0], "adjoint_ms": times[1], "adjoint_over_forward": times[1] / times[0],
            "target_ratio": 4.0}


def oracle_step_rate(lat, U0, nsteps, threads=0):
    """Time `nsteps` oracle SSP-RK2 steps (dt from the oracle) on the host cores."""
    from oracle import oracle as orc
    used = orc.set_threads(threads)
    o = orc.Oracle(lat)
    U = U0.copy()
    t0 = time.perf_counter()
    for _ in range(nsteps):
        dt = o.compute_dt(U)
        o.step(U, dt)
    secs = time.perf_counter() - t0
    return lat.interior_cells * nsteps / secs, used, secs


def cpu_baseline(args, U0, lat):
    rate, used, secs = oracle_step_rate(lat, U0, args.cpu_steps)
    # the same oracle on one thread, on the 128^3 lattice of the same workload
    import workloads as wl
    lat1 = wl.lattice_3d(8, 8, 8, 16, 16, 16, 4)
    rate1, _, secs1 = oracle_step_rate(lat1, wl.sedov(lat1), 1, threads=1)
    from oracle import oracle as orc
    orc.set_threads(0)
    return {"value": rate, "unit": UNIT, "cores": used, "cpu_model": host_cpu_model(), "kind": "oracle",
            "sample": f"{args.cpu_steps} oracle SSP-RK2 step(s) of the full 256^3 workload "
                      f"({secs:.1f} s, OpenMP over blocks, {used} threads)",
            "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                              "sample": f"1 oracle step of the 128^3 Sedov lattice on 1 thread ({secs1:.1f} s)"}}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    lat, U0 = make_problem(args.nb)
    from oracle import oracle as orc
    used = orc.set_threads(0)
    o = orc.Oracle(lat)
    U = U0.copy()
    for _ in range(args.warmup):
        o.step(U, o.compute_dt(U))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(U, o.compute_dt(U))
    secs = time.perf_counter() - t0
    value = lat.interior_cells * args.steps / secs
    sample = (f"{args.steps} oracle SSP-RK2 step(s) of the {lat.global_cells[0]}^3 Sedov lattice "
              f"({lat.nblocks} blocks of 16^3), OpenMP over blocks, {used} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Sedov initial condition)",
        "config": bench_config(lat),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "cpu_model": host_cpu_model(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gbhydro", "reference"], default="gbhydro")
    ap.add_argument("--nb", type=int, default=16, help="blocks per dimension (16 -> 256^3)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--two-level-steps", type=int, default=20)
    ap.add_argument("--ensemble-steps", type=int, default=100)
    ap.add_argument("--tl-ensemble-steps", type=int, default=10)
    ap.add_argument("--adjoint-steps", type=int, default=50)
    ap.add_argument("--variant-steps", type=int, default=10)
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--no-repeats", dest="repeats", action="store_false",
                    help="skip the 5 x 10-step repeats after the timed loop")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="time the default decompositions without running the autotuner first "
                         "(profiling runs: no trial launches before the captured ones)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        log("note: at least 3 warm-up steps are required; using 3")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
