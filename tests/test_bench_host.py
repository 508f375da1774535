"""Host-side logic of bench.py: the multi-rank aggregation (gloo, 2 ranks on
the CPU), the reference arm's rank handling, and the clock-sample parser."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate(1.0 + rank, 10.0 * (rank + 1), world)
    q.put((rank, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u in out:
        assert t == 2.0            # slowest rank's clock
        assert u == 30.0           # all ranks' work


def test_reference_arm_nonzero_rank_is_silent():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--nb", "2"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--nb", "2"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_clock_sampler_summary(tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    p = tmp_path / "c.csv"
    p.write_text("0, 2070, 2070, 250.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 1980, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, 2070, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = bench.ClockSampler(0)
    s.path = str(p)
    out = s.summary()
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3


def test_fp64_issue_rate_and_ncu_record():
    sys.path.insert(0, ROOT)
    import bench
    # 401.6 instructions per zone over 16.8 M zones in 11.01 ms at 2070 MHz on 152 SMs
    r = bench.fp64_issue(401.6 * 256 ** 3, 11.01, 2070.0, 152)
    assert abs(r["lanes_per_sm_clock"] - 401.6 * 256 ** 3 / (11.01e-3 * 2070e6 * 152)) < 1e-12
    assert abs(r["of_peak_lanes"] - r["lanes_per_sm_clock"] / 2) < 1e-15
    assert bench.fp64_issue(1e9, 1.0, None, 152)["sm_mhz_source"].startswith("nominal")
    assert bench.fp64_issue(None, 1.0, 2070.0, 152) is None
    # the committed ncu record counts only while it belongs to the current kernel source
    rec = json.load(open(os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")))
    z = 256 ** 3
    if rec["source_hash"] == bench.source_hash():
        assert bench.measured_fp64_inst(z) == 0.5 * (rec["fp64_inst_per_zone_stage1"]
                                                     + rec["fp64_inst_per_zone_stage2"]) * z
        assert bench.measured_traffic(z) == rec["dram_bytes_per_launch"] / rec["zones"] * z
    else:
        assert bench.measured_fp64_inst(z) is None and bench.measured_traffic(z) is None
