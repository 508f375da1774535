"""Compile the C++ oracle into oracle/liboracle.so and the op counter.

TEST INFRASTRUCTURE: builds the checker only.  Plain g++, -O2, no fused
multiply-add (-ffp-contract=off) so that the oracle's arithmetic is exactly
the order written in oracle_pointwise.h; OpenMP over blocks only.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
OPCOUNT = os.path.join(HERE, "opcount")
CXXFLAGS = ["-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wextra"]


def _stale(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def build(force: bool = False, verbose: bool = False):
    """Return the list of Popen handles started (callers may run this in parallel)."""
    hdr = os.path.join(HERE, "oracle_pointwise.h")
    lib_src = os.path.join(HERE, "hydro_oracle.cpp")
    cnt_src = os.path.join(HERE, "opcount.cpp")
    jobs = []
    if force or _stale(LIB, [lib_src, hdr]):
        cmd = ["g++", *CXXFLAGS, "-fopenmp", "-shared", "-fPIC", lib_src, "-o", LIB + ".tmp"]
        jobs.append((subprocess.Popen(cmd), LIB))
    if force or _stale(OPCOUNT, [cnt_src, hdr]):
        cmd = ["g++", *CXXFLAGS, cnt_src, "-o", OPCOUNT + ".tmp"]
        jobs.append((subprocess.Popen(cmd), OPCOUNT))
    return jobs


def finish(jobs):
    for proc, target in jobs:
        if proc.wait() != 0:
            raise RuntimeError(f"oracle build failed for {target}")
        os.replace(target + ".tmp", target)


def main():
    finish(build(force="--force" in sys.argv))


if __name__ == "__main__":
    main()
