"""Build libgbhydro.so in-tree with nvcc for sm_103a (GB300).

Each .cu translation unit is compiled in parallel to an object file under
paper_2401_03378_gb300/_build/, then linked into
paper_2401_03378_gb300/libgbhydro.so (static CUDA runtime, C ABI only).
The same sources compiled with -DGBH_CHECK (objects under _build/check/)
give libgbhydro_check.so, the checked build whose kernels count and
redirect out-of-range indices (gbh_check.cuh).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgbhydro.so")
SOURCES = ["gbh_abi.cu", "gbh_stage.cu", "gbh_aux.cu", "gbh_static.cu", "gbh_amr.cu", "gbh_adjoint.cu"]
HEADERS = ["gbh_internal.h", "gbh_device.cuh", "gbh_fastmath.cuh", "gbh_gather.cuh", "gbh_check.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    out = [os.path.join(CSRC, h) for h in HEADERS]
    out.append(os.path.join(ROOT, "include", "gbhydro.h"))
    return out


def _stale(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


LIB_CHECK = os.path.join(HERE, "libgbhydro_check.so")
VARIANTS = ((LIB, BUILD, []), (LIB_CHECK, os.path.join(BUILD, "check"), ["-DGBH_CHECK"]))


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Build both libraries (nvcc processes in parallel); returns the normal one's path."""
    cc = nvcc()
    deps = _deps()
    procs, links = [], []
    for lib, bdir, defs in VARIANTS:
        os.makedirs(bdir, exist_ok=True)
        objs = []
        for src in SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(bdir, src.replace(".cu", ".o"))
            objs.append(o)
            if force or _stale(o, [s] + deps):
                cmd = [cc, *ARCH, *NVCC_FLAGS, *defs, "-I", os.path.join(ROOT, "include"), "-c", s, "-o", o]
                if verbose_ptxas and not defs:
                    cmd += ["-Xptxas", "-v"]
                procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        links.append((lib, objs))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((src, text))
        elif verbose_ptxas and text:
            sys.stdout.write(f"--- {src}\n{text}")
    if failed:
        msg = "\n".join(f"--- {s}\n{t}" for s, t in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    for lib, objs in links:
        if force or _stale(lib, objs):
            tmp = lib + ".tmp"
            subprocess.run([cc, *ARCH, "-shared", *objs, "-o", tmp], check=True)
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    path = build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(path)
