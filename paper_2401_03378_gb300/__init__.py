"""GB300-native FP64 block-structured Euler update (guard fill, MC-limited
PLM, HLLC, SSP-RK2, CFL dt) behind the C ABI of libgbhydro.so.

The hydrodynamics hot path of the Flash-X Spark variants the paper generates
(Sec. 4.2).  ``Hydro`` marshals PyTorch CUDA tensors to the C ABI declared in
include/gbhydro.h; nothing is computed in Python and there is no CPU fallback.
"""
from ._abi import GbhError, load  # noqa: F401
from .grid import neighbour_table, uniform_widths  # noqa: F401


def __getattr__(name):
    # torch-dependent binding is imported on first use
    if name in ("Hydro", "fp64_probe", "sm_count"):
        from . import hydro
        return getattr(hydro, name)
    raise AttributeError(name)
