"""ctypes declarations of the C ABI in include/gbhydro.h (marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbhydro.so")

GBH_OK = 0
GBH_ERR_INVAL = -1
GBH_ERR_CUDA = -2
GBH_ERR_UNPHYSICAL = -3
GBH_ERR_NOMEM = -4
GBH_ERR_UNSUPPORTED = -5
GBH_BC_OUTFLOW = -1
GBH_NBR_COARSER = -2

ERROR_NAMES = {
    GBH_ERR_INVAL: "GBH_ERR_INVAL",
    GBH_ERR_CUDA: "GBH_ERR_CUDA",
    GBH_ERR_UNPHYSICAL: "GBH_ERR_UNPHYSICAL",
    GBH_ERR_NOMEM: "GBH_ERR_NOMEM",
    GBH_ERR_UNSUPPORTED: "GBH_ERR_UNSUPPORTED",
}


class GbhParams(C.Structure):
    _fields_ = [
        ("ndim", C.c_int),
        ("nxb", C.c_int),
        ("nyb", C.c_int),
        ("nzb", C.c_int),
        ("nguard", C.c_int),
        ("nblocks", C.c_int),
        ("gamma", C.c_double),
        ("cfl", C.c_double),
        ("small_rho", C.c_double),
        ("small_p", C.c_double),
        ("nbr", C.POINTER(C.c_int32)),
        ("dx", C.POINTER(C.c_double)),
    ]


class GbhRefinement(C.Structure):
    _fields_ = [("parent", C.POINTER(C.c_int32)), ("children", C.POINTER(C.c_int32))]


# name -> (restype, argtypes); the exported symbols of libgbhydro.so
_vp = C.c_void_p
_dp = C.c_void_p          # device or host double* passed as an address
SIGNATURES = {
    "gbh_create": (C.c_int, [C.POINTER(GbhParams), C.POINTER(_vp)]),
    "gbh_create_refined": (C.c_int, [C.POINTER(GbhParams), C.POINTER(GbhRefinement), C.POINTER(_vp)]),
    "gbh_create_batched": (C.c_int, [C.POINTER(GbhParams), C.POINTER(C.c_int32), C.c_int, C.POINTER(_vp)]),
    "gbh_create_refined_batched": (C.c_int, [C.POINTER(GbhParams), C.POINTER(GbhRefinement), C.POINTER(C.c_int32),
                                             C.c_int, C.POINTER(_vp)]),
    "gbh_autotune": (C.c_int, [_vp, _dp, C.POINTER(C.c_int), C.POINTER(C.c_int), _vp]),
    "gbh_set_decomposition": (C.c_int, [_vp, C.c_int, C.c_int]),
    "gbh_set_tile_split": (C.c_int, [_vp, C.c_int, C.c_int]),
    "gbh_get_tile_split": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int)]),
    "gbh_set_telescoping": (C.c_int, [_vp, C.c_int]),
    "gbh_set_rk_stages": (C.c_int, [_vp, C.c_int]),
    "gbh_set_prim_carry": (C.c_int, [_vp, C.c_int]),
    "gbh_get_prim_carry": (C.c_int, [_vp, C.POINTER(C.c_int)]),
    "gbh_set_face_prepass": (C.c_int, [_vp, C.c_int]),
    "gbh_get_face_prepass": (C.c_int, [_vp, C.POINTER(C.c_int)]),
    "hydro_advance_graph": (C.c_int, [_vp, _dp, C.c_int, _dp, _vp]),
    "hydro_stage_vjp": (C.c_int, [_vp, _dp, _dp, C.c_double, _dp, C.c_double, _dp, C.c_double, _dp, _vp]),
    "hydro_step_adjoint": (C.c_int, [_vp, _dp, C.c_double, _dp, _dp, _vp]),
    "hydro_step_adjoint_stored": (C.c_int, [_vp, _dp, _dp, C.c_double, _dp, _dp, _vp]),
    "hydro_prim_to_cons": (C.c_int, [_vp, _dp, _dp, _vp]),
    "hydro_prim_to_cons_vjp": (C.c_int, [_vp, _dp, _dp, _dp, _vp]),
    "gbh_destroy": (C.c_int, [_vp]),
    "gbh_last_error": (C.c_char_p, [_vp]),
    "gbh_state_bytes": (C.c_longlong, [_vp]),
    "hydro_fill_guardcells": (C.c_int, [_vp, _dp, _vp]),
    "hydro_compute_dt": (C.c_int, [_vp, _dp, _dp, _vp]),
    "hydro_stage": (C.c_int, [_vp, _dp, _dp, _dp, C.c_double, C.c_double, C.c_double, _vp]),
    "hydro_stage_guarded": (C.c_int, [_vp, _dp, _dp, _dp, C.c_double, C.c_double, C.c_double, _vp]),
    "hydro_step": (C.c_int, [_vp, _dp, C.c_double, _vp]),
    "hydro_step_static": (C.c_int, [C.POINTER(GbhParams), _dp, C.c_double, _vp]),
    "hydro_step_cfl": (C.c_int, [_vp, _dp, _dp, _vp]),
    "hydro_advance": (C.c_int, [_vp, _dp, C.c_int, _dp, _dp, _vp]),
    "hydro_advance_host": (C.c_int, [_vp, _dp, C.c_int, _dp, _vp]),
    "hydro_advance_host_interior": (C.c_int, [_vp, _dp, C.c_int, _dp, _vp]),
    "hydro_step_host": (C.c_int, [_vp, _dp, _dp, _vp]),
    "hydro_step_host_interior": (C.c_int, [_vp, _dp, _dp, _vp]),
    "gbh_set_host_pipeline": (C.c_int, [_vp, C.c_int]),
    "hydro_check_state": (C.c_int, [_vp, _dp, C.POINTER(C.c_longlong), _vp]),
    "hydro_floor_hits": (C.c_int, [_vp, C.POINTER(C.c_longlong), _vp]),
    "gbh_set_kernel_timing": (C.c_int, [_vp, C.c_int]),
    "gbh_stage_kernel_time": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong), _vp]),
    "gbh_fp64_probe": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _vp]),
    "gbh_op_count_probe": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, _dp, _vp]),
    "gbh_fastmath_selftest": (C.c_int, [_dp, _dp, C.c_longlong, _vp]),
    "gbh_bits_selftest": (C.c_int, [_dp, _dp, _dp, C.c_longlong, _vp]),
    "gbh_device_sm_count": (C.c_int, []),
    "gbh_check_violations": (C.c_int, [C.POINTER(C.c_longlong)]),
    "gbh_check_selftest": (C.c_int, [C.POINTER(C.c_longlong)]),
}

LIB_PATH_CHECK = os.path.join(HERE, "libgbhydro_check.so")

_lock = threading.Lock()
_libs = {}


class GbhError(RuntimeError):
    def __init__(self, code: int, msg: str):
        self.code = code
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")


def load(path: str | None = None, checked: bool = False):
    """Load libgbhydro.so (or, checked=True, the checked build
    libgbhydro_check.so), built in-tree.  Raises if it is missing: there is
    no fallback implementation."""
    p = path or (LIB_PATH_CHECK if checked else LIB_PATH)
    with _lock:
        if p not in _libs:
            if not os.path.exists(p):
                raise RuntimeError(
                    f"{p} is missing: build it with `python -m paper_2401_03378_gb300.build` "
                    "(there is no CPU fallback)")
            lib = C.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _libs[p] = lib
        return _libs[p]
