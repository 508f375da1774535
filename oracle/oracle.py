"""ctypes harness of the FP64 CPU oracle (oracle/hydro_oracle.cpp).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs import this module.  It takes numpy arrays in
the block layout U[nblk][5][nz][ny][nx] and a ``workloads.Lattice``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None


class OrcAmr2(C.Structure):
    _fields_ = [("lo", C.c_int * 3), ("hi", C.c_int * 3), ("refined", C.c_void_p)]


class OrcGrid(C.Structure):
    _fields_ = [
        ("ndim", C.c_int),
        ("nb", C.c_int * 3),
        ("n", C.c_int * 3),
        ("ng", C.c_int),
        ("periodic", C.c_int * 3),
        ("dx", C.c_double * 3),
        ("gamma", C.c_double),
        ("cfl", C.c_double),
        ("small_rho", C.c_double),
        ("small_p", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            from . import build_oracle
            build_oracle.finish(build_oracle.build())
            L = C.CDLL(build_oracle.LIB)
            dp = C.POINTER(C.c_double)
            gp = C.POINTER(OrcGrid)
            L.orc_num_threads.argtypes = [C.c_int]
            L.orc_num_threads.restype = C.c_int
            L.orc_prim.argtypes = [dp, C.c_double, C.c_double, C.c_double, dp]
            L.orc_prim.restype = C.c_int
            L.orc_mc_slope.argtypes = [C.c_double] * 3
            L.orc_mc_slope.restype = C.c_double
            L.orc_euler_flux.argtypes = [dp, C.c_double, dp]
            L.orc_euler_flux.restype = None
            L.orc_hllc.argtypes = [dp, dp, C.c_double, dp, dp]
            L.orc_hllc.restype = None
            L.orc_fill_guardcells.argtypes = [gp, dp]
            L.orc_fill_guardcells.restype = None
            L.orc_compute_dt.argtypes = [gp, dp]
            L.orc_compute_dt.restype = C.c_double
            L.orc_stage.argtypes = [gp, dp, dp, dp, C.c_double, C.c_double, C.c_double,
                                    C.POINTER(C.c_longlong), C.c_longlong]
            L.orc_stage.restype = C.c_longlong
            L.orc_stage_ext.argtypes = [gp, dp, dp, dp, C.c_double, C.c_double, C.c_double, C.c_int]
            L.orc_stage_ext.restype = C.c_longlong
            L.orc_step.argtypes = [gp, dp, C.c_double]
            L.orc_step.restype = C.c_longlong
            L.orc_step_telescoping.argtypes = [gp, dp, C.c_double]
            L.orc_step_telescoping.restype = C.c_longlong
            L.orc_step_rk.argtypes = [gp, dp, C.c_double, C.c_int, C.c_int]
            L.orc_step_rk.restype = C.c_longlong
            L.orc_run.argtypes = [gp, dp, C.c_int, dp, C.c_int, C.c_int]
            L.orc_run.restype = C.c_longlong
            L.orc_stage_vjp.argtypes = [gp, dp, dp, C.c_double, dp]
            L.orc_stage_vjp.restype = None
            L.orc_step_adjoint.argtypes = [gp, dp, C.c_double, dp, dp]
            L.orc_step_adjoint.restype = None
            L.orc_step_adjoint_rk.argtypes = [gp, dp, C.c_double, dp, dp, C.c_int]
            L.orc_step_adjoint_rk.restype = C.c_int
            L.orc_step_adjoint_telescoping.argtypes = [gp, dp, C.c_double, dp, dp, C.c_int]
            L.orc_step_adjoint_telescoping.restype = C.c_int
            ap = C.POINTER(OrcAmr2)
            L.orc2_restrict.argtypes = [gp, ap, dp]
            L.orc2_restrict.restype = None
            L.orc2_fill.argtypes = [gp, ap, dp]
            L.orc2_fill.restype = None
            L.orc2_compute_dt.argtypes = [gp, ap, dp]
            L.orc2_compute_dt.restype = C.c_double
            L.orc2_step.argtypes = [gp, ap, dp, C.c_double]
            L.orc2_step.restype = C.c_longlong
            L.orc2_stage.argtypes = [gp, ap, dp, dp, dp, C.c_double, C.c_double, C.c_double, C.c_int]
            L.orc2_stage.restype = C.c_longlong
            L.orc2_step_telescoping.argtypes = [gp, ap, dp, C.c_double]
            L.orc2_step_telescoping.restype = C.c_longlong
            L.orc2_step_rk.argtypes = [gp, ap, dp, C.c_double, C.c_int, C.c_int]
            L.orc2_step_rk.restype = C.c_longlong
            L.orc2_run.argtypes = [gp, ap, dp, C.c_int, dp, C.c_int, C.c_int]
            L.orc2_run.restype = C.c_longlong
            _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(U, lat):
    if U.shape != lat.shape:
        raise ValueError(f"U shape {U.shape} != lattice shape {lat.shape}")
    if U.dtype != np.float64 or not U.flags.c_contiguous:
        raise ValueError("U must be C-contiguous float64")


def grid(lat, gamma=1.4, cfl=0.8, small_rho=1e-12, small_p=1e-14):
    g = OrcGrid()
    g.ndim = lat.ndim
    for d in range(3):
        g.nb[d] = lat.nb[d]
        g.n[d] = lat.n[d]
        g.periodic[d] = 1 if lat.bc[d] == "periodic" else 0
        g.dx[d] = lat.dx[d]
    g.ng = lat.ng
    g.gamma, g.cfl, g.small_rho, g.small_p = gamma, cfl, small_rho, small_p
    return g


def set_threads(n: int) -> int:
    return lib().orc_num_threads(int(n))


class Oracle:
    """The oracle bound to one lattice and one set of parameters."""

    def __init__(self, lat, gamma=1.4, cfl=0.8, small_rho=1e-12, small_p=1e-14):
        self.lat = lat
        self.g = grid(lat, gamma, cfl, small_rho, small_p)
        self.L = lib()

    def fill_guardcells(self, U):
        _check(U, self.lat)
        self.L.orc_fill_guardcells(C.byref(self.g), _dp(U))
        return U

    def compute_dt(self, U):
        _check(U, self.lat)
        return float(self.L.orc_compute_dt(C.byref(self.g), _dp(U)))

    def stage(self, Uin, Un, Uout, dt, a, b, blocks=None, ext=0):
        """Uout = a Un + b (Uin + dt L(Uin)) on the interior (widened by ext
        cells per side); Uin's guards must be filled."""
        _check(Uin, self.lat)
        _check(Uout, self.lat)
        if Un is not None:
            _check(Un, self.lat)
        if ext:
            if blocks is not None:
                raise ValueError("ext and blocks are exclusive")
            hits = int(self.L.orc_stage_ext(C.byref(self.g), _dp(Uin), _dp(Un), _dp(Uout), dt, a, b, int(ext)))
            if hits < 0:
                raise ValueError("invalid ring width for the guard width")
            return hits
        lst, nl = None, 0
        if blocks is not None:
            arr = np.ascontiguousarray(np.asarray(blocks, dtype=np.int64))
            lst, nl = arr.ctypes.data_as(C.POINTER(C.c_longlong)), len(arr)
            self._keep = arr
        return int(self.L.orc_stage(C.byref(self.g), _dp(Uin), _dp(Un), _dp(Uout), dt, a, b, lst, nl))

    def step(self, U, dt, telescoping=False, stages=2):
        """One SSP-RK step in place (stages 2 or 3); telescoping=True: one guard
        fill per step and earlier stages that also update a ring of guard cells
        (needs ng >= 2 * stages)."""
        _check(U, self.lat)
        if stages == 2 and not telescoping:
            return int(self.L.orc_step(C.byref(self.g), _dp(U), float(dt)))
        hits = int(self.L.orc_step_rk(C.byref(self.g), _dp(U), float(dt), int(stages), int(bool(telescoping))))
        if hits < 0:
            raise ValueError("stages must be 2 or 3; the telescoping mode needs 2 * stages guard cells")
        return hits

    def stage_vjp(self, U, M, scale):
        """J_L(U)^T (scale M) on interior cells (dt held fixed, branches frozen)."""
        _check(U, self.lat)
        _check(M, self.lat)
        out = np.zeros_like(U)
        self.L.orc_stage_vjp(C.byref(self.g), _dp(U), _dp(M), float(scale), _dp(out))
        return out

    def step_adjoint(self, Un, dt, lam_next, stages=2, telescoping=False):
        """dJ/dU^n of one step(Un, dt, stages=stages, telescoping=telescoping)
        from dJ/dU^{n+1} (interior cells)."""
        _check(Un, self.lat)
        _check(lam_next, self.lat)
        out = np.zeros_like(Un)
        if telescoping:
            if self.L.orc_step_adjoint_telescoping(C.byref(self.g), _dp(Un), float(dt), _dp(lam_next), _dp(out),
                                                   int(stages)) != 0:
                raise ValueError("stages must be 2 or 3, with at least 2 * stages guard cells")
        elif stages == 2:
            self.L.orc_step_adjoint(C.byref(self.g), _dp(Un), float(dt), _dp(lam_next), _dp(out))
        elif self.L.orc_step_adjoint_rk(C.byref(self.g), _dp(Un), float(dt), _dp(lam_next), _dp(out),
                                        int(stages)) != 0:
            raise ValueError("stages must be 2 or 3")
        return out

    def run(self, U, nsteps, telescoping=False, stages=2):
        """Advance U in place by nsteps; returns (dt history, floor hits)."""
        _check(U, self.lat)
        hist = np.zeros(max(nsteps, 1))
        hits = int(self.L.orc_run(C.byref(self.g), _dp(U), int(nsteps), _dp(hist), int(bool(telescoping)),
                                  int(stages)))
        if hits < 0:
            raise ValueError("stages must be 2 or 3; the telescoping mode needs 2 * stages guard cells")
        return hist[:nsteps], hits


class Oracle2:
    """The oracle on a two-level composite grid (workloads.TwoLevel).  Its
    arrays hold the coarse lattice, then the fine lattice over the bounding box
    of the refined blocks, including the slots of fine blocks that do not exist
    (their parent is not refined), which it neither reads nor writes."""

    def __init__(self, tl, gamma=1.4, cfl=0.8, small_rho=1e-12, small_p=1e-14):
        self.tl = tl
        self.g = grid(tl.coarse, gamma, cfl, small_rho, small_p)
        self.r = OrcAmr2()
        for d in range(3):
            self.r.lo[d] = tl.lo[d]
            self.r.hi[d] = tl.hi[d]
        # the refined coarse blocks (all of the box when the grid names none)
        self._mask = np.ascontiguousarray(tl.refined_mask(), dtype=np.uint8)
        self.r.refined = self._mask.ctypes.data
        self.L = lib()

    def _chk(self, U):
        if U.shape != self.tl.shape or U.dtype != np.float64 or not U.flags.c_contiguous:
            raise ValueError(f"U must be C-contiguous float64 of shape {self.tl.shape}")

    def restrict(self, U):
        self._chk(U)
        self.L.orc2_restrict(C.byref(self.g), C.byref(self.r), _dp(U))
        return U

    def fill(self, U):
        """restriction, coarse guard fill, fine guard fill (copies + prolongation)"""
        self._chk(U)
        self.L.orc2_fill(C.byref(self.g), C.byref(self.r), _dp(U))
        return U

    def compute_dt(self, U):
        self._chk(U)
        return float(self.L.orc2_compute_dt(C.byref(self.g), C.byref(self.r), _dp(U)))

    def stage(self, Uin, Un, Uout, dt, a, b, reflux=True):
        for X in (Uin, Uout) + ((Un,) if Un is not None else ()):
            self._chk(X)
        return int(self.L.orc2_stage(C.byref(self.g), C.byref(self.r), _dp(Uin), _dp(Un), _dp(Uout),
                                     dt, a, b, 1 if reflux else 0))

    def step(self, U, dt, telescoping=False, stages=2):
        """One step: all-levels non-telescoping (default), or level-by-level
        telescoping (one fill, every stage per block, correction at the end)."""
        self._chk(U)
        if stages == 2 and not telescoping:
            return int(self.L.orc2_step(C.byref(self.g), C.byref(self.r), _dp(U), float(dt)))
        hits = int(self.L.orc2_step_rk(C.byref(self.g), C.byref(self.r), _dp(U), float(dt), int(stages),
                                       int(bool(telescoping))))
        if hits < 0:
            raise ValueError("stages must be 2 or 3; the telescoping mode needs 2 * stages guard cells")
        return hits

    def run(self, U, nsteps, telescoping=False, stages=2):
        self._chk(U)
        hist = np.zeros(max(nsteps, 1))
        hits = int(self.L.orc2_run(C.byref(self.g), C.byref(self.r), _dp(U), int(nsteps), _dp(hist),
                                   int(bool(telescoping)), int(stages)))
        if hits < 0:
            raise ValueError("stages must be 2 or 3; the telescoping mode needs 2 * stages guard cells")
        return hist[:nsteps], hits


# ---------------------------------------------------------------------------
# pointwise entry points (for the pin tests)
# ---------------------------------------------------------------------------

def prim(U5, gamma=1.4, small_rho=1e-12, small_p=1e-14):
    u = np.ascontiguousarray(U5, dtype=np.float64)
    w = np.zeros(5)
    hit = lib().orc_prim(_dp(u), gamma, small_rho, small_p, _dp(w))
    return w, hit


def mc_slope(qm, q0, qp):
    return float(lib().orc_mc_slope(qm, q0, qp))


def euler_flux(W5, gamma=1.4):
    w = np.ascontiguousarray(W5, dtype=np.float64)
    f = np.zeros(5)
    lib().orc_euler_flux(_dp(w), gamma, _dp(f))
    return f


_DETAIL_KEYS = ["UL", "UR", "FL", "FR", "UsL", "UsR", "FsL", "FsR", "F"]


def hllc(WL, WR, gamma=1.4, detail=False):
    """HLLC flux with the normal along the first velocity component."""
    wl = np.ascontiguousarray(WL, dtype=np.float64)
    wr = np.ascontiguousarray(WR, dtype=np.float64)
    f = np.zeros(5)
    if not detail:
        lib().orc_hllc(_dp(wl), _dp(wr), gamma, _dp(f), None)
        return f
    d = np.zeros(4 + 5 * len(_DETAIL_KEYS))
    lib().orc_hllc(_dp(wl), _dp(wr), gamma, _dp(f), _dp(d))
    out = {"SL": d[0], "SR": d[1], "Ss": d[2], "region": int(d[3])}
    for i, k in enumerate(_DETAIL_KEYS):
        out[k] = d[4 + 5 * i: 9 + 5 * i].copy()
    return f, out
