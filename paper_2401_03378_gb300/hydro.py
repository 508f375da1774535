"""Thin Python binding of libgbhydro.so for PyTorch CUDA tensors.

Argument marshalling only: every step of the update runs in the library's
CUDA kernels.  Tensors are float64, C-contiguous, on the context's CUDA
device, shaped (nblocks, 5, nz_pad, ny_pad, nx_pad); work is enqueued on
torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _abi
from .grid import neighbour_table, uniform_widths


def _stream_handle() -> int:
    return torch.cuda.current_stream().cuda_stream


class Hydro:
    """One block-structured Euler problem bound to the current CUDA device.

    Parameters mirror ``gbh_params``: block sizes, guard width, gamma, CFL
    number, floors, and either an explicit neighbour table / cell widths or a
    rectangular lattice (``nb`` blocks per dimension, ``periodic`` flags,
    domain ``extent``) from which they are built.
    """

    def __init__(self, ndim: int, n: Sequence[int], nguard: int = 4, *,
                 nb: Optional[Sequence[int]] = None, periodic=(False, False, False),
                 extent=(1.0, 1.0, 1.0), nbr: Optional[np.ndarray] = None,
                 dx: Optional[np.ndarray] = None, gamma: float = 1.4, cfl: float = 0.8,
                 small_rho: float = 1e-12, small_p: float = 1e-14,
                 parent: Optional[np.ndarray] = None, children: Optional[np.ndarray] = None,
                 problem: Optional[np.ndarray] = None, nproblems: int = 1, checked: bool = False):
        self.lib = _abi.load(checked=checked)
        self.ndim = int(ndim)
        nx, ny, nz = (int(n[0]), int(n[1]), int(n[2]) if ndim == 3 else 1)
        if nbr is None:
            if nb is None:
                raise ValueError("give either nbr/dx tables or a lattice (nb)")
            nbr = neighbour_table(ndim, nb, periodic)
            nblk = nbr.shape[0]
            cells = (nb[0] * nx, nb[1] * ny, (nb[2] if ndim == 3 else 1) * nz)
            dx = uniform_widths(nblk, [extent[d] / cells[d] for d in range(3)])
        self.nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        self.dx = np.ascontiguousarray(dx, dtype=np.float64)
        self.nblocks = int(self.nbr.shape[0])
        self.n = (nx, ny, nz)
        self.nguard = int(nguard)
        gz = self.nguard if ndim == 3 else 0
        self.shape = (self.nblocks, 5, nz + 2 * gz, ny + 2 * self.nguard, nx + 2 * self.nguard)
        self.interior_shape = (self.nblocks, 5, nz, ny, nx)
        p = _abi.GbhParams()
        p.ndim, p.nxb, p.nyb, p.nzb = self.ndim, nx, ny, nz
        p.nguard, p.nblocks = self.nguard, self.nblocks
        p.gamma, p.cfl, p.small_rho, p.small_p = gamma, cfl, small_rho, small_p
        p.nbr = self.nbr.ctypes.data_as(C.POINTER(C.c_int32))
        p.dx = self.dx.ctypes.data_as(C.POINTER(C.c_double))
        ctx = C.c_void_p()
        self.refined = parent is not None
        self.nproblems = int(nproblems) if problem is not None else 1
        if self.refined:
            self.parent = np.ascontiguousarray(parent, dtype=np.int32)
            self.children = np.ascontiguousarray(children, dtype=np.int32)
            r = _abi.GbhRefinement()
            r.parent = self.parent.ctypes.data_as(C.POINTER(C.c_int32))
            r.children = self.children.ctypes.data_as(C.POINTER(C.c_int32))
        if problem is not None:
            self.problem = np.ascontiguousarray(problem, dtype=np.int32)
            pp = self.problem.ctypes.data_as(C.POINTER(C.c_int32))
            if self.refined:
                rc = self.lib.gbh_create_refined_batched(C.byref(p), C.byref(r), pp, self.nproblems, C.byref(ctx))
            else:
                rc = self.lib.gbh_create_batched(C.byref(p), pp, self.nproblems, C.byref(ctx))
        elif self.refined:
            rc = self.lib.gbh_create_refined(C.byref(p), C.byref(r), C.byref(ctx))
        else:
            rc = self.lib.gbh_create(C.byref(p), C.byref(ctx))
        if rc != 0:
            raise _abi.GbhError(rc, self.lib.gbh_last_error(None).decode())
        self.ctx = ctx
        self.device = torch.cuda.current_device()
        self.nstages = 2
        self.telescoping = False

    @classmethod
    def from_lattice(cls, lat, **kw):
        """Build from any object with ndim, nb, n, ng, bc, extent (e.g. workloads.Lattice)."""
        return cls(lat.ndim, lat.n, lat.ng, nb=lat.nb,
                   periodic=tuple(b == "periodic" for b in lat.bc), extent=lat.extent, **kw)

    @classmethod
    def from_two_level(cls, tl, **kw):
        """Two-level composite grid: any object with `coarse` (a lattice), `lo`, `hi`
        (the fine region in coarse blocks, or the bounding box of `refined`, an
        optional list of refined coarse block coordinates), e.g. workloads.TwoLevel.
        The state holds the coarse blocks, then the children of the refined
        blocks in fine-lattice order over [lo, hi)."""
        from .grid import two_level_tables
        c = tl.coarse
        nbr, dx, parent, children = two_level_tables(
            c.ndim, c.nb, c.n, tl.lo, tl.hi, tuple(b == "periodic" for b in c.bc), c.dx, getattr(tl, "refined", None))
        return cls(c.ndim, c.n, c.ng, nbr=nbr, dx=dx, parent=parent, children=children, **kw)

    @classmethod
    def from_two_level_batch(cls, grids, **kw):
        """Independent two-level composite grids (objects like those
        from_two_level takes, with equal block shapes and guard widths) in one
        context; the state array holds their blocks one problem after another,
        each problem's coarse blocks before its fine blocks."""
        from .grid import batched_two_level_tables
        tls = list(grids)
        c = tls[0].coarse
        nbr, dx, parent, children, problem = batched_two_level_tables(
            [(t.coarse.ndim, t.coarse.nb, t.coarse.n, t.lo, t.hi,
              tuple(b == "periodic" for b in t.coarse.bc), t.coarse.dx, getattr(t, "refined", None)) for t in tls])
        return cls(c.ndim, c.n, c.ng, nbr=nbr, dx=dx, parent=parent, children=children,
                   problem=problem, nproblems=len(tls), **kw)

    @classmethod
    def from_batch(cls, lattices, **kw):
        """Independent problems (uniform lattices with equal block shapes) in one
        context; the state array holds their blocks one problem after another."""
        from .grid import batched_tables
        lats = list(lattices)
        c = lats[0]
        nbr, dx, problem = batched_tables(
            [(l.ndim, l.nb, tuple(b == "periodic" for b in l.bc), l.dx) for l in lats])
        return cls(c.ndim, c.n, c.ng, nbr=nbr, dx=dx, problem=problem, nproblems=len(lats), **kw)

    # -- helpers -----------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.gbh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise _abi.GbhError(rc, self.lib.gbh_last_error(self.ctx).decode())

    def _state(self, U: torch.Tensor, name="U") -> int:
        if not isinstance(U, torch.Tensor) or U.dtype != torch.float64 or not U.is_cuda:
            raise TypeError(f"{name} must be a float64 CUDA tensor")
        if tuple(U.shape) != self.shape or not U.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {self.shape}, got {tuple(U.shape)}")
        return U.data_ptr()

    def _scalar(self, t: torch.Tensor, name="dt", n: int = 1) -> int:
        """Device pointer of a contiguous float64 CUDA tensor of at least n values."""
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
        if t.numel() < n:
            raise ValueError(f"{name} holds {t.numel()} values, {n} are needed")
        return t.data_ptr()

    def _dt(self, t: torch.Tensor, name="dt_dev") -> int:
        """One time step per problem (nproblems values)."""
        return self._scalar(t, name, self.nproblems)

    def empty_state(self) -> torch.Tensor:
        return torch.empty(self.shape, dtype=torch.float64, device="cuda")

    # -- the ABI -----------------------------------------------------------
    def fill_guardcells(self, U):
        self._check(self.lib.hydro_fill_guardcells(self.ctx, self._state(U), _stream_handle()))
        return U

    def compute_dt(self, U, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.nproblems, dtype=torch.float64, device="cuda")
        self._check(self.lib.hydro_compute_dt(self.ctx, self._state(U), self._dt(out, "out"), _stream_handle()))
        return out

    def stage(self, Uin, Un, Uout, dt: float, a: float, b: float, guarded: bool = False):
        fn = self.lib.hydro_stage_guarded if guarded else self.lib.hydro_stage
        un = self._state(Un, "Un") if Un is not None else None
        self._check(fn(self.ctx, self._state(Uin, "Uin"), un, self._state(Uout, "Uout"),
                       float(dt), float(a), float(b), _stream_handle()))
        return Uout

    def step(self, U, dt: float):
        self._check(self.lib.hydro_step(self.ctx, self._state(U), float(dt), _stream_handle()))
        return U

    def step_cfl(self, U, dt_dev: torch.Tensor):
        self._check(self.lib.hydro_step_cfl(self.ctx, self._state(U), self._dt(dt_dev), _stream_handle()))
        return U

    def advance(self, U, nsteps: int, dt_dev: torch.Tensor, dt_hist: Optional[torch.Tensor] = None):
        h = None
        if dt_hist is not None:
            h = self._scalar(dt_hist, "dt_hist", int(nsteps) * self.nproblems)
        self._check(self.lib.hydro_advance(self.ctx, self._state(U), int(nsteps), self._dt(dt_dev), h,
                                           _stream_handle()))
        return U

    def advance_graph(self, U, nsteps: int, dt_dev: torch.Tensor):
        """nsteps of step_cfl as one CUDA graph (captured on first use)."""
        self._check(self.lib.hydro_advance_graph(self.ctx, self._state(U), int(nsteps), self._dt(dt_dev),
                                                 _stream_handle()))
        return U

    def autotune(self, U):
        kc, ipc = C.c_int(0), C.c_int(0)
        self._check(self.lib.gbh_autotune(self.ctx, self._state(U), C.byref(kc), C.byref(ipc), _stream_handle()))
        return int(kc.value), int(ipc.value)

    def set_decomposition(self, kchunk: int, items_per_cta: int):
        self._check(self.lib.gbh_set_decomposition(self.ctx, int(kchunk), int(items_per_cta)))

    def set_tile_split(self, ring: int, ysplit: int):
        """Row bands per plane tile of the stage kernel for ring width 0, 2 or 4."""
        self._check(self.lib.gbh_set_tile_split(self.ctx, int(ring), int(ysplit)))

    def tile_split(self, ring: int = 0) -> int:
        out = C.c_int(0)
        self._check(self.lib.gbh_get_tile_split(self.ctx, int(ring), C.byref(out)))
        return int(out.value)

    def set_telescoping(self, enable: bool = True):
        """Telescoping SSP-RK (one guard fill per step; needs nguard >= 2 * stages)."""
        self._check(self.lib.gbh_set_telescoping(self.ctx, int(bool(enable))))
        self.telescoping = bool(enable)

    def set_rk_stages(self, nstages: int):
        """2 (SSP-RK2, the default) or 3 (SSP-RK3) Shu-Osher stages per step."""
        self._check(self.lib.gbh_set_rk_stages(self.ctx, int(nstages)))
        self.nstages = int(nstages)

    def set_prim_carry(self, enable: bool = True):
        """Carry each stage's primitive variables to the next stage (on by default;
        the results do not depend on it, bit for bit; telescoping steps never carry)."""
        self._check(self.lib.gbh_set_prim_carry(self.ctx, int(bool(enable))))

    def prim_carry(self) -> bool:
        out = C.c_int(0)
        self._check(self.lib.gbh_get_prim_carry(self.ctx, C.byref(out)))
        return bool(out.value)

    def set_face_prepass(self, enable: bool = True):
        """Solve every block face once in a pre-pass before each interior stage
        (on by default on 3-D uniform contexts; the results do not depend on it, bit for bit)."""
        self._check(self.lib.gbh_set_face_prepass(self.ctx, int(bool(enable))))

    def face_prepass(self) -> bool:
        out = C.c_int(0)
        self._check(self.lib.gbh_get_face_prepass(self.ctx, C.byref(out)))
        return bool(out.value)

    # -- adjoint ------------------------------------------------------------
    def step_adjoint(self, Un, dt: float, lam_next, lam_prev=None, U1=None):
        """dJ/dU^n of step(Un, dt) from dJ/dU^{n+1} (dt held fixed, forward branches frozen).
        U1: that step's first-stage state if the caller kept it (saves a stage)."""
        if lam_prev is None:
            lam_prev = torch.zeros_like(lam_next)
        if U1 is None:
            rc = self.lib.hydro_step_adjoint(self.ctx, self._state(Un, "Un"), float(dt),
                                             self._state(lam_next, "lam_next"), self._state(lam_prev, "lam_prev"),
                                             _stream_handle())
        else:
            rc = self.lib.hydro_step_adjoint_stored(self.ctx, self._state(Un, "Un"), self._state(U1, "U1"), float(dt),
                                                    self._state(lam_next, "lam_next"),
                                                    self._state(lam_prev, "lam_prev"), _stream_handle())
        self._check(rc)
        return lam_prev

    def stage_vjp(self, U, M, scale: float, A=None, cA: float = 0.0, B=None, cB: float = 0.0, out=None):
        """out = cA A + cB B + J_L(U)^T (scale M) on interior cells."""
        if out is None:
            out = torch.zeros_like(U)
        a = self._state(A, "A") if A is not None else None
        b = self._state(B, "B") if B is not None else None
        self._check(self.lib.hydro_stage_vjp(self.ctx, self._state(U), self._state(M, "M"), float(scale), a,
                                             float(cA), b, float(cB), self._state(out, "out"), _stream_handle()))
        return out

    def prim_to_cons(self, W, U=None):
        if U is None:
            U = torch.zeros_like(W)
        self._check(self.lib.hydro_prim_to_cons(self.ctx, self._state(W, "W"), self._state(U), _stream_handle()))
        return U

    def prim_to_cons_vjp(self, W, lamU, lamW=None):
        if lamW is None:
            lamW = torch.zeros_like(W)
        self._check(self.lib.hydro_prim_to_cons_vjp(self.ctx, self._state(W, "W"), self._state(lamU, "lamU"),
                                                    self._state(lamW, "lamW"), _stream_handle()))
        return lamW

    def _host_state(self, U_host, shape=None) -> int:
        shape = self.shape if shape is None else shape
        if isinstance(U_host, torch.Tensor):
            if U_host.is_cuda or U_host.dtype != torch.float64 or not U_host.is_contiguous():
                raise TypeError("U_host must be a contiguous float64 CPU tensor")
            ptr = U_host.data_ptr()
        else:
            if U_host.dtype != np.float64 or not U_host.flags.c_contiguous:
                raise TypeError("U_host must be a C-contiguous float64 array")
            ptr = U_host.ctypes.data
        if tuple(U_host.shape) != shape:
            raise ValueError(f"U_host must have shape {shape}")
        return ptr

    def step_host(self, U_host, dt_host):
        """One step of a host-resident state with the copies overlapped with the
        stages.  dt_host: float64 numpy array of nproblems entries, in and out
        (<= 0 on the first call: computed from U_host); returns U_host."""
        if not (isinstance(dt_host, np.ndarray) and dt_host.dtype == np.float64 and dt_host.size >= self.nproblems
                and dt_host.flags.c_contiguous):
            raise TypeError("dt_host must be a contiguous float64 array with one entry per problem")
        self._check(self.lib.hydro_step_host(self.ctx, self._host_state(U_host), dt_host.ctypes.data,
                                             _stream_handle()))
        return U_host

    def step_host_interior(self, U_host, dt_host):
        """step_host for a host state of the interior cells only, shape
        interior_shape = (nblocks, 5, nz, ny, nx): only those bytes cross the
        host link.  dt_host as in step_host; returns U_host."""
        if not (isinstance(dt_host, np.ndarray) and dt_host.dtype == np.float64 and dt_host.size >= self.nproblems
                and dt_host.flags.c_contiguous):
            raise TypeError("dt_host must be a contiguous float64 array with one entry per problem")
        self._check(self.lib.hydro_step_host_interior(self.ctx, self._host_state(U_host, self.interior_shape),
                                                      dt_host.ctypes.data, _stream_handle()))
        return U_host

    def set_host_pipeline(self, chunks: int = 0):
        """Block chunks of step_host (0: the fewest chunks of one stage-kernel wave each)."""
        self._check(self.lib.gbh_set_host_pipeline(self.ctx, int(chunks)))

    def advance_host(self, U_host, nsteps: int, dt_hist_host=None, interior: bool = False):
        """U_host: a float64 CPU tensor (pinned or not) or numpy array of the state
        shape (interior=True: of interior_shape, the interior cells only)."""
        ptr = self._host_state(U_host, self.interior_shape if interior else None)
        h = None
        if dt_hist_host is not None:
            need = int(nsteps) * self.nproblems
            if isinstance(dt_hist_host, np.ndarray):
                if dt_hist_host.dtype != np.float64 or not dt_hist_host.flags.c_contiguous or dt_hist_host.size < need:
                    raise ValueError(f"dt_hist_host must be a contiguous float64 array of >= {need} values")
                h = dt_hist_host.ctypes.data
            else:
                if (dt_hist_host.is_cuda or dt_hist_host.dtype != torch.float64 or not dt_hist_host.is_contiguous()
                        or dt_hist_host.numel() < need):
                    raise ValueError(f"dt_hist_host must be a contiguous float64 CPU tensor of >= {need} values")
                h = dt_hist_host.data_ptr()
        fn = self.lib.hydro_advance_host_interior if interior else self.lib.hydro_advance_host
        self._check(fn(self.ctx, ptr, int(nsteps), h, _stream_handle()))
        return U_host

    def check_state(self, U) -> int:
        n = C.c_longlong(0)
        rc = self.lib.hydro_check_state(self.ctx, self._state(U), C.byref(n), _stream_handle())
        if rc not in (0, _abi.GBH_ERR_UNPHYSICAL):
            self._check(rc)
        return int(n.value)

    def floor_hits(self) -> int:
        n = C.c_longlong(0)
        self._check(self.lib.hydro_floor_hits(self.ctx, C.byref(n), _stream_handle()))
        return int(n.value)

    def set_kernel_timing(self, on: bool):
        self._check(self.lib.gbh_set_kernel_timing(self.ctx, 1 if on else 0))

    def stage_kernel_time(self):
        ms, n = C.c_double(0), C.c_longlong(0)
        self._check(self.lib.gbh_stage_kernel_time(self.ctx, C.byref(ms), C.byref(n), _stream_handle()))
        return float(ms.value), int(n.value)


def fp64_probe(blocks: int, threads: int, iters: int, out: torch.Tensor, lanes: int = 32, form: int = 1):
    """FP64 throughput probe (gbh_fp64_probe): form 0 = FMA with constant
    operands, 1 = FMA with per-thread register operands, 2 = add, 3 = multiply,
    4 = FMA with warp-uniform register operands."""
    lib = _abi.load()
    rc = lib.gbh_fp64_probe(int(blocks), int(threads), int(iters), int(lanes), int(form), out.data_ptr(),
                            _stream_handle())
    if rc != 0:
        raise _abi.GbhError(rc, lib.gbh_last_error(None).decode())


def sm_count() -> int:
    return int(_abi.load().gbh_device_sm_count())
