"""hydro_step_static: the entry point for callers that cannot allocate device
memory (its scratch is a fixed file-scope device array).  Checked through the
C ABI against hydro_step, the context-based entry point, on two consecutive
calls; oversized requests must be rejected.  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import workloads as wl
from tests.gridutil import relerr_per_var, to_global

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-13   # the single-step tolerance of the other GPU tests


def _params(h, lat, keep):
    from paper_2401_03378_gb300 import _abi
    p = _abi.GbhParams()
    p.ndim, p.nxb, p.nyb, p.nzb = lat.ndim, lat.n[0], lat.n[1], lat.n[2]
    p.nguard, p.nblocks = lat.ng, lat.nblocks
    p.gamma, p.cfl, p.small_rho, p.small_p = 1.4, 0.8, 1e-12, 1e-14
    nbr = np.ascontiguousarray(h.nbr if h is not None else
                               __import__("paper_2401_03378_gb300").neighbour_table(
                                   lat.ndim, lat.nb, [b == "periodic" for b in lat.bc]), dtype=np.int32)
    dx = np.ascontiguousarray(np.tile(np.array(lat.dx), (lat.nblocks, 1)))
    keep += [nbr, dx]
    p.nbr = nbr.ctypes.data_as(C.POINTER(C.c_int32))
    p.dx = dx.ctypes.data_as(C.POINTER(C.c_double))
    return p


@pytest.mark.parametrize("lat,ic", [
    (wl.lattice_3d(2, 2, 2, 16, 16, 16, 4), "sedov"),
    (wl.lattice_2d(8, 8, 16, 16, 4), "sod"),
    (wl.lattice_3d(2, 2, 2, 8, 8, 8, 4, bc="periodic"), "random"),
])
def test_static_step_matches_context_step_twice(lat, ic):
    import paper_2401_03378_gb300 as gb
    lib = gb.load()
    U0 = {"sedov": wl.sedov, "sod": wl.sod, "random": lambda l: wl.random_state(l, seed=5)}[ic](lat)
    h = gb.Hydro.from_lattice(lat)
    keep = []
    p = _params(h, lat, keep)
    Ua = torch.from_numpy(U0.copy()).cuda()
    Ub = torch.from_numpy(U0.copy()).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        dt = float(h.compute_dt(Ua).cpu()[0])
        h.step(Ua, dt)
        rc = lib.hydro_step_static(C.byref(p), Ub.data_ptr(), dt, stream)
        assert rc == 0, lib.gbh_last_error(None)
        torch.cuda.synchronize()
        err = relerr_per_var(to_global(Ub.cpu().numpy(), lat), to_global(Ua.cpu().numpy(), lat))
        assert np.all(err <= TOL), err


def test_static_step_rejects_oversized_state():
    import paper_2401_03378_gb300 as gb
    lib = gb.load()
    lat = wl.lattice_3d(6, 6, 6, 16, 16, 16, 4)      # 119 MB state > 40 MiB
    keep = []
    p = _params(None, lat, keep)
    U = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.hydro_step_static(C.byref(p), U.data_ptr(), 1e-3, torch.cuda.current_stream().cuda_stream)
    assert rc == -1
    assert b"static scratch" in lib.gbh_last_error(None)
