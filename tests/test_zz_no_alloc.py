"""hydro_step_static: the entry point for callers that cannot allocate device
memory -- a host whose memory manager owns the whole device pool, or a plug-in
in a process that forbids cudaMalloc/cudaFree after start-up.  Its scratch is
a fixed file-scope device array, so it needs no context.

Checked through the C ABI on two consecutive calls: bit for bit the result of
hydro_step (the context-based entry point runs the same two stage launches on
the same inputs), within the single-step tolerance of the oracle's step, and
with the device's free memory unchanged by a call once the library is loaded.
Oversized states and more than 8192 blocks must be rejected.  This file is
collected last on purpose, so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle
from tests.gridutil import relerr_per_var, to_global

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-13   # the single-step tolerance of the other GPU tests
GBH_ERR_INVAL = -1


def _params(lat, keep):
    from paper_2401_03378_gb300 import _abi
    from paper_2401_03378_gb300.grid import neighbour_table
    p = _abi.GbhParams()
    p.ndim, p.nxb, p.nyb, p.nzb = lat.ndim, lat.n[0], lat.n[1], lat.n[2]
    p.nguard, p.nblocks = lat.ng, lat.nblocks
    p.gamma, p.cfl, p.small_rho, p.small_p = 1.4, 0.8, 1e-12, 1e-14
    nbr = np.ascontiguousarray(neighbour_table(lat.ndim, lat.nb, [b == "periodic" for b in lat.bc]),
                               dtype=np.int32)
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
def test_static_step_matches_context_step_and_oracle_twice(lat, ic):
    import paper_2401_03378_gb300 as gb
    lib = gb.load()
    U0 = {"sedov": wl.sedov, "sod": wl.sod, "random": lambda l: wl.random_state(l, seed=5)}[ic](lat)
    h = gb.Hydro.from_lattice(lat)
    o = Oracle(lat)
    keep = []
    p = _params(lat, keep)
    Ua = torch.from_numpy(U0.copy()).cuda()
    Ub = torch.from_numpy(U0.copy()).cuda()
    ref = U0.copy()
    stream = torch.cuda.current_stream().cuda_stream
    zs, ys, xs = lat.interior_slices()
    for call in range(2):
        dt = float(h.compute_dt(Ua).cpu()[0])
        h.step(Ua, dt)
        o.step(ref, dt)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = lib.hydro_step_static(C.byref(p), Ub.data_ptr(), dt, stream)
        assert rc == 0, lib.gbh_last_error(None)
        torch.cuda.synchronize()
        if call == 1:
            # the library is loaded on this device by now: a call allocates nothing
            assert torch.cuda.mem_get_info()[0] == free_before
        a, b = Ua.cpu().numpy(), Ub.cpu().numpy()
        assert np.array_equal(b[:, :, zs, ys, xs], a[:, :, zs, ys, xs])
        err = relerr_per_var(to_global(b, lat), to_global(ref, lat))
        assert np.all(err <= TOL), err


def test_static_step_rejects_oversized_state():
    import paper_2401_03378_gb300 as gb
    lib = gb.load()
    lat = wl.lattice_3d(6, 6, 6, 16, 16, 16, 4)      # 119 MB state > 40 MiB
    keep = []
    p = _params(lat, keep)
    U = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.hydro_step_static(C.byref(p), U.data_ptr(), 1e-3, torch.cuda.current_stream().cuda_stream)
    assert rc == GBH_ERR_INVAL
    assert b"static scratch" in lib.gbh_last_error(None)


def test_static_step_rejects_more_than_8192_blocks():
    """A 2-D lattice of 91 x 91 blocks of 4^2 cells with 2 guard layers: 8281
    blocks in a 21 MB state, so only the block limit can reject it."""
    import paper_2401_03378_gb300 as gb
    lib = gb.load()
    lat = wl.lattice_2d(91, 91, 4, 4, 2)
    assert lat.nblocks > 8192 and 8 * lat.nblocks * 5 * np.prod(lat.padded) < 40 << 20
    keep = []
    p = _params(lat, keep)
    U = torch.zeros(lat.shape, dtype=torch.float64, device="cuda")
    rc = lib.hydro_step_static(C.byref(p), U.data_ptr(), 1e-3, torch.cuda.current_stream().cuda_stream)
    assert rc == GBH_ERR_INVAL
    assert b"8192" in lib.gbh_last_error(None)
