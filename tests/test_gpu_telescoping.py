"""GPU telescoping mode (gbh_set_telescoping; Sec. 4.2, one guard fill per
step) against the oracle's telescoping step, and against the GPU's own
non-telescoping step where neighbours supply every halo (bitwise)."""
import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle
from tests.gridutil import relerr_per_var, to_global

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2401_03378_gb300 as pkg
    pkg.load()
    return pkg


def dev(U):
    return torch.from_numpy(np.ascontiguousarray(U)).cuda()


def host(T):
    torch.cuda.synchronize()
    return T.cpu().numpy()


def interior(U, lat):
    zs, ys, xs = lat.interior_slices()
    return U[:, :, zs, ys, xs]


LATTICES = [
    wl.lattice_2d(3, 2, 16, 16, 4),
    wl.lattice_2d(4, 4, 8, 8, 4, bc="periodic"),
    wl.lattice_2d(3, 3, 4, 4, 4, bc=("periodic", "outflow")),
    wl.lattice_3d(2, 2, 2, 4, 4, 4, 4),
    wl.lattice_3d(2, 3, 2, 8, 8, 8, 4, bc=("outflow", "periodic", "outflow")),
    wl.lattice_3d(2, 2, 3, 16, 16, 16, 4),
    wl.lattice_3d(1, 1, 2, 16, 16, 16, 5, bc="periodic"),
]


@pytest.mark.parametrize("lat", LATTICES)
def test_one_step_matches_oracle(gb, lat):
    U = wl.random_state(lat, seed=31, rough=True)
    o = Oracle(lat)
    dt = o.compute_dt(U)
    ref = U.copy()
    hits_o = o.step(ref, dt, telescoping=True)
    h = gb.Hydro.from_lattice(lat)
    h.set_telescoping(True)
    Ug = dev(U)
    h.step(Ug, dt)
    err = relerr_per_var(to_global(host(Ug), lat), to_global(ref, lat))
    assert np.all(err <= 1e-13), err
    assert h.floor_hits() == hits_o == 0


@pytest.mark.parametrize("lat", LATTICES[:6])
def test_run_with_cfl_dt_matches_oracle(gb, lat):
    U = wl.random_state(lat, seed=32, rough=False)
    n = 12
    ref = U.copy()
    hist_o, _ = Oracle(lat).run(ref, n, telescoping=True)
    h = gb.Hydro.from_lattice(lat)
    h.set_telescoping(True)
    Ug = dev(U)
    dt = h.compute_dt(Ug)
    hist = torch.zeros(n, dtype=torch.float64, device="cuda")
    h.advance(Ug, n, dt, hist)
    assert np.max(np.abs(host(hist) / hist_o - 1)) <= 1e-12
    err = relerr_per_var(to_global(host(Ug), lat), to_global(ref, lat))
    assert np.all(err <= 1e-11), err


@pytest.mark.parametrize("lat", [wl.lattice_2d(4, 3, 16, 16, 4, bc="periodic"),
                                 wl.lattice_3d(2, 3, 2, 16, 16, 16, 4, bc="periodic"),
                                 wl.lattice_3d(3, 2, 2, 8, 8, 8, 4, bc="periodic")])
def test_periodic_equals_non_telescoping_bitwise(gb, lat):
    U = wl.random_state(lat, seed=33, rough=True)
    h = gb.Hydro.from_lattice(lat)
    A, B = dev(U), dev(U)
    da, db = h.compute_dt(A), h.compute_dt(B)
    h.advance(A, 6, da)
    h.set_telescoping(True)
    h.advance(B, 6, db)
    assert torch.equal(da, db)
    assert np.array_equal(interior(host(A), lat), interior(host(B), lat))


@pytest.mark.parametrize("kchunk,ipc", [(8, 1), (6, 3), (0, 37), (2, 2)])
def test_decomposition_does_not_change_results(gb, kchunk, ipc):
    lat = wl.lattice_3d(3, 2, 2, 16, 16, 16, 4)
    U0 = wl.sedov(lat)
    h = gb.Hydro.from_lattice(lat)
    h.set_telescoping(True)
    A = dev(U0)
    da = h.compute_dt(A)
    h.advance(A, 3, da)
    h.set_decomposition(kchunk, ipc)
    B = dev(U0)
    db = h.compute_dt(B)
    h.advance(B, 3, db)
    assert torch.equal(da, db)
    assert np.array_equal(interior(host(A), lat), interior(host(B), lat))


def test_graph_and_batched_contexts(gb):
    probs = wl.ensemble(count=4, seed=5, choices=(32, 64))
    lats = [l for l, _ in probs]
    U0 = np.concatenate([u for _, u in probs])
    h = gb.Hydro.from_batch(lats)
    h.set_telescoping(True)
    A, B = dev(U0), dev(U0)
    da, db = h.compute_dt(A), h.compute_dt(B)
    h.advance(A, 8, da)
    h.advance_graph(B, 8, db)
    assert torch.equal(A, B) and torch.equal(da, db)
    # every problem of the batch against the oracle's telescoping run
    o = 0
    out = host(A)
    for lat, (_, Ui) in zip(lats, probs):
        ref = Ui.copy()
        Oracle(lat).run(ref, 8, telescoping=True)
        err = relerr_per_var(to_global(out[o:o + lat.nblocks], lat), to_global(ref, lat))
        assert np.all(err <= 1e-11), err
        o += lat.nblocks


def test_sedov_3d_128_20_steps(gb):
    lat = wl.lattice_3d(8, 8, 8)
    U0 = wl.sedov(lat)
    ref = U0.copy()
    hist_o, _ = Oracle(lat).run(ref, 20, telescoping=True)
    h = gb.Hydro.from_lattice(lat)
    h.set_telescoping(True)
    Ug = dev(U0)
    dt = h.compute_dt(Ug)
    hist = torch.zeros(20, dtype=torch.float64, device="cuda")
    h.advance(Ug, 20, dt, hist)
    assert np.max(np.abs(host(hist) / hist_o - 1)) <= 1e-12
    assert np.all(relerr_per_var(to_global(host(Ug), lat), to_global(ref, lat)) <= 1e-11)


def test_mode_errors(gb):
    from paper_2401_03378_gb300._abi import GbhError
    h = gb.Hydro.from_lattice(wl.lattice_2d(2, 2, 8, 8, 3))
    with pytest.raises(GbhError):
        h.set_telescoping(True)
    lat = wl.lattice_2d(2, 2, 8, 8, 4)
    h = gb.Hydro.from_lattice(lat)
    h.set_telescoping(True)
    U = dev(wl.random_state(lat, seed=1))
    # the adjoint of the telescoping step recomputes its stages; the stored
    # variant (first stage passed in) belongs to the plain step only
    h.step_adjoint(U, 1e-4, torch.zeros_like(U))
    with pytest.raises(GbhError):
        h.step_adjoint(U, 1e-4, torch.zeros_like(U), U1=U.clone())
    h.set_telescoping(False)
    h.step_adjoint(U, 1e-4, torch.zeros_like(U), U1=U.clone())
    tl = wl.two_level(wl.lattice_2d(4, 4, 16, 16, 3, bc="periodic"), (1, 1), (3, 3))
    h2 = gb.Hydro.from_two_level(tl)
    with pytest.raises(GbhError):
        h2.set_telescoping(True)


# ---- two-level grids: the level-by-level telescoping variant ----------------

from tests.test_gpu_amr import GRIDS, leaf_err, smooth  # noqa: E402
from oracle.oracle import Oracle2  # noqa: E402


@pytest.mark.parametrize("tl", GRIDS)
def test_two_level_one_step_matches_oracle(gb, tl):
    U = smooth(tl, 12)
    o = Oracle2(tl)
    o.restrict(U)
    dt = o.compute_dt(U)
    ref = U.copy()
    o.step(ref, dt, telescoping=True)
    h = gb.Hydro.from_two_level(tl)
    h.set_telescoping(True)
    Ug = dev(U)
    h.step(Ug, dt)
    out = host(Ug)
    assert np.all(leaf_err(out, ref, tl) <= 1e-13), leaf_err(out, ref, tl)
    cov = [b for b in range(tl.n0) if tl.covered(b)]
    zs, ys, xs = tl.coarse.interior_slices()
    a = np.moveaxis(out[cov][:, :, zs, ys, xs], 1, 0)
    b = np.moveaxis(ref[cov][:, :, zs, ys, xs], 1, 0)
    assert np.all(relerr_per_var(a, b) <= 1e-13)


def test_two_level_sedov_run_and_conservation(gb):
    tl = wl.two_level(wl.lattice_3d(8, 8, 8), (2, 2, 2), (6, 6, 6))
    U0 = wl.sedov_two_level(tl)
    ref = U0.copy()
    hist_o, hits = Oracle2(tl).run(ref, 20, telescoping=True)
    h = gb.Hydro.from_two_level(tl)
    h.set_telescoping(True)
    Ug = dev(U0)
    h.fill_guardcells(Ug)
    dt = h.compute_dt(Ug)
    hist = torch.zeros(20, dtype=torch.float64, device="cuda")
    h.advance(Ug, 20, dt, hist)
    assert np.max(np.abs(host(hist) / hist_o - 1)) <= 1e-12
    assert np.all(leaf_err(host(Ug), ref, tl) <= 1e-11)
    assert hits == 0 and h.floor_hits() == 0


def test_two_level_periodic_conservation_and_graph(gb):
    tl = GRIDS[0]
    U = smooth(tl, 13)
    Oracle2(tl).restrict(U)

    def totals(A):
        zs, ys, xs = tl.coarse.interior_slices()
        vc, vf = np.prod(tl.coarse.dx), np.prod(tl.fine.dx)
        t = np.zeros(5)
        for b in range(tl.nblocks):
            if b < tl.n0 and tl.covered(b):
                continue
            t += A[b][:, zs, ys, xs].sum(axis=(1, 2, 3)) * (vc if b < tl.n0 else vf)
        return t
    t0, scale = totals(U), totals(np.abs(U))
    h = gb.Hydro.from_two_level(tl)
    h.set_telescoping(True)
    A, B = dev(U), dev(U)
    da, db = h.compute_dt(A), h.compute_dt(B)
    h.advance(A, 10, da)
    h.advance_graph(B, 10, db)
    assert torch.equal(A, B) and torch.equal(da, db)
    assert np.all(np.abs(totals(host(A)) - t0) <= 10 * 64 * np.finfo(float).eps * scale)
