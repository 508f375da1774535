"""GPU three-stage SSP-RK (gbh_set_rk_stages) on every step path against the
oracle's three-stage steps: non-telescoping and telescoping on uniform and
batched grids, all-levels and level-by-level telescoping on two levels."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle, Oracle2
from tests.gridutil import relerr_per_var, to_global
from tests.test_gpu_amr import leaf_err, smooth

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
    wl.lattice_2d(4, 4, 8, 8, 6, bc="periodic"),
    wl.lattice_3d(2, 2, 2, 4, 4, 4, 4),
    wl.lattice_3d(2, 3, 2, 8, 8, 8, 6, bc=("outflow", "periodic", "outflow")),
    wl.lattice_3d(2, 2, 2, 16, 16, 16, 6),
]


# the telescoping three-stage step needs 6 guard cells
@pytest.mark.parametrize("lat,telescoping", [(l, t) for l in LATTICES for t in (False, True) if not t or l.ng >= 6])
def test_one_step_and_run_match_oracle(gb, lat, telescoping):
    U = wl.random_state(lat, seed=51, rough=True)
    o = Oracle(lat)
    dt = o.compute_dt(U)
    ref = U.copy()
    o.step(ref, dt, telescoping=telescoping, stages=3)
    h = gb.Hydro.from_lattice(lat)
    h.set_rk_stages(3)
    h.set_telescoping(telescoping)
    Ug = dev(U)
    h.step(Ug, dt)
    err = relerr_per_var(to_global(host(Ug), lat), to_global(ref, lat))
    assert np.all(err <= 1e-13), err
    # 8 steps with the device CFL dt
    U = wl.random_state(lat, seed=52, rough=False)
    ref = U.copy()
    hist_o, _ = o.run(ref, 8, telescoping=telescoping, stages=3)
    Ug = dev(U)
    dtd = h.compute_dt(Ug)
    hist = torch.zeros(8, dtype=torch.float64, device="cuda")
    h.advance(Ug, 8, dtd, hist)
    assert np.max(np.abs(host(hist) / hist_o - 1)) <= 1e-12
    assert np.all(relerr_per_var(to_global(host(Ug), lat), to_global(ref, lat)) <= 1e-11)


@pytest.mark.parametrize("lat", [wl.lattice_2d(4, 3, 16, 16, 6, bc="periodic"),
                                 wl.lattice_3d(2, 2, 3, 8, 8, 8, 6, bc="periodic")])
def test_telescoping_periodic_equals_non_telescoping_bitwise(gb, lat):
    U = wl.random_state(lat, seed=53, rough=True)
    h = gb.Hydro.from_lattice(lat)
    h.set_rk_stages(3)
    A, B = dev(U), dev(U)
    da, db = h.compute_dt(A), h.compute_dt(B)
    h.advance(A, 4, da)
    h.set_telescoping(True)
    h.advance(B, 4, db)
    assert torch.equal(da, db)
    assert np.array_equal(interior(host(A), lat), interior(host(B), lat))


def test_sedov_3d_128_rk3(gb):
    lat = wl.lattice_3d(8, 8, 8)
    U0 = wl.sedov(lat)
    ref = U0.copy()
    hist_o, _ = Oracle(lat).run(ref, 15, stages=3)
    h = gb.Hydro.from_lattice(lat)
    h.set_rk_stages(3)
    Ug = dev(U0)
    dt = h.compute_dt(Ug)
    hist = torch.zeros(15, dtype=torch.float64, device="cuda")
    h.advance(Ug, 15, dt, hist)
    assert np.max(np.abs(host(hist) / hist_o - 1)) <= 1e-12
    assert np.all(relerr_per_var(to_global(host(Ug), lat), to_global(ref, lat)) <= 1e-11)


def test_batched_and_graph(gb):
    probs = wl.ensemble(count=4, seed=6, choices=(32, 64))
    lats = [l for l, _ in probs]
    U0 = np.concatenate([u for _, u in probs])
    h = gb.Hydro.from_batch(lats)
    h.set_rk_stages(3)
    A, B = dev(U0), dev(U0)
    da, db = h.compute_dt(A), h.compute_dt(B)
    h.advance(A, 6, da)
    h.advance_graph(B, 6, db)
    assert torch.equal(A, B) and torch.equal(da, db)
    out, o = host(A), 0
    for lat, (_, Ui) in zip(lats, probs):
        ref = Ui.copy()
        Oracle(lat).run(ref, 6, stages=3)
        assert np.all(relerr_per_var(to_global(out[o:o + lat.nblocks], lat), to_global(ref, lat)) <= 1e-11)
        o += lat.nblocks


GRIDS = [
    wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 6, bc="periodic"), (1, 1, 1), (3, 3, 3)),
    wl.two_level(wl.lattice_3d(4, 3, 4, 8, 8, 8, 6), (1, 1, 2), (2, 2, 3)),
    wl.two_level(wl.lattice_2d(4, 4, 16, 16, 6, bc="periodic"), (1, 1), (3, 3)),
    wl.two_level(wl.lattice_2d(5, 4, 8, 8, 6), (1, 1), (4, 3)),
]


@pytest.mark.parametrize("telescoping", [False, True])
@pytest.mark.parametrize("tl", GRIDS)
def test_two_level_matches_oracle(gb, tl, telescoping):
    U = smooth(tl, 54)
    o = Oracle2(tl)
    o.restrict(U)
    dt = o.compute_dt(U)
    ref = U.copy()
    o.step(ref, dt, telescoping=telescoping, stages=3)
    h = gb.Hydro.from_two_level(tl)
    h.set_rk_stages(3)
    h.set_telescoping(telescoping)
    Ug = dev(U)
    h.step(Ug, dt)
    assert np.all(leaf_err(host(Ug), ref, tl) <= 1e-13)
    ref2 = U.copy()
    hist_o, _ = o.run(ref2, 6, telescoping=telescoping, stages=3)
    Ug = dev(U)
    dtd = h.compute_dt(Ug)
    hist = torch.zeros(6, dtype=torch.float64, device="cuda")
    h.advance(Ug, 6, dtd, hist)
    assert np.max(np.abs(host(hist) / hist_o - 1)) <= 1e-12
    assert np.all(leaf_err(host(Ug), ref2, tl) <= 1e-11)


def test_errors(gb):
    from paper_2401_03378_gb300._abi import GbhError
    lat = wl.lattice_2d(2, 2, 8, 8, 4)
    h = gb.Hydro.from_lattice(lat)
    with pytest.raises(GbhError):
        h.set_rk_stages(4)
    h.set_telescoping(True)
    with pytest.raises(GbhError):
        h.set_rk_stages(3)            # telescoping three-stage needs 6 guard cells
    h.set_telescoping(False)
    h.set_rk_stages(3)
    with pytest.raises(GbhError):
        h.set_telescoping(True)
    U = dev(wl.random_state(lat, seed=2))
    h.step_adjoint(U, 1e-4, torch.zeros_like(U))          # the three-stage adjoint
    with pytest.raises(GbhError):                          # the stored-state form is two-stage only
        h.step_adjoint(U, 1e-4, torch.zeros_like(U), U1=U.clone())
    h.set_rk_stages(2)
    h.step_adjoint(U, 1e-4, torch.zeros_like(U), U1=U.clone())
