"""Batched ensembles (gbh_create_batched), the CUDA-graph advance and the
stage-kernel work decomposition (gbh_autotune / gbh_set_decomposition)."""
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


def split(U, lats):
    out, o = [], 0
    for l in lats:
        out.append(U[o:o + l.nblocks])
        o += l.nblocks
    return out


def small_ensemble():
    probs = wl.ensemble(count=6, seed=3, choices=(32, 64, 128))
    return [l for l, _ in probs], np.concatenate([u for _, u in probs])


def test_batched_ensemble_matches_oracle_per_problem(gb):
    lats, U0 = small_ensemble()
    nsteps = 30
    h = gb.Hydro.from_batch(lats)
    Ug = dev(U0)
    dt = h.compute_dt(Ug)
    hist = torch.zeros(nsteps * len(lats), dtype=torch.float64, device="cuda")
    h.advance(Ug, nsteps, dt, hist)
    hist = host(hist).reshape(nsteps, len(lats))
    for i, (lat, Ui, Uo) in enumerate(zip(lats, split(host(Ug), lats), split(U0, lats))):
        ref = Uo.copy()
        hist_o, hits = Oracle(lat).run(ref, nsteps)
        assert np.max(np.abs(hist[:, i] / hist_o - 1)) <= 1e-12
        assert np.all(relerr_per_var(to_global(Ui, lat), to_global(ref, lat)) <= 1e-11)


def test_batched_equals_separate_contexts_bitwise(gb):
    lats, U0 = small_ensemble()
    h = gb.Hydro.from_batch(lats)
    Ug = dev(U0)
    dt = h.compute_dt(Ug)
    h.advance(Ug, 5, dt)
    for lat, Ui, Uo in zip(lats, split(host(Ug), lats), split(U0, lats)):
        hs = gb.Hydro.from_lattice(lat)
        Us = dev(Uo)
        d = hs.compute_dt(Us)
        hs.advance(Us, 5, d)
        zs, ys, xs = lat.interior_slices()
        assert np.array_equal(host(Us)[:, :, zs, ys, xs], Ui[:, :, zs, ys, xs])


def test_graph_advance_bitwise_equal_to_plain(gb):
    lats, U0 = small_ensemble()
    h = gb.Hydro.from_batch(lats)
    A, B = dev(U0), dev(U0)
    da, db = h.compute_dt(A), h.compute_dt(B)
    h.advance(A, 12, da)
    h.advance_graph(B, 6, db)
    h.advance_graph(B, 6, db)      # replays the cached graph
    assert torch.equal(A, B) and torch.equal(da, db)


@pytest.mark.parametrize("kchunk,ipc", [(8, 1), (16, 2), (8, 4), (0, 37), (4, 3)])
def test_decomposition_does_not_change_results(gb, kchunk, ipc):
    lat = wl.lattice_3d(3, 2, 2, 16, 16, 16, 4)
    U0 = wl.sedov(lat)
    h = gb.Hydro.from_lattice(lat)
    A = dev(U0)
    da = h.compute_dt(A)
    h.advance(A, 3, da)
    h.set_decomposition(kchunk, ipc)
    B = dev(U0)
    db = h.compute_dt(B)
    h.advance(B, 3, db)
    zs, ys, xs = lat.interior_slices()
    assert torch.equal(A[:, :, zs, ys, xs], B[:, :, zs, ys, xs]) and torch.equal(da, db)


def test_autotune_and_refined_decomposition(gb):
    lat = wl.lattice_3d(4, 4, 4, 16, 16, 16, 4)
    U0 = wl.sedov(lat)
    h = gb.Hydro.from_lattice(lat)
    U = dev(U0)
    kc, ipc = h.autotune(U)
    assert kc in (8, 16) and ipc >= 1
    assert torch.equal(U, dev(U0))            # autotune leaves U untouched
    tl = wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4), (1, 1, 1), (3, 3, 3))
    V0 = wl.sedov_two_level(tl)
    hr = gb.Hydro.from_two_level(tl)
    A = dev(V0)
    hr.fill_guardcells(A)
    B = A.clone()
    da = hr.compute_dt(A)
    hr.advance(A, 3, da)
    hr.autotune(B)
    db = hr.compute_dt(B)
    hr.advance(B, 3, db)
    assert torch.equal(da, db)


def _split_case(case):
    """(context factory, initial state, rings the case's steps use)"""
    if case in ("3d", "telescoping_rk2", "telescoping_rk3", "2d"):
        ng = 6 if case == "telescoping_rk3" else 4
        lat = (wl.lattice_2d(3, 2, 16, 16, ng, bc=("periodic", "outflow")) if case == "2d" else
               wl.lattice_3d(2, 3, 2, 16, 16, 16, ng, bc=("outflow", "periodic", "outflow")))
        U0 = wl.random_state(lat, seed=61, rough=True)

        def make():
            h = gb_pkg().Hydro.from_lattice(lat)
            if case == "telescoping_rk3":
                h.set_rk_stages(3)
            h.set_telescoping(case.startswith("telescoping"))
            return h
        rings = {"telescoping_rk2": (0, 2), "telescoping_rk3": (0, 2, 4)}.get(case, (0,))
        return make, U0, rings, lat.interior_slices()
    if case in ("two_level", "two_level_lbl"):
        tl = wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4), (1, 1, 1), (3, 3, 3))
        U0 = wl.sedov_two_level(tl)

        def make():
            h = gb_pkg().Hydro.from_two_level(tl)
            h.set_telescoping(case == "two_level_lbl")
            return h
        return make, U0, ((0, 2) if case == "two_level_lbl" else (0,)), tl.coarse.interior_slices()
    lats, U0 = small_ensemble()
    return (lambda: gb_pkg().Hydro.from_batch(lats)), U0, (0,), lats[0].interior_slices()


def gb_pkg():
    import paper_2401_03378_gb300 as pkg
    return pkg


@pytest.mark.parametrize("case", ["3d", "2d", "telescoping_rk2", "telescoping_rk3", "two_level", "two_level_lbl",
                                  "batched"])
def test_tile_split_does_not_change_results(gb, case):
    """The stage kernel's plane tile cut into two row bands (one CTA each), on
    the interior stage and on every ring stage the mode uses, alone and with
    z-chunks and several items per CTA: the same state and dt bit for bit."""
    make, U0, rings, sl = _split_case(case)
    zs, ys, xs = sl
    results = []
    for split, kc, ipc in ((1, 0, 1), (2, 0, 1), (2, 8, 3)):
        h = make()
        for r in rings:
            h.set_tile_split(r, split)
        if kc or ipc != 1:
            h.set_decomposition(kc if h.ndim == 3 else 0, ipc)
        assert all(h.tile_split(r) == split for r in rings)
        U = dev(U0)
        if h.refined:
            h.fill_guardcells(U)
        dt = h.compute_dt(U)
        h.advance(U, 3, dt)
        results.append((host(U)[:, :, zs, ys, xs], host(dt), h.floor_hits()))
        h.close()
    for U, dt, hits in results[1:]:
        assert np.array_equal(U, results[0][0]) and np.array_equal(dt, results[0][1])
        assert hits == results[0][2]


def test_tile_split_rejections(gb):
    h = gb.Hydro.from_lattice(wl.lattice_3d(2, 2, 2, 4, 4, 4, 4))
    with pytest.raises(gb.GbhError):
        h.set_tile_split(0, 2)          # bands of 2 rows are not built
    h2 = gb.Hydro.from_lattice(wl.lattice_3d(2, 2, 2, 8, 8, 8, 4))
    for ring, split in ((1, 1), (0, 3), (6, 1)):
        with pytest.raises(gb.GbhError):
            h2.set_tile_split(ring, split)
    h2.set_tile_split(4, 2)
    assert h2.tile_split(4) == 2 and h2.tile_split(0) == 1


def test_autotune_picks_tile_splits_for_ring_stages(gb):
    lat = wl.lattice_3d(2, 2, 2, 16, 16, 16, 6)
    U0 = wl.sedov(lat)
    h = gb.Hydro.from_lattice(lat)
    h.set_rk_stages(3)
    h.set_telescoping(True)
    U = dev(U0)
    h.autotune(U)
    assert torch.equal(U, dev(U0))
    assert all(h.tile_split(r) in (1, 2) for r in (0, 2, 4))
    ref = gb.Hydro.from_lattice(lat)
    ref.set_rk_stages(3)
    ref.set_telescoping(True)
    A, B = dev(U0), dev(U0)
    da, db = h.compute_dt(A), ref.compute_dt(B)
    h.advance(A, 2, da)
    ref.advance(B, 2, db)
    zs, ys, xs = lat.interior_slices()
    assert torch.equal(A[:, :, zs, ys, xs], B[:, :, zs, ys, xs]) and torch.equal(da, db)
