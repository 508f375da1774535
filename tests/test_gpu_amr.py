"""GPU parity of the two-level composite grid (gbh_create_refined) against the
oracle's two-level path: guard fill (restriction + prolongation + copies)
bitwise, single steps <= 1e-13, runs <= 1e-11, conservation with the flux
correction, and the 4096 + 4096-block Sedov variant sampled at its last step."""
import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle2
from tests.gridutil import relerr_per_var

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


def leaf_err(A, B, tl):
    """relative error per variable over the interiors of leaf blocks"""
    zs, ys, xs = tl.coarse.interior_slices()
    leaf = [b for b in range(tl.nblocks) if not (b < tl.n0 and tl.covered(b))]
    a = np.moveaxis(A[leaf][:, :, zs, ys, xs], 1, 0)
    b = np.moveaxis(B[leaf][:, :, zs, ys, xs], 1, 0)
    return relerr_per_var(a, b)


def smooth(tl, seed):
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, 8)
    nd = tl.coarse.ndim
    def fn(X, Y, Z):
        s = np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1])
        if nd == 3:
            s = s * np.cos(2 * np.pi * Z + ph[2])
        return (1 + 0.4 * s, 0.5 * np.sin(2 * np.pi * Y + ph[3]) + 0 * X, 0.4 * np.cos(2 * np.pi * X + ph[4]),
                (0.3 * np.sin(2 * np.pi * X + ph[5]) if nd == 3 else 0 * X), 1 + 0.3 * s)
    return wl.two_level_state(tl, fn)


GRIDS = [
    wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4, bc="periodic"), (1, 1, 1), (3, 3, 3)),
    wl.two_level(wl.lattice_3d(4, 3, 4, 8, 8, 8, 4), (1, 1, 2), (2, 2, 3)),
    wl.two_level(wl.lattice_3d(3, 3, 3, 16, 16, 16, 4), (1, 1, 1), (2, 2, 2)),
    wl.two_level(wl.lattice_2d(4, 4, 16, 16, 4, bc="periodic"), (1, 1), (3, 3)),
    wl.two_level(wl.lattice_2d(5, 4, 8, 8, 4), (1, 1), (4, 3)),
]


@pytest.mark.parametrize("tl", GRIDS)
def test_refined_fill_bitwise(gb, tl):
    U = smooth(tl, 1)
    U = np.concatenate([wl.poison_guards(U[:tl.n0], tl.coarse, np.nan),
                        wl.poison_guards(U[tl.n0:], tl.fine, np.nan)])
    ref = U.copy()
    Oracle2(tl).fill(ref)
    h = gb.Hydro.from_two_level(tl)
    Ug = dev(U)
    h.fill_guardcells(Ug)
    out = host(Ug)
    assert np.array_equal(np.isnan(out), np.isnan(ref))
    assert np.array_equal(np.nan_to_num(out), np.nan_to_num(ref))


@pytest.mark.parametrize("tl", GRIDS)
def test_refined_one_step(gb, tl):
    U = smooth(tl, 2)
    o = Oracle2(tl)
    o.restrict(U)
    dt = o.compute_dt(U)
    ref = U.copy()
    o.step(ref, dt)
    h = gb.Hydro.from_two_level(tl)
    Ug = dev(U)
    assert abs(float(host(h.compute_dt(Ug))[0]) / dt - 1) < 1e-14
    h.step(Ug, dt)
    out = host(Ug)
    assert np.all(leaf_err(out, ref, tl) <= 1e-13)
    # covered blocks hold the restriction of the new fine data
    cov = [b for b in range(tl.n0) if tl.covered(b)]
    zs, ys, xs = tl.coarse.interior_slices()
    a = np.moveaxis(out[cov][:, :, zs, ys, xs], 1, 0)
    b = np.moveaxis(ref[cov][:, :, zs, ys, xs], 1, 0)
    assert np.all(relerr_per_var(a, b) <= 1e-13)


def test_refined_sedov_trajectory(gb):
    """Two-level Sedov, coarse 128^3 (512 blocks of 16^3) + fine level over the
    central 64^3 coarse cells (512 fine blocks), 20 steps with device dt."""
    tl = wl.two_level(wl.lattice_3d(8, 8, 8), (2, 2, 2), (6, 6, 6))
    U0 = wl.sedov_two_level(tl)
    ref = U0.copy()
    hist_o, hits = Oracle2(tl).run(ref, 20)
    h = gb.Hydro.from_two_level(tl)
    Ug = dev(U0)
    h.fill_guardcells(Ug)                 # restriction of the initial data
    dt = h.compute_dt(Ug)
    hist = torch.zeros(20, dtype=torch.float64, device="cuda")
    h.advance(Ug, 20, dt, hist)
    assert np.max(np.abs(host(hist) / hist_o - 1)) <= 1e-12
    assert np.all(leaf_err(host(Ug), ref, tl) <= 1e-11)
    assert hits == 0 and h.floor_hits() == 0


def test_refined_conservation(gb):
    tl = GRIDS[0]
    U = smooth(tl, 3)
    o = Oracle2(tl)
    o.restrict(U)
    def totals(A):
        zs, ys, xs = tl.coarse.interior_slices()
        vc, vf = np.prod(tl.coarse.dx), np.prod(tl.fine.dx)
        t = np.zeros(5)
        for b in range(tl.nblocks):
            if b < tl.n0 and tl.covered(b):
                continue
            t += A[b][:, zs, ys, xs].sum(axis=(1, 2, 3)) * (vc if b < tl.n0 else vf)
        return t
    t0 = totals(U)
    scale = totals(np.abs(U))
    h = gb.Hydro.from_two_level(tl)
    Ug = dev(U)
    dt = h.compute_dt(Ug)
    h.advance(Ug, 10, dt)
    assert np.all(np.abs(totals(host(Ug)) - t0) <= 10 * 64 * np.finfo(float).eps * scale)


@pytest.mark.slow
def test_refined_sedov_4096_plus_4096_sampled(gb):
    """The two-level variant of the 256^3 Sedov workload (4096 coarse + 4096 fine
    blocks of 16^3) in the benchmark's launch configuration: step 50 against the
    oracle's step from the GPU state after 49 steps."""
    tl = wl.two_level(wl.lattice_3d(16, 16, 16), (4, 4, 4), (12, 12, 12))
    U0 = wl.sedov_two_level(tl)
    h = gb.Hydro.from_two_level(tl)
    Ug = dev(U0)
    h.fill_guardcells(Ug)
    dt = h.compute_dt(Ug)
    o = Oracle2(tl)
    first = U0.copy()
    o.restrict(first)
    assert abs(float(host(dt)[0]) / o.compute_dt(first) - 1) <= 1e-12
    h.advance(Ug, 49, dt)
    snap = host(Ug)
    dt_o = o.compute_dt(snap)
    assert abs(float(host(dt)[0]) / dt_o - 1) <= 1e-12
    ref = snap.copy()
    o.step(ref, dt_o)
    h.step(Ug, dt_o)
    assert np.all(leaf_err(host(Ug), ref, tl) <= 1e-13)
    assert h.floor_hits() == 0


def banded(tl, side, seed):
    """The smooth state with the pressure raised 30-fold in one layer of cells
    along the fine region's boundary, so that the largest CFL speeds sit there:
    side "coarse": the coarse cells just outside the box's faces (the cells the
    flux correction changes); "beside": the next coarse layer out (same
    blocks, not corrected); "fine": the first fine layer inside the box."""
    c = tl.coarse
    nd = c.ndim
    blk = [c.n[d] * c.dx[d] for d in range(nd)]
    lo = [tl.lo[d] * blk[d] for d in range(nd)]
    hi = [tl.hi[d] * blk[d] for d in range(nd)]
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, 8)

    def fn(X, Y, Z):
        P = (X, Y, Z)
        s = np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1])
        rho = 1 + 0.4 * s
        u = 0.5 * np.sin(2 * np.pi * Y + ph[3]) + 0 * X
        v = 0.4 * np.cos(2 * np.pi * X + ph[4])
        w = 0.3 * np.sin(2 * np.pi * X + ph[5]) if nd == 3 else 0 * X
        p = 1 + 0.3 * s
        od = [np.maximum(np.maximum(lo[d] - P[d], P[d] - hi[d]), 0) for d in range(nd)]
        one = np.sum([o > 0 for o in od], axis=0) == 1          # outside across one face only
        out = np.max(od, axis=0)
        inn = np.min([np.minimum(P[d] - lo[d], hi[d] - P[d]) for d in range(nd)], axis=0)
        if side == "coarse":
            band = one & (out < c.dx[0])
        elif side == "beside":
            band = one & (out > c.dx[0]) & (out < 2 * c.dx[0])
        else:
            band = (inn > 0) & (inn < 0.5 * c.dx[0])
        return rho, u, v, w, np.where(band, 30.0 * p, p)
    return wl.two_level_state(tl, fn)


@pytest.mark.parametrize("tl", [GRIDS[0], GRIDS[1], GRIDS[4]])
@pytest.mark.parametrize("side", ["coarse", "beside", "fine"])
@pytest.mark.parametrize("mode", ["all-levels", "level-by-level", "three-stage"])
def test_refined_step_dt_equals_a_separate_reduction(gb, tl, side, mode):
    """The CFL dt of a two-level step comes from the last stage's epilogue over
    the leaf cells the flux correction leaves alone and from the correction
    kernel over the cells it changes.  It must equal, bit for bit, a separate
    reduction over the final state, with the fastest cells on either side of
    the coarse-fine boundary."""
    U = banded(tl, side, 4)
    h = gb.Hydro.from_two_level(tl)
    if mode == "level-by-level":
        h.set_telescoping(True)
    if mode == "three-stage":
        h.set_rk_stages(3)
    Ug = dev(U)
    h.fill_guardcells(Ug)
    dt = h.compute_dt(Ug)
    for _ in range(4):
        h.step_cfl(Ug, dt)
        ref = h.compute_dt(Ug)
        assert host(dt)[0] == host(ref)[0]
    zs, ys, xs = tl.coarse.interior_slices()
    assert np.all(np.isfinite(host(Ug)[:, :, zs, ys, xs]))


def test_refined_batched_step_dt_equals_a_separate_reduction(gb):
    tls = [GRIDS[0], GRIDS[1]]
    parts = [banded(tls[0], "coarse", 5), banded(tls[1], "fine", 6)]
    h = gb.Hydro.from_two_level_batch(tls)
    Ug = dev(np.concatenate(parts))
    h.fill_guardcells(Ug)
    dt = h.compute_dt(Ug)
    for _ in range(3):
        h.step_cfl(Ug, dt)
        assert np.array_equal(host(dt), host(h.compute_dt(Ug)))
