"""Pins of the oracle's level-by-level telescoping step on the two-level grid
(Sec. 4.2, Fig. "Level-by-levels, Telescoping"): one guard fill, each level's
blocks through both stages on their own guard data, the coarse side
corrected with the fine fluxes, restriction.

References: conservation of the leaf totals on periodic grids (which the
flux correction must restore exactly); the single-level oracle stage (pinned
separately), run on each level's blocks from the same filled data, for every
cell the correction does not touch; uniform flow; Sedov symmetry.
"""
import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle, Oracle2
from tests.test_oracle_amr import leaf_totals, tl2, tl3


def smooth(tl):
    rng = np.random.default_rng(14)
    ph = rng.uniform(0, 2 * np.pi, 8)
    nd = tl.coarse.ndim

    def fn(X, Y, Z):
        s = np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1])
        if nd == 3:
            s = s * np.cos(2 * np.pi * Z + ph[2])
        return (1 + 0.4 * s, 0.5 * np.sin(2 * np.pi * Y + ph[3]) + 0 * X, 0.4 * np.cos(2 * np.pi * X + ph[4]),
                (0.3 * np.sin(2 * np.pi * X + ph[5]) if nd == 3 else 0 * X), 1 + 0.3 * s)
    return wl.two_level_state(tl, fn)


@pytest.mark.parametrize("mk", [tl3, tl2])
def test_conservation(mk):
    tl = mk()
    U = smooth(tl)
    o = Oracle2(tl)
    o.restrict(U)
    t0 = leaf_totals(U, tl)
    scale = leaf_totals(np.abs(U), tl)
    _, hits = o.run(U, 10, telescoping=True)
    assert hits == 0
    d = np.abs(leaf_totals(U, tl) - t0)
    assert np.all(d <= 10 * 64 * np.finfo(float).eps * scale), d / scale


def cf_adjacent(tl):
    """Mask of the coarse leaf cells next to a face towards a covered block."""
    c = tl.coarse
    zs, ys, xs = c.interior_slices()
    m = np.zeros((tl.n0,) + tuple(c.n[::-1]), dtype=bool)
    for b in range(tl.n0):
        if tl.covered(b):
            continue
        bc = c.block_coords(b)
        for d in range(c.ndim):
            for side in (0, 1):
                nc = list(bc)
                nc[d] += 1 if side else -1
                if not 0 <= nc[d] < c.nb[d]:
                    if c.bc[d] != "periodic":
                        continue
                    nc[d] %= c.nb[d]
                nb = nc[0] + c.nb[0] * (nc[1] + c.nb[1] * nc[2])
                if tl.covered(nb):
                    idx = [slice(None)] * 3
                    idx[2 - d] = c.n[d] - 1 if side else 0
                    m[(b,) + tuple(idx)] = True
    return m


@pytest.mark.parametrize("mk,bc", [(tl3, "outflow"), (tl2, "periodic"), (tl2, "outflow")])
def test_levels_equal_single_level_stages_on_the_filled_data(mk, bc):
    """Each level's leaf blocks evolve exactly as the single-level telescoping
    stages on the data of the one fill; only the coarse cells next to the
    fine region change further, by the flux correction."""
    tl = mk(bc)
    U0 = smooth(tl)
    o2 = Oracle2(tl)
    o2.restrict(U0)
    dt = 0.5 * o2.compute_dt(U0)
    U = U0.copy()
    o2.step(U, dt, telescoping=True)
    F = U0.copy()
    o2.fill(F)
    zs, ys, xs = tl.coarse.interior_slices()
    for lev, (lat, sl) in enumerate(((tl.coarse, slice(0, tl.n0)), (tl.fine, slice(tl.n0, tl.nblocks)))):
        o = Oracle(lat)
        Ul = np.ascontiguousarray(F[sl])
        U1 = Ul.copy()
        o.stage(Ul, None, U1, dt, 0.0, 1.0, ext=2)
        U2 = U1.copy()
        o.stage(U1, Ul, U2, dt, 0.5, 0.5)
        got, ref = U[sl][:, :, zs, ys, xs], U2[:, :, zs, ys, xs]
        if lev == 1:
            assert np.array_equal(got, ref)
        else:
            leaf = np.array([not tl.covered(b) for b in range(tl.n0)])
            adj = cf_adjacent(tl)
            keep = leaf[:, None, None, None] & ~adj
            assert np.array_equal(np.moveaxis(got, 1, -1)[keep], np.moveaxis(ref, 1, -1)[keep])
            assert not np.array_equal(np.moveaxis(got, 1, -1)[adj], np.moveaxis(ref, 1, -1)[adj])


@pytest.mark.parametrize("mk", [tl3, tl2])
def test_uniform_flow_stays_uniform(mk):
    tl = mk()
    st = (1.25, 0.5, -0.25, 0.125 if tl.coarse.ndim == 3 else 0.0, 2.0)
    U = wl.two_level_state(tl, lambda X, Y, Z: tuple(v + 0 * X for v in st))
    U0 = U.copy()
    Oracle2(tl).run(U, 3, telescoping=True)
    zs, ys, xs = tl.coarse.interior_slices()
    for b in range(tl.nblocks):
        if b < tl.n0 and tl.covered(b):
            continue
        assert np.max(np.abs(U[b][:, zs, ys, xs] - U0[b][:, zs, ys, xs])) <= 1e-14 * np.max(np.abs(U0))


def test_sedov_symmetry_and_energy():
    tl = wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4), (1, 1, 1), (3, 3, 3))
    U = wl.sedov_two_level(tl)
    o = Oracle2(tl)
    o.restrict(U)
    E0 = leaf_totals(U, tl)[4]
    _, hits = o.run(U, 15, telescoping=True)
    assert hits == 0
    assert abs(leaf_totals(U, tl)[4] / E0 - 1) < 1e-13
    from tests.gridutil import to_global
    Ff = to_global(U[tl.n0:], tl.fine)
    sgn = np.array([1, -1, 1, 1, 1.0])[:, None, None, None]
    assert np.max(np.abs(sgn * Ff[:, :, :, ::-1] - Ff)) <= 1e-10 * np.max(np.abs(Ff))


def test_close_to_all_levels_variant():
    """Both variants are second-order consistent with the same scheme: on
    smooth data their difference after a few steps is far below the change."""
    tl = tl2()
    U = smooth(tl)
    o = Oracle2(tl)
    o.restrict(U)
    A, B = U.copy(), U.copy()
    o.run(A, 4)
    o.run(B, 4, telescoping=True)
    zs, ys, xs = tl.coarse.interior_slices()
    leaf = [b for b in range(tl.nblocks) if not (b < tl.n0 and tl.covered(b))]
    diff = np.max(np.abs(A[leaf][:, :, zs, ys, xs] - B[leaf][:, :, zs, ys, xs]))
    change = np.max(np.abs(A[leaf][:, :, zs, ys, xs] - U[leaf][:, :, zs, ys, xs]))
    assert 0 < diff < 0.05 * change, (diff, change)


def test_needs_four_guard_cells():
    tl = wl.two_level(wl.lattice_2d(4, 4, 8, 8, 3, bc="periodic"), (1, 1), (3, 3))
    U = smooth(tl)
    with pytest.raises(ValueError):
        Oracle2(tl).step(U, 1e-4, telescoping=True)
