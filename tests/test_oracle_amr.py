"""Pins of the oracle's two-level composite grid (restriction, prolongation
into fine guard cells, all-levels flux correction): exact behaviour on
constant and linear data, conservation to round-off, symmetry."""
import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle2

G = 1.4


def leaf_totals(U, tl):
    """Sum over leaf cells of U * cell volume, per conserved variable."""
    c, f = tl.coarse, tl.fine
    zs, ys, xs = c.interior_slices()
    vc = np.prod(c.dx[: c.ndim])
    vf = np.prod(f.dx[: f.ndim])
    tot = np.zeros(5)
    for b in range(tl.n0):
        if not tl.covered(b):
            tot += U[b][:, zs, ys, xs].sum(axis=(1, 2, 3)) * vc
    tot += U[tl.n0:][:, :, zs, ys, xs].sum(axis=(0, 2, 3, 4)) * vf
    return tot


def tl3(bc="periodic", nb=4, n=8, lo=(1, 1, 1), hi=(3, 3, 3)):
    return wl.two_level(wl.lattice_3d(nb, nb, nb, n, n, n, 4, bc=bc), lo, hi)


def tl2(bc="periodic"):
    return wl.two_level(wl.lattice_2d(4, 4, 8, 8, 4, bc=bc), (1, 1), (3, 3))


def test_geometry():
    tl = wl.two_level(wl.lattice_3d(16, 16, 16), (4, 4, 4), (12, 12, 12))
    assert tl.n0 == 4096 and tl.n1 == 4096
    assert tl.leaf_cells == 256 ** 3 * 7 // 8 + 256 ** 3
    assert tl.fine.dx[0] == 1.0 / 512 and tl.fine.origin == (0.25, 0.25, 0.25)


@pytest.mark.parametrize("mk", [tl3, tl2])
def test_restriction_is_mean_of_children(mk):
    tl = mk()
    U = wl.two_level_state(tl, lambda X, Y, Z: (1 + 0.3 * np.sin(7 * X + 3 * Y + Z), 0.1 + 0 * X, 0.2 * Y, -0.1 + 0 * X,
                                                  1 + 0.5 * np.cos(5 * Y)))
    o = Oracle2(tl)
    R = U.copy()
    o.restrict(R)
    c, f = tl.coarse, tl.fine
    nd = c.ndim
    zs, ys, xs = c.interior_slices()
    # independent: assemble the fine level globally and average 2^d blocks
    from tests.gridutil import to_global
    Ff = to_global(U[tl.n0:], f)
    if nd == 3:
        Rf = Ff.reshape(5, Ff.shape[1] // 2, 2, Ff.shape[2] // 2, 2, Ff.shape[3] // 2, 2).mean(axis=(2, 4, 6))
    else:
        Rf = Ff.reshape(5, 1, Ff.shape[2] // 2, 2, Ff.shape[3] // 2, 2).mean(axis=(3, 5))
    n = c.n
    for b in range(tl.n0):
        if not tl.covered(b):
            assert np.array_equal(R[b], U[b])
            continue
        bi, bj, bk = c.block_coords(b)
        sl = (slice(None),
              slice((bk - tl.lo[2]) * n[2], (bk - tl.lo[2] + 1) * n[2]) if nd == 3 else slice(0, 1),
              slice((bj - tl.lo[1]) * n[1], (bj - tl.lo[1] + 1) * n[1]),
              slice((bi - tl.lo[0]) * n[0], (bi - tl.lo[0] + 1) * n[0]))
        assert np.allclose(R[b][:, zs, ys, xs], Rf[sl], rtol=2e-16 * 8, atol=0)


@pytest.mark.parametrize("mk", [tl3, tl2])
def test_linear_field_prolonged_exactly(mk):
    """Linear data: MC slopes equal the exact gradient, so the fine guard cells
    across the coarse-fine boundary receive the linear function's values."""
    tl = mk("outflow")
    a = (0.3, -0.2, 0.15)
    lin = lambda X, Y, Z: 2.0 + a[0] * X + a[1] * Y + (a[2] * Z if tl.coarse.ndim == 3 else 0.0)
    U = wl.two_level_state(tl, lambda X, Y, Z: (lin(X, Y, Z), 0 * X, 0 * X, 0 * X, lin(X, Y, Z)))
    Uf = U.copy()
    Uf[tl.n0:] = wl.poison_guards(U[tl.n0:], tl.fine, np.nan)
    Oracle2(tl).fill(Uf)
    X, Y, Z = wl.cell_centers(tl.fine)
    expect = lin(X, Y, Z)
    got = Uf[tl.n0:, 0]
    # face regions of fine blocks on the fine-region boundary
    mask = ~np.isnan(wl.poison_guards(U[tl.n0:], tl.fine, np.nan, corners_only=False)[:, 0])
    sel = ~mask  # guard cells
    err = np.nanmax(np.abs(got[sel] - expect[sel]))
    assert err < 5e-15, err


@pytest.mark.parametrize("mk", [tl3, tl2])
def test_uniform_flow_stays_uniform(mk):
    tl = mk()
    st = (1.25, 0.5, -0.25, 0.125 if tl.coarse.ndim == 3 else 0.0, 2.0)
    U = wl.two_level_state(tl, lambda X, Y, Z: tuple(v + 0 * X for v in st))
    U0 = U.copy()
    Oracle2(tl).run(U, 3)
    zs, ys, xs = tl.coarse.interior_slices()
    for b in range(tl.nblocks):
        if b < tl.n0 and tl.covered(b):
            continue
        assert np.max(np.abs(U[b][:, zs, ys, xs] - U0[b][:, zs, ys, xs])) <= 1e-14 * np.max(np.abs(U0))


@pytest.mark.parametrize("mk", [tl3, tl2])
def test_conservation_with_flux_correction(mk):
    """Periodic composite grid, random smooth data: leaf totals change by
    round-off only; without the flux correction they do not."""
    tl = mk()
    rng = np.random.default_rng(4)
    ph = rng.uniform(0, 2 * np.pi, 8)
    def fn(X, Y, Z):
        s = np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1])
        if tl.coarse.ndim == 3:
            s = s * np.cos(2 * np.pi * Z + ph[2])
        return (1 + 0.4 * s, 0.5 * np.sin(2 * np.pi * Y + ph[3]) + 0 * X, 0.4 * np.cos(2 * np.pi * X + ph[4]),
                (0.3 * np.sin(2 * np.pi * X + ph[5]) if tl.coarse.ndim == 3 else 0 * X), 1 + 0.3 * s)
    U = wl.two_level_state(tl, fn)
    o = Oracle2(tl)
    o.restrict(U)
    t0 = leaf_totals(U, tl)
    scale = leaf_totals(np.abs(U), tl)
    hist, hits = o.run(U, 10)
    assert hits == 0
    d = np.abs(leaf_totals(U, tl) - t0)
    assert np.all(d <= 10 * 64 * np.finfo(float).eps * scale), d / scale
    # one stage without the correction is not conservative
    V = U.copy()
    Vout = U.copy()
    W = U.copy()
    Wout = U.copy()
    dt = o.compute_dt(U)
    o.stage(V, None, Vout, dt, 0.0, 1.0, reflux=False)
    o.stage(W, None, Wout, dt, 0.0, 1.0, reflux=True)
    t1 = leaf_totals(U, tl)
    loss = np.abs(leaf_totals(Vout, tl) - t1)
    keep = np.abs(leaf_totals(Wout, tl) - t1)
    assert np.all(keep <= 64 * np.finfo(float).eps * scale)
    assert np.max(loss[[0, 4]] / scale[[0, 4]]) > 1e-12


def test_two_level_sedov_symmetry_and_energy():
    tl = wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4), (1, 1, 1), (3, 3, 3))
    U = wl.sedov_two_level(tl)
    o = Oracle2(tl)
    o.restrict(U)
    E0 = leaf_totals(U, tl)[4]
    hist, hits = o.run(U, 15)
    assert hits == 0
    assert abs(leaf_totals(U, tl)[4] / E0 - 1) < 1e-13
    from tests.gridutil import to_global
    Ff = to_global(U[tl.n0:], tl.fine)
    sgn = np.array([1, -1, 1, 1, 1.0])[:, None, None, None]
    mir = sgn * Ff[:, :, :, ::-1]
    assert np.max(np.abs(mir - Ff)) <= 1e-10 * np.max(np.abs(Ff))
