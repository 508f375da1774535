"""Pins of the oracle's two-level grid when the refined coarse blocks are not
a box (an L shape, a notch whose coarse block borders the fine region through
three faces, blocks touching at a corner, a 3-D tripod): conservation to
round-off on periodic domains with the all-levels flux correction (and a loss
without it), uniform flow kept uniform, linear data prolonged exactly, the
transpose symmetry of symmetric regions, and a box listed block by block
giving the box's bits.  Paramesh-style all-levels updates of Sec. 4.2 on
whole refined blocks; reading C9 for the level transfer."""
import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle2

L2 = [(1, 1), (2, 1), (3, 1), (1, 2), (1, 3)]              # L: block (2, 2) borders it through 2 faces
NOTCH2 = [(1, 1), (2, 1), (3, 1), (1, 2), (3, 2)]          # block (2, 2) borders it through 3 faces
DIAG2 = [(1, 1), (2, 2)]                                   # fine blocks touching at a corner
TRIPOD3 = [(1, 1, 1), (2, 1, 1), (1, 2, 1), (1, 1, 2)]


def grid2(blocks, bc="periodic"):
    return wl.two_level_blocks(wl.lattice_2d(5, 5, 8, 8, 4, bc=bc), blocks)


def grid3(blocks, bc="periodic"):
    return wl.two_level_blocks(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4, bc=bc), blocks)


GRIDS = [("L2", lambda bc="periodic": grid2(L2, bc)), ("notch2", lambda bc="periodic": grid2(NOTCH2, bc)),
         ("diag2", lambda bc="periodic": grid2(DIAG2, bc)), ("tripod3", lambda bc="periodic": grid3(TRIPOD3, bc))]


def leaf_totals(U, tl):
    """Sum over leaf cells (uncovered coarse blocks, existing fine blocks) of U x cell volume."""
    c, f = tl.coarse, tl.fine
    zs, ys, xs = c.interior_slices()
    vc, vf = np.prod(c.dx[: c.ndim]), np.prod(f.dx[: f.ndim])
    tot = np.zeros(5)
    for b in range(tl.n0):
        if not tl.covered(b):
            tot += U[b][:, zs, ys, xs].sum(axis=(1, 2, 3)) * vc
    for fb in range(tl.n1):
        if tl.fine_exists(fb):
            tot += U[tl.n0 + fb][:, zs, ys, xs].sum(axis=(1, 2, 3)) * vf
    return tot


def smooth_state(tl, seed):
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


def test_region_geometry():
    tl = grid2(NOTCH2)
    assert tl.lo == (1, 1, 0) and tl.hi == (4, 3, 1)
    assert sum(tl.covered(b) for b in range(tl.n0)) == 5
    assert sum(tl.fine_exists(f) for f in range(tl.n1)) == 5 * 4
    assert len(tl.gpu_blocks) == tl.n0 + 20
    assert tl.leaf_cells == (25 - 5 + 20) * 64
    with pytest.raises(ValueError):
        grid2([(0, 1)])                       # at the domain edge
    box = wl.two_level(wl.lattice_2d(5, 5, 8, 8, 4), (1, 1), (3, 3))
    assert np.array_equal(box.gpu_blocks, np.arange(box.nblocks))


@pytest.mark.parametrize("ndim", [2, 3])
def test_box_listed_block_by_block_gives_the_box(ndim):
    if ndim == 2:
        c = wl.lattice_2d(5, 5, 8, 8, 4)
        box, listed = wl.two_level(c, (1, 1), (3, 4)), wl.two_level_blocks(c, [(i, j) for i in (1, 2) for j in (1, 2, 3)])
    else:
        c = wl.lattice_3d(4, 4, 4, 8, 8, 8, 4)
        box = wl.two_level(c, (1, 1, 1), (3, 3, 2))
        listed = wl.two_level_blocks(c, [(i, j, 1) for i in (1, 2) for j in (1, 2)])
    assert box.lo == listed.lo and box.hi == listed.hi
    U = smooth_state(box, 2)
    A, B = U.copy(), U.copy()
    ha, _ = Oracle2(box).run(A, 4)
    hb, _ = Oracle2(listed).run(B, 4)
    assert np.array_equal(ha, hb) and np.array_equal(A, B)


@pytest.mark.parametrize("name,mk", GRIDS)
def test_conservation_with_flux_correction(name, mk):
    """Periodic composite grid, smooth data: leaf totals change by round-off
    over 8 steps; one stage without the flux correction loses mass and energy.
    A coarse cell next to two or three refined faces takes every face's
    correction, so a missing or doubled one shows here."""
    tl = mk()
    U = smooth_state(tl, 4)
    o = Oracle2(tl)
    o.restrict(U)
    t0 = leaf_totals(U, tl)
    scale = leaf_totals(np.abs(U), tl)
    hist, hits = o.run(U, 8)
    assert hits == 0
    d = np.abs(leaf_totals(U, tl) - t0)
    assert np.all(d <= 8 * 64 * np.finfo(float).eps * scale), d / scale
    dt = o.compute_dt(U)
    t1 = leaf_totals(U, tl)
    V, Vout, W, Wout = U.copy(), U.copy(), U.copy(), U.copy()
    o.stage(V, None, Vout, dt, 0.0, 1.0, reflux=False)
    o.stage(W, None, Wout, dt, 0.0, 1.0, reflux=True)
    assert np.all(np.abs(leaf_totals(Wout, tl) - t1) <= 64 * np.finfo(float).eps * scale)
    loss = np.abs(leaf_totals(Vout, tl) - t1)
    assert np.max(loss[[0, 4]] / scale[[0, 4]]) > 1e-12


@pytest.mark.parametrize("name,mk", GRIDS)
def test_uniform_flow_stays_uniform(name, mk):
    tl = mk()
    st = (1.25, 0.5, -0.25, 0.125 if tl.coarse.ndim == 3 else 0.0, 2.0)
    U = wl.two_level_state(tl, lambda X, Y, Z: tuple(v + 0 * X for v in st))
    U0 = U.copy()
    Oracle2(tl).run(U, 3)
    zs, ys, xs = tl.coarse.interior_slices()
    for b in tl.gpu_blocks:
        if b < tl.n0 and tl.covered(b):
            continue
        assert np.max(np.abs(U[b][:, zs, ys, xs] - U0[b][:, zs, ys, xs])) <= 1e-14 * np.max(np.abs(U0))


@pytest.mark.parametrize("name,mk", GRIDS)
def test_linear_field_prolonged_exactly(name, mk):
    """Linear data: MC slopes equal the gradient, so every fine guard cell
    filled from the coarse level gets the linear function's value (the same
    level's copies are exact anyway)."""
    tl = mk("outflow")
    a = (0.3, -0.2, 0.15)
    nd = tl.coarse.ndim
    lin = lambda X, Y, Z: 2.0 + a[0] * X + a[1] * Y + (a[2] * Z if nd == 3 else 0.0)
    U = wl.two_level_state(tl, lambda X, Y, Z: (lin(X, Y, Z), 0 * X, 0 * X, 0 * X, lin(X, Y, Z)))
    Uf = U.copy()
    Uf[tl.n0:] = wl.poison_guards(U[tl.n0:], tl.fine, np.nan)
    Oracle2(tl).fill(Uf)
    X, Y, Z = wl.cell_centers(tl.fine)
    expect = lin(X, Y, Z)
    guard = np.isnan(wl.poison_guards(U[tl.n0:], tl.fine, np.nan)[:, 0])
    exists = np.array([tl.fine_exists(f) for f in range(tl.n1)])
    sel = guard & exists[:, None, None, None]
    got = Uf[tl.n0:, 0][sel]
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - expect[sel])) < 5e-15


@pytest.mark.parametrize("blocks", [L2, NOTCH2, DIAG2])
def test_transpose_symmetry(blocks):
    """A region symmetric under x <-> y (L2, DIAG2) or mirrored (NOTCH2 under
    x -> -x about the middle of its bounding box) and data with the same
    symmetry stay symmetric: the flux correction's faces and tangential
    indices are placed the same way in every direction."""
    tl = grid2(blocks, "outflow")
    sym = sorted(blocks) == sorted((j, i) for i, j in blocks)
    nx = tl.coarse.nb[0] * tl.coarse.n[0]
    cx = (tl.lo[0] + tl.hi[0]) / 2 * tl.coarse.n[0] * tl.coarse.dx[0]
    cy = (tl.lo[1] + tl.hi[1]) / 2 * tl.coarse.n[1] * tl.coarse.dx[1]
    r0 = 0.12

    def fn(X, Y, Z):
        r2 = (X - cx) ** 2 + (Y - cy) ** 2
        bump = np.exp(-r2 / r0 ** 2)
        return 1 + 0.5 * bump, 0 * X, 0 * X, 0 * X, 1 + 2.0 * bump
    U = wl.two_level_state(tl, fn)
    o = Oracle2(tl)
    o.run(U, 6)
    from tests.gridutil import to_global
    # compare on the coarse leaf level and on the fine level, as global arrays
    Gc = to_global(U[:tl.n0], tl.coarse)
    Gf = to_global(U[tl.n0:], tl.fine)
    cov = np.kron(tl.refined_mask().reshape(tl.coarse.nb[1], tl.coarse.nb[0]), np.ones((8, 8))) > 0
    ex = np.kron(np.array([tl.fine_exists(f) for f in range(tl.n1)]).reshape(tl.fine.nb[1], tl.fine.nb[0]),
                 np.ones((8, 8))) > 0
    if sym:
        # x <-> y: transpose the arrays and swap the momenta
        def mirror(G):
            return G[[0, 2, 1, 3, 4]].transpose(0, 1, 3, 2)
        c_ok, f_ok = ~cov, ex
        assert np.array_equal(c_ok, c_ok.T) and np.array_equal(f_ok, f_ok.T)
    else:
        sx = np.array([1, -1, 1, 1, 1.0])[:, None, None, None]

        def mirror(G):
            return sx * G[:, :, :, ::-1]
        assert abs(cx - 0.5 * nx * tl.coarse.dx[0]) < 1e-14
        c_ok, f_ok = ~cov, ex
        assert np.array_equal(c_ok, c_ok[:, ::-1]) and np.array_equal(f_ok, f_ok[:, ::-1])
    for G, ok in ((Gc, c_ok), (Gf, f_ok)):
        M = mirror(G)
        d = np.abs(M - G)[:, 0][:, ok]
        assert np.max(d) <= 1e-13 * np.max(np.abs(G))
