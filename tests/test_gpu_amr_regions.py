"""GPU parity of two-level grids whose refined coarse blocks are not a box (an
L, a notch whose coarse block borders the fine region through three faces,
blocks touching at a corner, a 3-D tripod, an L of 16^3 blocks) against the
oracle's two-level path: the guard fill bitwise, one step <= 1e-13 in the
all-levels, level-by-level telescoping and three-stage variants, 20-step runs
<= 1e-11 with the dt history <= 1e-12, conservation with the flux correction,
and the step's CFL dt bitwise equal to a separate reduction with the fastest
cells at the inner corner, where one coarse cell takes two or three
corrections.  The library's state holds only the fine blocks that exist
(workloads.TwoLevel.gpu_blocks maps it onto the oracle's arrays)."""
import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle2
from tests.gridutil import relerr_per_var

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L2 = [(1, 1), (2, 1), (3, 1), (1, 2), (1, 3)]
NOTCH2 = [(1, 1), (2, 1), (3, 1), (1, 2), (3, 2)]
DIAG2 = [(1, 1), (2, 2)]
TRIPOD3 = [(1, 1, 1), (2, 1, 1), (1, 2, 1), (1, 1, 2)]


def grids(bc="outflow"):
    return [wl.two_level_blocks(wl.lattice_2d(5, 5, 8, 8, 4, bc=bc), L2),
            wl.two_level_blocks(wl.lattice_2d(5, 5, 8, 8, 4, bc=bc), NOTCH2),
            wl.two_level_blocks(wl.lattice_2d(5, 5, 16, 16, 4, bc=bc), DIAG2),
            wl.two_level_blocks(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4, bc=bc), TRIPOD3),
            wl.two_level_blocks(wl.lattice_3d(4, 4, 3, 16, 16, 16, 4, bc=bc), [(1, 1, 1), (2, 1, 1), (1, 2, 1)])]


GRIDS = grids()
IDS = ["L2", "notch2", "diag2-16", "tripod3", "L3-16"]


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


def leaf_err(G, O, tl):
    """Relative error per variable over the interiors of leaf blocks; G in
    the library's layout, O in the oracle's."""
    zs, ys, xs = tl.coarse.interior_slices()
    blocks = tl.gpu_blocks
    leaf = [i for i, b in enumerate(blocks) if not (b < tl.n0 and tl.covered(b))]
    a = np.moveaxis(G[leaf][:, :, zs, ys, xs], 1, 0)
    b = np.moveaxis(O[blocks[leaf]][:, :, zs, ys, xs], 1, 0)
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


@pytest.mark.parametrize("tl", GRIDS, ids=IDS)
def test_fill_bitwise(gb, tl):
    U = smooth(tl, 1)
    U = np.concatenate([wl.poison_guards(U[:tl.n0], tl.coarse, np.nan),
                        wl.poison_guards(U[tl.n0:], tl.fine, np.nan)])
    ref = U.copy()
    Oracle2(tl).fill(ref)
    h = gb.Hydro.from_two_level(tl)
    Ug = dev(U[tl.gpu_blocks])
    h.fill_guardcells(Ug)
    out = host(Ug)
    exp = ref[tl.gpu_blocks]
    assert np.array_equal(np.isnan(out), np.isnan(exp))
    assert np.array_equal(np.nan_to_num(out), np.nan_to_num(exp))


@pytest.mark.parametrize("mode", ["all-levels", "level-by-level", "three-stage"])
@pytest.mark.parametrize("tl", GRIDS, ids=IDS)
def test_one_step(gb, tl, mode):
    tele, stages = mode == "level-by-level", 3 if mode == "three-stage" else 2
    U = smooth(tl, 2)
    o = Oracle2(tl)
    o.restrict(U)
    dt = o.compute_dt(U)
    ref = U.copy()
    o.step(ref, dt, telescoping=tele, stages=stages)
    h = gb.Hydro.from_two_level(tl)
    h.set_rk_stages(stages)
    h.set_telescoping(tele)
    Ug = dev(U[tl.gpu_blocks])
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


@pytest.mark.parametrize("tl", GRIDS, ids=IDS)
def test_twenty_step_run(gb, tl):
    U = smooth(tl, 3)
    ref = U.copy()
    hist_o, hits = Oracle2(tl).run(ref, 20)
    h = gb.Hydro.from_two_level(tl)
    Ug = dev(U[tl.gpu_blocks])
    h.fill_guardcells(Ug)
    dt = h.compute_dt(Ug)
    hist = torch.zeros(20, dtype=torch.float64, device="cuda")
    h.advance(Ug, 20, dt, hist)
    assert np.max(np.abs(host(hist) / hist_o - 1)) <= 1e-12
    assert np.all(leaf_err(host(Ug), ref, tl) <= 1e-11)
    assert hits == 0 and h.floor_hits() == 0


def leaf_totals(G, tl):
    """Leaf totals (cell volume weighted) of a state in the library's layout."""
    c, f = tl.coarse, tl.fine
    zs, ys, xs = c.interior_slices()
    vc, vf = np.prod(c.dx[: c.ndim]), np.prod(f.dx[: f.ndim])
    t = np.zeros(5)
    for i, b in enumerate(tl.gpu_blocks):
        if b < tl.n0 and tl.covered(b):
            continue
        t += G[i][:, zs, ys, xs].sum(axis=(1, 2, 3)) * (vc if b < tl.n0 else vf)
    return t


@pytest.mark.parametrize("tl", grids("periodic"), ids=IDS)
def test_periodic_conservation(gb, tl):
    U = smooth(tl, 4)
    o = Oracle2(tl)
    o.restrict(U)
    G = U[tl.gpu_blocks]
    t0, scale = leaf_totals(G, tl), leaf_totals(np.abs(G), tl)
    h = gb.Hydro.from_two_level(tl)
    Ug = dev(G)
    dt = h.compute_dt(Ug)
    h.advance(Ug, 10, dt)
    assert np.all(np.abs(leaf_totals(host(Ug), tl) - t0) <= 10 * 64 * np.finfo(float).eps * scale)


def corner_band(tl, seed):
    """The smooth state with the pressure raised 30-fold in the coarse cells
    next to the refined region, so the largest CFL speeds sit in the cells the
    flux correction changes, the inner corners included."""
    U = smooth(tl, seed)
    c = tl.coarse
    nd = c.ndim
    zs, ys, xs = c.interior_slices()
    n = c.n[0]
    for b in range(tl.n0):
        if tl.covered(b):
            continue
        bc = c.block_coords(b)
        for d in range(nd):
            for side in (0, 1):
                nbc = list(bc)
                nbc[d] += 1 if side else -1
                if not (0 <= nbc[d] < c.nb[d]):
                    continue
                nb = nbc[0] + c.nb[0] * (nbc[1] + c.nb[1] * nbc[2])
                if not tl.covered(nb):
                    continue
                sl = [slice(None)] * 3
                ax = 2 - d                       # (z, y, x) interior axes
                sl[ax] = slice(n - 1, n) if side else slice(0, 1)
                blk = U[b][:, zs, ys, xs]
                cell = blk[(slice(None),) + tuple(sl)]
                rho, E = cell[0], cell[4]
                kin = 0.5 * (cell[1] ** 2 + cell[2] ** 2 + cell[3] ** 2) / rho
                cell[4] = kin + 30.0 * (E - kin)
                blk[(slice(None),) + tuple(sl)] = cell
                U[b][:, zs, ys, xs] = blk
    return U


@pytest.mark.parametrize("mode", ["all-levels", "level-by-level", "three-stage"])
@pytest.mark.parametrize("tl", GRIDS, ids=IDS)
def test_step_dt_equals_a_separate_reduction(gb, tl, mode):
    U = corner_band(tl, 5)
    h = gb.Hydro.from_two_level(tl)
    if mode == "level-by-level":
        h.set_telescoping(True)
    if mode == "three-stage":
        h.set_rk_stages(3)
    Ug = dev(U[tl.gpu_blocks])
    h.fill_guardcells(Ug)
    dt = h.compute_dt(Ug)
    for _ in range(3):
        h.step_cfl(Ug, dt)
        assert host(dt)[0] == host(h.compute_dt(Ug))[0]
