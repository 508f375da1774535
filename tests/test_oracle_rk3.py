"""Pins of the oracle's three-stage SSP-RK steps (Shu-Osher form; Sec. 4.2
names SSP-RK, multistage): the temporal order of accuracy at fixed space
discretisation, conservation, exactness on uniform flow, the Sod solution,
and the telescoping form against the non-telescoping one and against an
independent padded-grid construction."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import exact_riemann as er
from oracle.oracle import Oracle, Oracle2
from tests.gridutil import from_global, padded_global, to_global
from tests.test_oracle_amr import leaf_totals, tl2, tl3


def interior(U, lat):
    zs, ys, xs = lat.interior_slices()
    return U[:, :, zs, ys, xs]


def acoustic(lat):
    X, Y, Z = wl.cell_centers(lat)
    rho = 1 + 0.1 * np.sin(2 * np.pi * X + 0.3) * np.cos(2 * np.pi * Y)
    p = 1 + 0.1 * np.cos(2 * np.pi * (X + Y))
    return wl._assemble(lat, rho, 0.2 * np.sin(2 * np.pi * Y), 0.1 * np.cos(2 * np.pi * X), 0 * X, p, 1.4)


def test_temporal_order():
    """Smooth periodic acoustics on a fixed 64^2 grid to T = 0.08 with N
    equal steps: against a 1024-step three-stage solution, the L1 error falls
    as N^-2 with two stages and as N^-3 with three."""
    lat = wl.lattice_2d(4, 4, 16, 16, 4, bc="periodic")
    o = Oracle(lat)
    U0 = acoustic(lat)
    T = 0.08

    def run(N, stages):
        U = U0.copy()
        for _ in range(N):
            o.step(U, T / N, stages=stages)
        return interior(U, lat)
    ref = run(1024, 3)
    for stages, lo, hi in ((2, 1.8, 2.2), (3, 2.6, 3.4)):
        e = [np.mean(np.abs(run(N, stages) - ref)) for N in (16, 32, 64)]
        rates = [np.log2(e[i] / e[i + 1]) for i in range(2)]
        assert all(lo <= r <= hi for r in rates), (stages, e, rates)
        if stages == 3:
            assert e[-1] < 0.02 * e2_64
        else:
            e2_64 = e[-1]


@pytest.mark.parametrize("lat", [wl.lattice_2d(4, 4, 16, 16, 4, bc="periodic"),
                                 wl.lattice_3d(2, 2, 2, 8, 8, 8, 4, bc="periodic")])
def test_conservation_periodic(lat):
    U = wl.random_state(lat, seed=41, rough=True)
    zs, ys, xs = lat.interior_slices()
    before = U[:, :, zs, ys, xs].sum(axis=(0, 2, 3, 4))
    scale = np.abs(U[:, :, zs, ys, xs]).sum(axis=(0, 2, 3, 4))
    _, hits = Oracle(lat).run(U, 20, stages=3)
    assert hits == 0
    after = U[:, :, zs, ys, xs].sum(axis=(0, 2, 3, 4))
    assert np.all(np.abs(after - before) <= 20 * 12 * np.finfo(float).eps * scale)


def test_uniform_flow_preserved_to_round_off():
    """L = 0 exactly on uniform flow; the stage combinations 3/4 x + 1/4 x and
    1/3 x + 2/3 x return x only to within an ulp or two."""
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8, 4)
    U = np.ascontiguousarray(np.moveaxis(
        wl.conserved(np.full((lat.nblocks,) + lat.padded, 1.1), 0.3, -0.2, 0.4, 0.8, 1.4), 0, 1))
    U0 = U.copy()
    Oracle(lat).run(U, 3, stages=3)
    a, b = interior(U, lat), interior(U0, lat)
    assert np.max(np.abs(a - b) / np.abs(b)) <= 8 * np.finfo(float).eps


def test_sod_2d_vs_exact():
    lat = wl.lattice_2d(8, 8)
    U = wl.sod(lat)
    hist, hits = Oracle(lat).run(U, 100, stages=3)
    assert hits == 0
    Gl = to_global(U, lat)
    rho = Gl[0, 0]
    assert np.all(rho == rho[0:1])
    exact = er.cell_average_density((1, 0, 1), (0.125, 0, 0.1), np.arange(129) / 128, 0.5, hist.sum())
    assert np.mean(np.abs(rho[0] - exact)) < 5e-3


@pytest.mark.parametrize("lat", [wl.lattice_2d(3, 2, 8, 8, 6, bc="periodic"),
                                 wl.lattice_3d(2, 2, 2, 8, 8, 8, 6, bc="periodic")])
def test_telescoping_periodic_equals_non_telescoping_bitwise(lat):
    U = wl.random_state(lat, seed=42, rough=True)
    A, B = U.copy(), U.copy()
    ha, _ = Oracle(lat).run(A, 3, stages=3)
    hb, _ = Oracle(lat).run(B, 3, stages=3, telescoping=True)
    assert np.array_equal(ha, hb)
    assert np.array_equal(interior(A, lat), interior(B, lat))


@pytest.mark.parametrize("lat", [wl.lattice_2d(1, 1, 16, 16, 6),
                                 wl.lattice_2d(1, 1, 8, 8, 6, bc=("periodic", "outflow")),
                                 wl.lattice_3d(1, 1, 1, 8, 8, 8, 6)])
def test_telescoping_equals_plain_step_on_padded_grid(lat):
    """Telescoping RK3 on one block = the non-telescoping RK3 step on the grid
    padded by 6 zero-gradient (or periodic) cells, restricted to the block:
    the cells used never see the padded grid's own boundary."""
    Gl = to_global(wl.random_state(lat, seed=43, rough=True), lat)
    o = Oracle(lat)
    U = from_global(Gl, lat)
    dt = 0.5 * o.compute_dt(U)
    o.step(U, dt, telescoping=True, stages=3)
    g = lat.ng
    P = padded_global(Gl, lat)
    n_p = tuple(lat.n[d] + (2 * g if d < lat.ndim else 0) for d in range(3))
    ext = tuple(lat.extent[d] * n_p[d] / lat.n[d] for d in range(3))
    latP = dataclasses.replace(lat, n=n_p, extent=ext, bc=("outflow",) * 3)
    assert latP.dx[:lat.ndim] == lat.dx[:lat.ndim]
    UP = from_global(P, latP)
    Oracle(latP).step(UP, dt, stages=3)
    GP = to_global(UP, latP)
    sz = slice(g, g + lat.n[2]) if lat.ndim == 3 else slice(0, 1)
    assert np.array_equal(to_global(U, lat), GP[:, sz, g:g + lat.n[1], g:g + lat.n[0]])


def test_telescoping_needs_six_guard_cells():
    lat = wl.lattice_2d(2, 2, 8, 8, 4)
    with pytest.raises(ValueError):
        Oracle(lat).step(wl.random_state(lat, seed=1), 1e-4, telescoping=True, stages=3)


@pytest.mark.parametrize("telescoping", [False, True])
@pytest.mark.parametrize("mk", [tl3, tl2])
def test_two_level_conservation(mk, telescoping):
    tl = mk()
    if telescoping:
        c = tl.coarse
        tl = wl.two_level(dataclasses.replace(c, ng=6), tl.lo[:c.ndim], tl.hi[:c.ndim])
    from tests.test_oracle_amr_telescoping import smooth
    U = smooth(tl)
    o = Oracle2(tl)
    o.restrict(U)
    t0, scale = leaf_totals(U, tl), leaf_totals(np.abs(U), tl)
    _, hits = o.run(U, 8, telescoping=telescoping, stages=3)
    assert hits == 0
    assert np.all(np.abs(leaf_totals(U, tl) - t0) <= 8 * 96 * np.finfo(float).eps * scale)
