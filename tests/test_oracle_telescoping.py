"""Pins of the oracle's telescoping-mode step (Sec. 4.2): one guard fill per
step; the first stage also updates a 2-cell ring of guard cells so that the
second stage needs no exchange.

References: the non-telescoping step (pinned separately) wherever a
neighbour supplies the halo -- there the two modes do the same arithmetic on
the same data and must agree bitwise -- and, at outflow edges, an
independent construction: pad the global data by 4 zero-gradient cells
(np.pad), take the plain first stage on that padded grid, and run the plain
second stage from its values on the ring.
"""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle
from tests.gridutil import from_global, padded_global, to_global


def interior(U, lat):
    zs, ys, xs = lat.interior_slices()
    return U[:, :, zs, ys, xs]


@pytest.mark.parametrize("lat", [
    wl.lattice_2d(3, 2, 8, 8, 4, bc="periodic"),
    wl.lattice_3d(2, 2, 2, 8, 8, 8, 4, bc="periodic"),
    wl.lattice_3d(1, 2, 3, 4, 4, 4, 4, bc="periodic"),
])
def test_periodic_equals_non_telescoping_bitwise(lat):
    U = wl.random_state(lat, seed=21, rough=True)
    A, B = U.copy(), U.copy()
    ha, _ = Oracle(lat).run(A, 4)
    hb, _ = Oracle(lat).run(B, 4, telescoping=True)
    assert np.array_equal(ha, hb)
    assert np.array_equal(interior(A, lat), interior(B, lat))


@pytest.mark.parametrize("lat", [
    wl.lattice_2d(3, 3, 8, 8, 4),
    wl.lattice_3d(2, 2, 2, 8, 8, 8, 4, bc=("outflow", "periodic", "outflow")),
])
def test_outflow_differs_only_within_two_cells_of_the_edge(lat):
    """The modes differ only in U1 on the guard ring at an outflow edge, which
    the second stage reads for the 2 cells next to that edge."""
    U = wl.random_state(lat, seed=22, rough=True)
    o = Oracle(lat)
    dt = o.compute_dt(U)
    A, B = U.copy(), U.copy()
    o.step(A, dt)
    o.step(B, dt, telescoping=True)
    GA, GB = to_global(A, lat), to_global(B, lat)
    near = np.zeros(GA.shape[1:], dtype=bool)
    for d in range(lat.ndim):
        if lat.bc[d] == "outflow":
            ax = 2 - d
            idx = [slice(None)] * 3
            idx[ax] = np.r_[0:2, GA.shape[1 + ax] - 2:GA.shape[1 + ax]]
            near[tuple(idx)] = True
    assert np.array_equal(GA[:, ~near], GB[:, ~near])
    assert not np.array_equal(GA[:, near], GB[:, near])


def padded_construction(Gl, lat, dt):
    """Telescoping step on a 1-block lattice, built from the plain stage."""
    g = lat.ng
    assert lat.nblocks == 1 and g == 4
    P = padded_global(Gl, lat)
    n_p = tuple(lat.n[d] + (2 * g if d < lat.ndim else 0) for d in range(3))
    ext = tuple(lat.extent[d] * n_p[d] / lat.n[d] for d in range(3))
    latP = dataclasses.replace(lat, n=n_p, extent=ext, bc=("outflow",) * 3)
    assert latP.dx[:lat.ndim] == lat.dx[:lat.ndim]
    oP = Oracle(latP)
    UP = from_global(P, latP)
    oP.fill_guardcells(UP)
    U1P = UP.copy()
    oP.stage(UP, None, U1P, dt, 0.0, 1.0)
    # the padded grid's cells 2..n+5 are the real block's cells -2..n+1
    U = from_global(Gl, lat)
    o = Oracle(lat)
    o.fill_guardcells(U)
    U1 = U.copy()
    gz = g if lat.ndim == 3 else 0
    sz = slice(gz - 2, gz + lat.n[2] + 2) if lat.ndim == 3 else slice(0, 1)
    szP = slice(2 * gz - 2, 2 * gz + lat.n[2] + 2) if lat.ndim == 3 else slice(0, 1)
    U1[0][:, sz, g - 2:g + lat.n[1] + 2, g - 2:g + lat.n[0] + 2] = \
        U1P[0][:, szP, 2 * g - 2:2 * g + lat.n[1] + 2, 2 * g - 2:2 * g + lat.n[0] + 2]
    out = U1.copy()
    o.stage(U1, U, out, dt, 0.5, 0.5)      # no fill: the second stage reads the ring
    return to_global(out, lat)


@pytest.mark.parametrize("lat", [
    wl.lattice_2d(1, 1, 16, 16, 4),
    wl.lattice_2d(1, 1, 8, 8, 4, bc=("periodic", "outflow")),
    wl.lattice_3d(1, 1, 1, 8, 8, 8, 4),
    wl.lattice_3d(1, 1, 1, 8, 8, 8, 4, bc=("outflow", "outflow", "periodic")),
])
def test_outflow_edge_equals_padded_construction_bitwise(lat):
    Gl = to_global(wl.random_state(lat, seed=23, rough=True), lat)
    o = Oracle(lat)
    U = from_global(Gl, lat)
    dt = 0.5 * o.compute_dt(U)
    o.step(U, dt, telescoping=True)
    assert np.array_equal(to_global(U, lat), padded_construction(Gl, lat, dt))


@pytest.mark.parametrize("bc", ["outflow", "periodic"])
def test_block_decomposition_invisible_bitwise(bc):
    base = wl.lattice_2d(1, 1, 32, 32, 4, bc=bc)
    Gl = to_global(wl.random_state(base, seed=24, rough=True), base)
    results = []
    for nb, n in ((1, 32), (2, 16), (4, 8), (8, 4)):
        lat = wl.lattice_2d(nb, nb, n, n, 4, bc=bc)
        U = from_global(Gl, lat)
        hist, _ = Oracle(lat).run(U, 3, telescoping=True)
        results.append((to_global(U, lat), hist))
    for Gi, hi in results[1:]:
        assert np.array_equal(Gi, results[0][0])
        assert np.array_equal(hi, results[0][1])


def test_block_decomposition_invisible_bitwise_3d():
    base = wl.lattice_3d(1, 1, 1, 16, 16, 16, 4)
    Gl = to_global(wl.random_state(base, seed=25, rough=True), base)
    results = []
    for nb, n in ((1, 16), (2, 8), (4, 4)):
        lat = wl.lattice_3d(nb, nb, nb, n, n, n, 4)
        U = from_global(Gl, lat)
        Oracle(lat).run(U, 2, telescoping=True)
        results.append(to_global(U, lat))
    for Gi in results[1:]:
        assert np.array_equal(Gi, results[0])


def test_uniform_flow_preserved_bitwise_with_outflow_edges():
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8, 4)
    U = np.ascontiguousarray(np.moveaxis(
        wl.conserved(np.full((lat.nblocks,) + lat.padded, 0.9), -0.3, 0.5, 0.2, 1.7, 1.4), 0, 1))
    U0 = U.copy()
    Oracle(lat).run(U, 3, telescoping=True)
    assert np.array_equal(interior(U, lat), interior(U0, lat))


def test_sod_matches_non_telescoping_while_waves_stay_inside():
    """Sod for 100 steps: the waves stay away from the outflow edges, where the
    state is uniform, so the two modes agree bitwise."""
    lat = wl.lattice_2d(8, 8)
    A = wl.sod(lat)
    B = A.copy()
    ha, _ = Oracle(lat).run(A, 100)
    hb, hits = Oracle(lat).run(B, 100, telescoping=True)
    assert hits == 0
    assert np.array_equal(ha, hb) and np.array_equal(interior(A, lat), interior(B, lat))


def test_mirror_symmetry_with_outflow_edges():
    lat = wl.lattice_2d(2, 2, 8, 8, 4)
    Gl = to_global(wl.random_state(lat, seed=26, rough=False), lat)
    M = Gl[:, :, :, ::-1].copy()
    M[1] = -M[1]
    o = Oracle(lat)
    A, B = from_global(Gl, lat), from_global(M, lat)
    dt = o.compute_dt(A)
    o.step(A, dt, telescoping=True)
    o.step(B, dt, telescoping=True)
    GA, GB = to_global(A, lat), to_global(B, lat)
    GB = GB[:, :, :, ::-1]
    GB[1] = -GB[1]
    scale = np.abs(GA).max(axis=(1, 2, 3))
    assert np.all(np.abs(GA - GB).max(axis=(1, 2, 3)) <= 1e-14 * scale)


def test_needs_four_guard_cells():
    lat = wl.lattice_2d(2, 2, 8, 8, 3)
    U = wl.random_state(lat, seed=1)
    with pytest.raises(ValueError):
        Oracle(lat).step(U, 1e-3, telescoping=True)
