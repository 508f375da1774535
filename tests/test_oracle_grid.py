"""Pins of the oracle's grid-level method (guard fill, stage, SSP-RK2 step, dt).

The references are exact solutions (Sod, Sedov), conservation laws, exact
invariances of the discrete scheme, and closed forms -- never the oracle's own
formulas.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import exact_riemann as er
from oracle import sedov
from oracle.oracle import Oracle
from tests.gridutil import from_global, padded_global, relerr_per_var, to_global

G = 1.4


def run_to(o, U, T):
    t, n = 0.0, 0
    while t < T - 1e-15:
        dt = min(o.compute_dt(U), T - t)
        o.step(U, dt)
        t += dt
        n += 1
    return n


# --------------------------------------------------------------- guard fill --

@pytest.mark.parametrize("lat", [
    wl.lattice_2d(3, 2, 8, 8, 4),
    wl.lattice_2d(2, 3, 8, 8, 4, bc=("periodic", "outflow")),
    wl.lattice_3d(2, 3, 2, 4, 4, 4, 4),
    wl.lattice_3d(2, 2, 3, 8, 8, 8, 4, bc=("outflow", "periodic", "periodic")),
    wl.lattice_3d(1, 2, 1, 8, 8, 8, 4, bc="periodic"),
])
def test_fill_equals_padded_global_array(lat):
    rng = np.random.default_rng(0)
    Gl = rng.normal(size=(5,) + lat.global_cells[::-1])
    U = from_global(Gl, lat, guard_value=np.nan)
    Oracle(lat).fill_guardcells(U)
    P = padded_global(Gl, lat)
    nx, ny, nz = lat.n
    for b in range(lat.nblocks):
        bi, bj, bk = lat.block_coords(b)
        kz = slice(bk * nz, bk * nz + lat.padded[0]) if lat.ndim == 3 else slice(0, 1)
        win = P[:, kz, bj * ny:bj * ny + lat.padded[1], bi * nx:bi * nx + lat.padded[2]]
        assert np.array_equal(U[b], win), b


# ----------------------------------------------------------------------- dt --

def test_dt_closed_form_uniform_state():
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8)
    r, u, v, w, p = 1.3, 0.2, -0.5, 0.7, 0.9
    U = np.ascontiguousarray(np.moveaxis(wl.conserved(np.full(lat.shape[:1] + lat.padded, r), u, v, w, p, G), 0, 1))
    dt = Oracle(lat).compute_dt(U)
    c = math.sqrt(G * p / r)
    dx = 1.0 / 16
    expect = 0.8 / ((abs(u) + c) / dx + (abs(v) + c) / dx + (abs(w) + c) / dx)
    assert abs(dt - expect) <= 4e-16 * expect


# ---------------------------------------------------------------- Sod (C-T3) --

def test_sod_config_2d_128_100_steps_vs_exact():
    lat = wl.lattice_2d(8, 8)
    U = wl.sod(lat)
    hist, hits = Oracle(lat).run(U, 100)
    assert hits == 0
    T = hist.sum()
    Gl = to_global(U, lat)
    rho = Gl[0, 0]
    assert np.all(rho == rho[0:1]), "every y-row must be bitwise identical"
    assert np.all(Gl[2] == 0.0) and np.all(Gl[3] == 0.0)
    xf = np.arange(129) / 128
    exact = er.cell_average_density((1, 0, 1), (0.125, 0, 0.1), xf, 0.5, T)
    L1 = np.mean(np.abs(rho[0] - exact))
    assert L1 < 5e-3, L1


def test_sod_first_order_convergence():
    errs = []
    for N in (64, 128, 256):
        lat = wl.lattice_2d(N // 16, 1, 16, 16)
        U = wl.sod(lat)
        run_to(Oracle(lat), U, 0.2)
        rho = to_global(U, lat)[0, 0]
        exact = er.cell_average_density((1, 0, 1), (0.125, 0, 0.1), np.arange(N + 1) / N, 0.5, 0.2)
        errs.append(np.mean(np.abs(rho[0] - exact)))
    assert errs[0] < 1e-2
    assert errs[0] / errs[1] > 1.7 and errs[1] / errs[2] > 1.7, errs


# ------------------------------------------------------------- Sedov (C-T4) --

@pytest.mark.slow
def test_sedov_radius_symmetry_energy():
    N = 48
    lat = wl.lattice_3d(3, 3, 3)
    U = wl.sedov(lat)
    assert wl.sedov_cells(lat).sum() == 160
    o = Oracle(lat)
    X, Y, Z = wl.cell_centers(lat)
    zs, ys, xs = lat.interior_slices()
    r = np.sqrt((X - .5) ** 2 + (Y - .5) ** 2 + (Z - .5) ** 2)[:, zs, ys, xs].ravel()
    bins = np.floor(r * N * 2).astype(int)
    E0 = U[:, 4, zs, ys, xs].sum()
    M0 = U[:, 0, zs, ys, xs].sum()
    t = 0.0
    peaks = []
    for n in range(1, 61):
        dt = o.compute_dt(U)
        assert o.step(U, dt) == 0
        t += dt
        if n in (20, 40, 60):
            peaks.append(U[:, 0, zs, ys, xs].max())
        if n in (40, 60):
            rho = U[:, 0, zs, ys, xs].ravel()
            prof = np.bincount(bins, rho) / np.maximum(np.bincount(bins), 1)
            rpk = (np.argmax(prof) + 0.5) / (2 * N)
            Rs = sedov.shock_radius(t)
            assert Rs * N >= 8
            assert abs(rpk / Rs - 1) < 0.05, (n, rpk, Rs)
    # the peak density climbs toward the strong-shock compression (gamma+1)/(gamma-1) = 6
    # as the shell spreads over more cells, and stays below it
    assert peaks[0] < peaks[1] < peaks[2] < 6.0 and peaks[0] > 1.5, peaks
    assert abs(U[:, 4, zs, ys, xs].sum() / E0 - 1) < 1e-13
    assert abs(U[:, 0, zs, ys, xs].sum() / M0 - 1) < 1e-13
    Gl = to_global(U, lat)
    sgn = np.array([1, -1, 1, 1, 1.0])[:, None, None, None]
    mir = sgn * Gl[:, :, :, ::-1]
    assert np.max(relerr_per_var(mir, Gl)) < 1e-11
    # x <-> y exchange
    sw = Gl[[0, 2, 1, 3, 4]].transpose(0, 1, 3, 2)
    assert np.max(relerr_per_var(sw, Gl)) < 1e-11


# ------------------------------------------------------- conservation (C-T5) --

@pytest.mark.parametrize("lat,steps,rough", [
    (wl.lattice_2d(4, 4, 16, 16, 4, bc="periodic"), 50, True),
    (wl.lattice_2d(4, 4, 16, 16, 4, bc="periodic"), 50, False),
    (wl.lattice_3d(2, 2, 2, 8, 8, 8, 4, bc="periodic"), 20, True),
    (wl.lattice_3d(2, 2, 2, 8, 8, 8, 4, bc="periodic"), 20, False),
])
def test_conservation_periodic(lat, steps, rough):
    U = wl.random_state(lat, seed=11, rough=rough)
    zs, ys, xs = lat.interior_slices()
    before = U[:, :, zs, ys, xs].sum(axis=(0, 2, 3, 4))
    scale = np.abs(U[:, :, zs, ys, xs]).sum(axis=(0, 2, 3, 4))
    _, hits = Oracle(lat).run(U, steps)
    assert hits == 0
    after = U[:, :, zs, ys, xs].sum(axis=(0, 2, 3, 4))
    ncell = lat.interior_cells
    assert np.all(np.abs(after - before) <= steps * 8 * np.finfo(float).eps * scale + 1e-300), (after - before) / scale


# ----------------------------------------------------------- invariance (C-T6) --

def test_uniform_flow_preserved_bitwise():
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8, 4, bc="periodic")
    U = np.ascontiguousarray(np.moveaxis(wl.conserved(np.full((lat.nblocks,) + lat.padded, 1.1), 0.3, -0.2, 0.4, 0.8, G), 0, 1))
    U0 = U.copy()
    Oracle(lat).run(U, 3)
    zs, ys, xs = lat.interior_slices()
    assert np.array_equal(U[:, :, zs, ys, xs], U0[:, :, zs, ys, xs])


@pytest.mark.parametrize("bc", ["outflow", "periodic"])
def test_block_decomposition_invisible_bitwise(bc):
    rng_lat = wl.lattice_3d(1, 1, 1, 32, 32, 32, 4, bc=bc)
    Gl = to_global(wl.random_state(rng_lat, seed=5, rough=True), rng_lat)
    results = []
    for nb, n in ((1, 32), (2, 16), (4, 8)):
        lat = wl.lattice_3d(nb, nb, nb, n, n, n, 4, bc=bc)
        U = from_global(Gl, lat)
        hist, _ = Oracle(lat).run(U, 3)
        results.append((to_global(U, lat), hist))
    for Gi, hi in results[1:]:
        assert np.array_equal(Gi, results[0][0])
        assert np.array_equal(hi, results[0][1])


def test_x_only_problem_rows_bitwise_identical_3d():
    lat = wl.lattice_3d(2, 2, 2, 16, 16, 16)
    U = wl.sod(lat)
    Oracle(lat).run(U, 10)
    Gl = to_global(U, lat)
    assert np.all(Gl == Gl[:, :1, :1, :])
    assert np.all(Gl[2] == 0) and np.all(Gl[3] == 0)


def test_axis_permutation():
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8, 4)
    Gl = to_global(wl.random_state(lat, seed=8, rough=False), lat)
    # new (x, y, z) = old (y, z, x): array axes (z, y, x) -> data transposed accordingly
    def perm(A):
        B = A[[0, 2, 3, 1, 4]]            # momentum components follow the axes
        return np.ascontiguousarray(B.transpose(0, 3, 1, 2))
    U1 = from_global(Gl, lat)
    U2 = from_global(perm(Gl), lat)
    o = Oracle(lat)
    h1, _ = o.run(U1, 4)
    h2, _ = o.run(U2, 4)
    assert np.max(np.abs(h1 - h2) / h1) < 1e-15
    assert np.max(relerr_per_var(to_global(U2, lat), perm(to_global(U1, lat)))) < 1e-14


def test_corner_guards_never_read():
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8, 4)
    U = wl.random_state(lat, seed=2)
    o = Oracle(lat)
    o.fill_guardcells(U)
    P = wl.poison_guards(U, lat, np.nan, corners_only=True)
    outs = []
    for Uin in (U, P):
        out = Uin.copy()
        o.stage(Uin, None, out, 1e-3, 0.0, 1.0)
        zs, ys, xs = lat.interior_slices()
        outs.append(out[:, :, zs, ys, xs])
    assert np.all(np.isfinite(outs[1]))
    assert np.array_equal(outs[0], outs[1])


def test_floor_hits_counted():
    lat = wl.lattice_2d(2, 2, 8, 8, 4)
    U = wl.random_state(lat, seed=3)
    U[1, 4, 0, 6, 6] = -1.0    # negative total energy -> negative pressure
    o = Oracle(lat)
    o.fill_guardcells(U)
    out = U.copy()
    assert o.stage(U, None, out, 1e-4, 0.0, 1.0) == 1
