"""Pins of the oracle's adjoint (dual-number Jacobians transposed): central
finite differences of the oracle's own forward map, dt held fixed."""
import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle


def interior_mask(lat):
    m = np.zeros(lat.shape, dtype=bool)
    zs, ys, xs = lat.interior_slices()
    m[:, :, zs, ys, xs] = True
    return m


def pick(lat, n, seed):
    """Random interior components.  In 2-D the z-momentum is identically zero,
    so every MC slope of w sits at the limiter's kink (both differences zero);
    a finite difference through more than one stage then activates those
    slopes at first order while the frozen-branch adjoint keeps them at zero.
    Both are valid one-sided linearisations; the comparison uses the others."""
    rng = np.random.default_rng(seed)
    m = interior_mask(lat)
    if lat.ndim == 2:
        m[:, 3] = False
    idx = np.argwhere(m)
    return [tuple(idx[i]) for i in rng.choice(len(idx), n, replace=False)]


LATS = [wl.lattice_2d(2, 2, 8, 8, 4), wl.lattice_3d(2, 2, 2, 4, 4, 4, 4, bc="periodic"),
        wl.lattice_2d(3, 2, 8, 8, 4, bc=("periodic", "outflow"))]


@pytest.mark.parametrize("lat", LATS)
def test_stage_vjp_matches_finite_differences(lat):
    o = Oracle(lat)
    U = wl.random_state(lat, seed=1, rough=False)
    rng = np.random.default_rng(2)
    M = rng.normal(size=U.shape) * interior_mask(lat)
    dt = 0.5 * o.compute_dt(U)

    def G(V):
        f = V.copy()
        o.fill_guardcells(f)
        out = f.copy()
        o.stage(f, None, out, dt, 0.0, 1.0)
        return float(np.sum(M * out * interior_mask(lat)))

    grad = M + o.stage_vjp(U, M, dt)
    scale = np.max(np.abs(grad))
    for c in pick(lat, 12, 3):
        h = 1e-6 * max(1.0, abs(U[c]))
        Up, Um = U.copy(), U.copy()
        Up[c] += h
        Um[c] -= h
        fd = (G(Up) - G(Um)) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * scale, (c, fd, grad[c])


@pytest.mark.parametrize("lat", LATS[:2])
def test_step_adjoint_matches_finite_differences(lat):
    o = Oracle(lat)
    U = wl.random_state(lat, seed=4, rough=False)
    rng = np.random.default_rng(5)
    w = rng.normal(size=U.shape) * interior_mask(lat)
    dt = o.compute_dt(U)

    def G(V):
        X = V.copy()
        o.step(X, dt)
        return float(np.sum(w * X * interior_mask(lat)))

    grad = o.step_adjoint(U, dt, w)
    scale = np.max(np.abs(grad))
    for c in pick(lat, 12, 6):
        h = 1e-6 * max(1.0, abs(U[c]))
        Up, Um = U.copy(), U.copy()
        Up[c] += h
        Um[c] -= h
        fd = (G(Up) - G(Um)) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * scale, (c, fd, grad[c])


def test_step_adjoint_linear_in_the_cotangent():
    lat = LATS[0]
    o = Oracle(lat)
    U = wl.random_state(lat, seed=7, rough=True)
    rng = np.random.default_rng(8)
    a = rng.normal(size=U.shape) * interior_mask(lat)
    b = rng.normal(size=U.shape) * interior_mask(lat)
    dt = o.compute_dt(U)
    lhs = o.step_adjoint(U, dt, 2.0 * a - 3.0 * b)
    rhs = 2.0 * o.step_adjoint(U, dt, a) - 3.0 * o.step_adjoint(U, dt, b)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(rhs))


@pytest.mark.parametrize("lat", LATS[:2])
def test_three_stage_step_adjoint_matches_finite_differences(lat):
    o = Oracle(lat)
    U = wl.random_state(lat, seed=14, rough=False)
    rng = np.random.default_rng(15)
    w = rng.normal(size=U.shape) * interior_mask(lat)
    dt = o.compute_dt(U)

    def G(V):
        X = V.copy()
        o.step(X, dt, stages=3)
        return float(np.sum(w * X * interior_mask(lat)))

    grad = o.step_adjoint(U, dt, w, stages=3)
    scale = np.max(np.abs(grad))
    for c in pick(lat, 12, 16):
        h = 1e-6 * max(1.0, abs(U[c]))
        Up, Um = U.copy(), U.copy()
        Up[c] += h
        Um[c] -= h
        fd = (G(Up) - G(Um)) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * scale, (c, fd, grad[c])


def test_three_stage_adjoint_differs_from_two_stage():
    """The stage count enters the adjoint: the three-stage adjoint is not the
    two-stage one (a planted stage count would be caught)."""
    lat = LATS[0]
    o = Oracle(lat)
    U = wl.random_state(lat, seed=17, rough=False)
    w = np.random.default_rng(18).normal(size=U.shape) * interior_mask(lat)
    dt = o.compute_dt(U)
    a, b = o.step_adjoint(U, dt, w, stages=3), o.step_adjoint(U, dt, w, stages=2)
    assert np.max(np.abs(a - b)) > 1e-6 * np.max(np.abs(a))


TELE_LATS = [wl.lattice_2d(2, 2, 8, 8, 4), wl.lattice_3d(2, 2, 2, 4, 4, 4, 4, bc="periodic"),
             wl.lattice_2d(3, 2, 8, 8, 4, bc=("periodic", "outflow"))]


@pytest.mark.parametrize("lat", TELE_LATS)
def test_telescoping_step_adjoint_matches_finite_differences(lat):
    """The adjoint of the telescoping step (one fill of all guard layers, the
    first stage on the interior widened by 2 from the block's own cells)
    against central differences of the oracle's telescoping step."""
    o = Oracle(lat)
    U = wl.random_state(lat, seed=21, rough=False)
    w = np.random.default_rng(22).normal(size=U.shape) * interior_mask(lat)
    dt = o.compute_dt(U)

    def G(V):
        X = V.copy()
        o.step(X, dt, telescoping=True)
        return float(np.sum(w * X * interior_mask(lat)))

    grad = o.step_adjoint(U, dt, w, telescoping=True)
    scale = np.max(np.abs(grad))
    # cells next to block and domain edges, where the ring and the fill matter, and random ones
    cells = pick(lat, 10, 23)
    zs, ys, xs = lat.interior_slices()
    cells += [(0, 0, zs.start, ys.start, xs.start), (1, 1, zs.stop - 1, ys.start, xs.stop - 1),
              (lat.nblocks - 1, 4, zs.stop - 1, ys.stop - 2, xs.start + 1)]
    for c in cells:
        h = 1e-6 * max(1.0, abs(U[c]))
        Up, Um = U.copy(), U.copy()
        Up[c] += h
        Um[c] -= h
        fd = (G(Up) - G(Um)) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * scale, (c, fd, grad[c])


def test_telescoping_three_stage_adjoint_matches_finite_differences():
    lat = wl.lattice_2d(2, 2, 8, 8, 6)
    o = Oracle(lat)
    U = wl.random_state(lat, seed=24, rough=False)
    w = np.random.default_rng(25).normal(size=U.shape) * interior_mask(lat)
    dt = o.compute_dt(U)

    def G(V):
        X = V.copy()
        o.step(X, dt, telescoping=True, stages=3)
        return float(np.sum(w * X * interior_mask(lat)))

    grad = o.step_adjoint(U, dt, w, stages=3, telescoping=True)
    scale = np.max(np.abs(grad))
    for c in pick(lat, 12, 26):
        h = 1e-6 * max(1.0, abs(U[c]))
        Up, Um = U.copy(), U.copy()
        Up[c] += h
        Um[c] -= h
        fd = (G(Up) - G(Um)) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * scale, (c, fd, grad[c])


@pytest.mark.parametrize("stages,ng", [(2, 4), (3, 6)])
def test_telescoping_adjoint_equals_plain_adjoint_on_periodic_lattices(stages, ng):
    """On a periodic lattice the telescoping step is the plain step bit for bit,
    so the two adjoints agree to rounding; at an outflow edge they differ (the
    first stage evolves the zero-gradient copies there)."""
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8, ng, bc="periodic")
    o = Oracle(lat)
    U = wl.random_state(lat, seed=27, rough=True)
    w = np.random.default_rng(28).normal(size=U.shape) * interior_mask(lat)
    dt = o.compute_dt(U)
    a = o.step_adjoint(U, dt, w, stages=stages, telescoping=True)
    b = o.step_adjoint(U, dt, w, stages=stages)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    lat2 = wl.lattice_2d(2, 2, 8, 8, ng)
    o2 = Oracle(lat2)
    U2 = wl.random_state(lat2, seed=29, rough=True)
    w2 = np.random.default_rng(30).normal(size=U2.shape) * interior_mask(lat2)
    dt2 = o2.compute_dt(U2)
    a2 = o2.step_adjoint(U2, dt2, w2, stages=stages, telescoping=True)
    b2 = o2.step_adjoint(U2, dt2, w2, stages=stages)
    assert np.max(np.abs(a2 - b2)) > 1e-8 * np.max(np.abs(b2))
