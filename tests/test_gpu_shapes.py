"""GPU parity on shapes the other tests leave out: blocks whose z extent
differs from x/y (nzb != nxb), anisotropic cell widths, and gamma = 5/3 --
through the plain, telescoping and three-stage steps and the stage VJP."""
import dataclasses

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


CASES = [
    (wl.lattice_3d(2, 2, 3, 16, 16, 8, 4), 1.4),
    (dataclasses.replace(wl.lattice_3d(3, 2, 2, 8, 8, 12, 6, bc=("periodic", "outflow", "periodic")),
                         extent=(1.0, 0.5, 2.0)), 5.0 / 3.0),
    (dataclasses.replace(wl.lattice_2d(3, 4, 16, 16, 6), extent=(2.0, 0.75, 1.0)), 5.0 / 3.0),
]


# the telescoping mode needs 2 * stages guard cells
@pytest.mark.parametrize("lat,gamma,stages,tele", [
    (l, g, s, t) for l, g in CASES for s, t in ((2, False), (2, True), (3, False), (3, True)) if not t or l.ng >= 2 * s])
def test_step_variants(gb, lat, gamma, stages, tele):
    U = wl.random_state(lat, seed=81, rough=True, gamma=gamma)
    o = Oracle(lat, gamma=gamma)
    dt = o.compute_dt(U)
    ref = U.copy()
    o.step(ref, dt, telescoping=tele, stages=stages)
    h = gb.Hydro.from_lattice(lat, gamma=gamma)
    h.set_rk_stages(stages)
    h.set_telescoping(tele)
    Ug = dev(U)
    assert abs(float(host(h.compute_dt(Ug))[0]) / dt - 1) < 1e-14
    h.step(Ug, dt)
    err = relerr_per_var(to_global(host(Ug), lat), to_global(ref, lat))
    assert np.all(err <= 1e-13), err


@pytest.mark.parametrize("lat,gamma", CASES)
def test_stage_vjp(gb, lat, gamma):
    U = wl.random_state(lat, seed=82, rough=False, gamma=gamma)
    m = np.zeros(lat.shape)
    zs, ys, xs = lat.interior_slices()
    m[:, :, zs, ys, xs] = 1.0
    M = np.random.default_rng(83).normal(size=U.shape) * m
    o = Oracle(lat, gamma=gamma)
    dt = 0.4 * o.compute_dt(U)
    ref = o.stage_vjp(U, M, dt)
    h = gb.Hydro.from_lattice(lat, gamma=gamma)
    out = host(h.stage_vjp(dev(U), dev(M), dt))
    err = relerr_per_var(to_global(out, lat), to_global(ref, lat))
    tol = np.where(np.arange(5) == 3, 1e-10, 1e-11) if lat.ndim == 2 else 1e-11
    assert np.all(err <= tol), err
