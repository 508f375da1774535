"""GPU adjoint of the telescoping step (one fill of all guard layers, ring
stages from the blocks' own guard cells; Sec. 4.2, readings C17, C18)
against the oracle's adjoint of the same step (step_adjoint_telescoping,
pinned by central differences of the oracle's telescoping step): one step
with two and three stages on outflow, periodic and mixed lattices in 2-D and
3-D, and a checkpointed run whose gradient equals the oracle's chain along its
own trajectory.  dt is held fixed and branches keep their forward decisions."""
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


def mask(lat):
    m = np.zeros(lat.shape)
    zs, ys, xs = lat.interior_slices()
    m[:, :, zs, ys, xs] = 1.0
    return m


def err(A, B, lat):
    return relerr_per_var(to_global(A, lat), to_global(B, lat))


CASES = [
    (wl.lattice_2d(3, 2, 16, 16, 4), 2),
    (wl.lattice_2d(4, 4, 8, 8, 4, bc="periodic"), 2),
    (wl.lattice_2d(3, 3, 8, 8, 6, bc=("periodic", "outflow")), 3),
    (wl.lattice_3d(2, 2, 2, 8, 8, 8, 4), 2),
    (wl.lattice_3d(2, 3, 2, 8, 8, 8, 4, bc=("outflow", "periodic", "outflow")), 2),
    (wl.lattice_3d(1, 2, 1, 16, 16, 16, 4, bc=("periodic", "outflow", "periodic")), 2),
    (wl.lattice_3d(2, 2, 2, 8, 8, 8, 6, bc="periodic"), 3),
    (wl.lattice_3d(2, 1, 2, 8, 8, 8, 6), 3),
]


@pytest.mark.parametrize("lat,stages", CASES)
def test_telescoping_step_adjoint_matches_oracle(gb, lat, stages):
    U = wl.random_state(lat, seed=71, rough=False)
    rng = np.random.default_rng(72)
    lam = rng.normal(size=U.shape)          # guard values must not matter
    o = Oracle(lat)
    dt = o.compute_dt(U)
    ref = o.step_adjoint(U, dt, lam * mask(lat), stages=stages, telescoping=True)
    h = gb.Hydro.from_lattice(lat)
    h.set_rk_stages(stages)
    h.set_telescoping(True)
    out = h.step_adjoint(dev(U), dt, dev(lam))
    e = err(host(out), ref, lat)
    tol = np.where(np.arange(5) == 3, 1e-9, 1e-10) if lat.ndim == 2 else 1e-10
    assert np.all(e <= tol), e


@pytest.mark.parametrize("stages,ng", [(2, 4), (3, 6)])
def test_checkpointed_telescoping_gradient_equals_oracle_chain(gb, stages, ng):
    from paper_2401_03378_gb300.adjoint import CheckpointedRun
    lat = wl.lattice_2d(4, 4, 16, 16, ng)
    U0 = wl.sod_smooth(lat)
    lamF = np.random.default_rng(73).normal(size=U0.shape) * mask(lat)
    h = gb.Hydro.from_lattice(lat)
    h.set_rk_stages(stages)
    h.set_telescoping(True)
    run = CheckpointedRun(h, 6, every=4)
    run.forward(dev(U0))
    g = host(run.backward(dev(lamF)))
    o = Oracle(lat)
    ost = [U0.copy()]
    for s in range(6):
        X = ost[-1].copy()
        o.step(X, run.dts[s], telescoping=True, stages=stages)
        ost.append(X)
    lo = lamF.copy()
    for s in reversed(range(6)):
        lo = o.step_adjoint(ost[s], run.dts[s], lo, stages=stages, telescoping=True)
    e = err(g, lo, lat)
    assert np.all(e[[0, 1, 2, 4]] <= 1e-9), e


def test_telescoping_adjoint_differs_from_plain_at_outflow_edges(gb):
    """At an outflow edge the telescoping step evolves the zero-gradient
    copies (reading C17), so its adjoint differs from the plain step's there;
    on a periodic lattice the two steps are the same map and so are their
    adjoints (to rounding)."""
    for bc, same in (("periodic", True), ("outflow", False)):
        lat = wl.lattice_2d(3, 3, 8, 8, 4, bc=bc)
        U = wl.random_state(lat, seed=74, rough=False)
        lam = dev(np.random.default_rng(75).normal(size=U.shape) * mask(lat))
        dt = Oracle(lat).compute_dt(U)
        ht = gb.Hydro.from_lattice(lat)
        ht.set_telescoping(True)
        hp = gb.Hydro.from_lattice(lat)
        a, b = host(ht.step_adjoint(dev(U), dt, lam)), host(hp.step_adjoint(dev(U), dt, lam))
        e = err(a, b, lat)
        if same:
            assert np.all(e[[0, 1, 2, 4]] <= 1e-12), e
        else:
            assert np.max(e) > 1e-8
