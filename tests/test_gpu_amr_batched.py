"""GPU ensembles of two-level composite grids (gbh_create_refined_batched):
every problem against the oracle's two-level path on its own, per-problem CFL
steps and histories, bitwise agreement with separate two-level contexts and
with the graph-captured advance, both stage counts, the level-by-level
telescoping variant, and the constructor's table checks."""
import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle2
from tests.test_gpu_amr import leaf_err, smooth

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


def batch_2d(ng):
    return [wl.two_level(wl.lattice_2d(4, 4, 16, 16, ng, bc="periodic"), (1, 1), (3, 3)),
            wl.two_level(wl.lattice_2d(5, 4, 16, 16, ng), (1, 1), (4, 3)),
            wl.two_level(wl.lattice_2d(6, 6, 16, 16, ng), (2, 1), (4, 5))]


def batch_3d(ng):
    return [wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, ng, bc="periodic"), (1, 1, 1), (3, 3, 3)),
            wl.two_level(wl.lattice_3d(4, 3, 4, 8, 8, 8, ng), (1, 1, 2), (2, 2, 3)),
            wl.two_level(wl.lattice_3d(3, 3, 3, 8, 8, 8, ng), (1, 1, 1), (2, 2, 2))]


def split(U, tls):
    out, o = [], 0
    for tl in tls:
        out.append(U[o:o + tl.nblocks])
        o += tl.nblocks
    return out


def states(tls, seed):
    parts = []
    for i, tl in enumerate(tls):
        U = smooth(tl, seed + i)
        Oracle2(tl).restrict(U)
        parts.append(U)
    return parts


@pytest.mark.parametrize("stages", [2, 3])
@pytest.mark.parametrize("make", [batch_2d, batch_3d])
def test_batched_two_level_matches_oracle(gb, make, stages):
    tls = make(4 if stages == 2 else 6)
    parts = states(tls, 70)
    h = gb.Hydro.from_two_level_batch(tls)
    h.set_rk_stages(stages)
    assert h.nproblems == len(tls)
    # one step with one host dt for every problem
    dt = min(Oracle2(tl).compute_dt(U) for tl, U in zip(tls, parts))
    Ug = dev(np.concatenate(parts))
    h.step(Ug, dt)
    for tl, U, got in zip(tls, parts, split(host(Ug), tls)):
        ref = U.copy()
        Oracle2(tl).step(ref, dt, stages=stages)
        assert np.all(leaf_err(got, ref, tl) <= 1e-13)
    # 5 steps, each problem with its own device CFL dt
    Ug = dev(np.concatenate(parts))
    dtd = h.compute_dt(Ug)
    assert dtd.numel() == len(tls)
    hist = torch.zeros(5, len(tls), dtype=torch.float64, device="cuda")
    h.advance(Ug, 5, dtd, hist)
    hg = host(hist)
    for i, (tl, U, got) in enumerate(zip(tls, parts, split(host(Ug), tls))):
        ref = U.copy()
        hist_o, _ = Oracle2(tl).run(ref, 5, stages=stages)
        assert np.max(np.abs(hg[:, i] / hist_o - 1)) <= 1e-12
        assert np.all(leaf_err(got, ref, tl) <= 1e-11)


@pytest.mark.parametrize("telescoping", [False, True])
@pytest.mark.parametrize("make", [batch_2d, batch_3d])
def test_batched_equals_separate_contexts_bitwise(gb, make, telescoping):
    tls = make(4)
    parts = states(tls, 80)
    h = gb.Hydro.from_two_level_batch(tls)
    h.set_telescoping(telescoping)
    A, B = dev(np.concatenate(parts)), dev(np.concatenate(parts))
    da, db = h.compute_dt(A), h.compute_dt(B)
    ha = torch.zeros(4, len(tls), dtype=torch.float64, device="cuda")
    h.advance(A, 4, da, ha)
    h.advance_graph(B, 4, db)
    assert torch.equal(A, B) and torch.equal(da, db)
    out = split(host(A), tls)
    for i, (tl, U) in enumerate(zip(tls, parts)):
        s = gb.Hydro.from_two_level(tl)
        s.set_telescoping(telescoping)
        Us = dev(U)
        ds = s.compute_dt(Us)
        hs = torch.zeros(4, dtype=torch.float64, device="cuda")
        s.advance(Us, 4, ds, hs)
        assert np.array_equal(host(hs), host(ha)[:, i])
        assert np.array_equal(host(Us), out[i])


def test_two_level_sedov_ensemble(gb):
    """Uneven 3-D two-level Sedov problems (coarse 4^3, 6^3 or 8^3 blocks of 16^3
    cells, the central half refined), 3 steps, against the oracle per problem."""
    probs = wl.two_level_ensemble(count=3, seed=5, choices=(4, 6))
    tls = [t for t, _ in probs]
    h = gb.Hydro.from_two_level_batch(tls)
    Ug = dev(np.concatenate([u for _, u in probs]))
    dtd = h.compute_dt(Ug)
    hist = torch.zeros(3, len(tls), dtype=torch.float64, device="cuda")
    h.advance(Ug, 3, dtd, hist)
    hg = host(hist)
    for i, ((tl, U), got) in enumerate(zip(probs, split(host(Ug), tls))):
        ref = U.copy()
        o = Oracle2(tl)
        o.restrict(ref)
        hist_o, _ = o.run(ref, 3)
        assert np.max(np.abs(hg[:, i] / hist_o - 1)) <= 1e-12
        assert np.all(leaf_err(got, ref, tl) <= 1e-11)


def test_constructor_checks(gb):
    from paper_2401_03378_gb300._abi import GbhError
    from paper_2401_03378_gb300.grid import batched_two_level_tables
    tls = batch_2d(4)
    c = tls[0].coarse
    args = [(t.coarse.ndim, t.coarse.nb, t.coarse.n, t.lo, t.hi,
             tuple(b == "periodic" for b in t.coarse.bc), t.coarse.dx) for t in tls]
    nbr, dx, parent, children, problem = batched_two_level_tables(args)
    kw = dict(nbr=nbr, dx=dx, parent=parent, children=children, nproblems=3)
    gb.Hydro(2, c.n, c.ng, problem=problem, **kw).close()
    bad = problem.copy()
    bad[tls[0].n0] = 1                      # a fine block of problem 0 labelled as problem 1
    with pytest.raises(GbhError):
        gb.Hydro(2, c.n, c.ng, problem=bad, **kw)
    bad = problem.copy()
    bad[0] = 3                              # out of range
    with pytest.raises(GbhError):
        gb.Hydro(2, c.n, c.ng, problem=bad, **kw)
    h = gb.Hydro(2, c.n, c.ng, problem=problem, **kw)
    U = dev(np.concatenate(states(tls, 90)))
    with pytest.raises(GbhError):           # the adjoint takes one dt and one level
        h.step_adjoint(U, 1e-4, torch.zeros_like(U))
