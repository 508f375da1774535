"""Whole-run parity at the stated step counts of every workload.

Each test advances the GPU through its whole run, in the launch configuration
the benchmark times (the CFL dt computed on the device every step), and
compares the final state and the dt of every step with the oracle's run of the
same length from the same initial data:

- 3-D Sedov 128^3 (512 blocks of 16^3 + 4 guards), 200 steps;
- 3-D Sedov 256^3 (4096 blocks), 50 steps;
- its two-level variant (4096 coarse + 4096 fine blocks, the central eighth of
  the volume at half the cell width), 50 steps, all-levels update with
  restriction, prolongation and flux correction every stage;
- the 96-problem batched ensemble (periodic 2-D Sod / Kelvin-Helmholtz, sizes
  drawn from 64^2 ... 512^2), 100 steps in one captured CUDA graph, every
  problem with its own dt;
- the gradient workload (2-D Sod-like 256^2, 50 steps, checkpoint every 10):
  the GPU's checkpointed adjoint against the oracle's step adjoint chained
  backwards along the oracle's own trajectory with the same dt sequence.

Bar: relative L-infinity <= 1e-11 per conserved variable over interior (leaf)
cells, exact zero where the oracle's variable is identically zero, dt of every
step <= 1e-12 relative (the SSP-RK steps and all-levels update of Sec. 4.2).
The gradient is compared at <= 1e-9 relative to each variable's largest
component (the chain of 100 stage VJPs accumulates rounding of the two forward
trajectories and of the adjoint sums).
"""
import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle, Oracle2
from tests.gridutil import relerr_per_var, to_global

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL_RUN = 1e-11
TOL_DT = 1e-12
TOL_GRAD = 1e-9


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


def report(name, err, dterr=None):
    """One line with the measured figures (shown by pytest -rP)."""
    line = f"PARITY {name}: rel Linf per variable " + " ".join("%.2e" % e for e in err)
    if dterr is not None:
        line += f"; dt history {dterr:.2e}"
    print(line)


def stepped(h, U, nsteps):
    """nsteps of hydro_step_cfl (the benchmark's loop); returns the dt of every step."""
    dt = h.compute_dt(U)
    hist = torch.zeros((nsteps, h.nproblems), dtype=torch.float64, device="cuda")
    for s in range(nsteps):
        hist[s].copy_(dt)
        h.step_cfl(U, dt)
    return host(hist), dt


def test_sedov_3d_128_200_steps_whole_run(gb):
    lat = wl.lattice_3d(8, 8, 8)
    U0 = wl.sedov(lat)
    ref = U0.copy()
    hist_o, hits_o = Oracle(lat).run(ref, 200)
    h = gb.Hydro.from_lattice(lat)
    Ug = dev(U0)
    hist, _ = stepped(h, Ug, 200)
    out = host(Ug)
    err = relerr_per_var(to_global(out, lat), to_global(ref, lat))
    dterr = np.max(np.abs(hist[:, 0] / hist_o - 1))
    report("Sedov 128^3 x 200", err, dterr)
    assert np.all(err <= TOL_RUN), err
    assert dterr <= TOL_DT, dterr
    assert h.floor_hits() == hits_o == 0
    zs, ys, xs = lat.interior_slices()
    E0 = U0[:, 4, zs, ys, xs].sum()
    assert abs(out[:, 4, zs, ys, xs].sum() / E0 - 1) < 1e-12


def test_sedov_3d_256_50_steps_whole_run(gb):
    lat = wl.lattice_3d(16, 16, 16)
    U0 = wl.sedov(lat)
    h = gb.Hydro.from_lattice(lat)
    Ug = dev(U0)
    hist, _ = stepped(h, Ug, 50)
    out = host(Ug)
    del Ug
    torch.cuda.empty_cache()
    ref = U0
    hist_o, hits_o = Oracle(lat).run(ref, 50)
    err = relerr_per_var(to_global(out, lat), to_global(ref, lat))
    dterr = np.max(np.abs(hist[:, 0] / hist_o - 1))
    report("Sedov 256^3 x 50", err, dterr)
    assert np.all(err <= TOL_RUN), err
    assert dterr <= TOL_DT, dterr
    assert h.floor_hits() == hits_o == 0


def leaf_err(A, B, tl):
    """Per-variable relative error over leaf cells of both levels."""
    zs, ys, xs = tl.coarse.interior_slices()
    leaf = [b for b in range(tl.nblocks) if not (b < tl.n0 and tl.covered(b))]
    a = A[leaf][:, :, zs, ys, xs]
    b = B[leaf][:, :, zs, ys, xs]
    out = []
    for v in range(5):
        m = np.max(np.abs(b[:, v]))
        d = np.max(np.abs(a[:, v] - b[:, v]))
        out.append(d / m if m > 0 else (0.0 if d == 0 else np.inf))
    return np.array(out)


def test_refined_sedov_4096_plus_4096_50_steps_whole_run(gb):
    tl = wl.two_level(wl.lattice_3d(16, 16, 16), (4, 4, 4), (12, 12, 12))
    U0 = wl.sedov_two_level(tl)
    h = gb.Hydro.from_two_level(tl)
    Ug = dev(U0)
    h.fill_guardcells(Ug)
    hist, _ = stepped(h, Ug, 50)
    out = host(Ug)
    del Ug
    torch.cuda.empty_cache()
    ref = U0
    hist_o, hits_o = Oracle2(tl).run(ref, 50)
    err = leaf_err(out, ref, tl)
    dterr = np.max(np.abs(hist[:, 0] / hist_o - 1))
    report("two-level Sedov 4096+4096 blocks x 50", err, dterr)
    assert np.all(err <= TOL_RUN), err
    assert dterr <= TOL_DT, dterr
    assert h.floor_hits() == hits_o == 0


def test_ensemble_96_problems_100_steps_whole_run(gb):
    """The batched ensemble as the benchmark runs it (autotuned decomposition,
    100 steps in one captured graph); the dt of every step of every problem
    from the uncaptured advance, which must give the graph's bits."""
    probs = wl.ensemble(count=96, seed=0)
    lats = [l for l, _ in probs]
    U0 = np.concatenate([u for _, u in probs])
    h = gb.Hydro.from_batch(lats)
    Ug = dev(U0)
    h.autotune(Ug)
    dt = h.compute_dt(Ug)
    h.advance_graph(Ug, 100, dt)
    out = host(Ug)
    dt_end = host(dt)
    Up = dev(U0)
    dp = h.compute_dt(Up)
    hist = torch.zeros(100 * len(lats), dtype=torch.float64, device="cuda")
    h.advance(Up, 100, dp, hist)
    assert np.array_equal(host(Up), out) and np.array_equal(host(dp), dt_end)
    hist = host(hist).reshape(100, len(lats))
    del Ug, Up
    torch.cuda.empty_cache()
    worst, worst_dt = np.zeros(5), 0.0
    off = 0
    for i, (lat, u0) in enumerate(probs):
        ref = u0.copy()
        o = Oracle(lat)
        hist_o, hits_o = o.run(ref, 100)
        got = out[off:off + lat.nblocks]
        off += lat.nblocks
        err = relerr_per_var(to_global(got, lat), to_global(ref, lat))
        assert np.all(err <= TOL_RUN), (i, lat.global_cells, err)
        worst = np.maximum(worst, err)
        dterr = max(np.max(np.abs(hist[:, i] / hist_o - 1)), abs(dt_end[i] / o.compute_dt(ref) - 1))
        assert dterr <= TOL_DT, (i, dterr)
        worst_dt = max(worst_dt, dterr)
        assert hits_o == 0
    report("96-problem ensemble x 100 (worst problem per variable)", worst, worst_dt)
    assert h.floor_hits() == 0


def prim_to_cons_vjp_plain(W, lam, gamma=1.4):
    """Transposed Jacobian of U(W) = (rho, rho u, rho v, rho w, p/(gamma-1) +
    rho |u|^2 / 2) applied to lam, written from that definition."""
    rho, u, v, w, p = (W[:, k] for k in range(5))
    out = np.zeros_like(W)
    out[:, 0] = lam[:, 0] + u * lam[:, 1] + v * lam[:, 2] + w * lam[:, 3] + 0.5 * (u * u + v * v + w * w) * lam[:, 4]
    out[:, 1] = rho * (lam[:, 1] + u * lam[:, 4])
    out[:, 2] = rho * (lam[:, 2] + v * lam[:, 4])
    out[:, 3] = rho * (lam[:, 3] + w * lam[:, 4])
    out[:, 4] = lam[:, 4] / (gamma - 1.0)
    return out


def test_sod_like_256_gradient_vs_oracle_adjoint(gb):
    """Config-5 gradient: 256^2 in 16^2 blocks, sod_smooth, 50 steps, checkpoint
    every 10, loss = sum over interior cells of (rho - rho_target)^2 with
    rho_target = the final density + 0.01 N(0,1) (seed 7).  The GPU gradient
    with respect to the initial conserved state (CheckpointedRun) and to the
    initial primitives (the torch.autograd path) against the oracle's step
    adjoints chained backwards along the oracle's trajectory with the GPU's dt
    sequence, dt held fixed on both sides."""
    from paper_2401_03378_gb300.adjoint import CheckpointedRun, run_differentiable
    lat = wl.lattice_2d(16, 16, 16, 16, 4)
    zs, ys, xs = lat.interior_slices()
    mask = np.zeros(lat.shape)
    mask[:, :, zs, ys, xs] = 1.0
    W0 = wl.sod_smooth(lat, primitive=True)
    h = gb.Hydro.from_lattice(lat)
    run = CheckpointedRun(h, 50, every=10)
    UF = run.forward(h.prim_to_cons(dev(W0)))
    rng = np.random.default_rng(7)
    m0 = mask[:, 0]
    target = (host(UF)[:, 0] + 0.01 * rng.standard_normal(UF.shape[:1] + UF.shape[2:])) * m0
    lamF = np.zeros(lat.shape)
    lamF[:, 0] = 2.0 * (host(UF)[:, 0] - target) * m0
    lam0 = host(run.backward(dev(lamF)))
    gW = host(h.prim_to_cons_vjp(dev(W0), dev(lam0)))
    # the autograd path gives the same bits
    W = dev(W0).requires_grad_(True)
    U = run_differentiable(h, W, 50, every=10)
    loss = torch.sum(((U[:, 0] - dev(target)) * dev(m0)) ** 2)
    loss.backward()
    assert np.array_equal(host(W.grad)[:, :, zs, ys, xs], gW[:, :, zs, ys, xs])
    # the oracle along its own trajectory with the same dts
    o = Oracle(lat)
    states = [wl.sod_smooth(lat)]
    for s in range(50):
        X = states[-1].copy()
        o.step(X, run.dts[s])
        states.append(X)
    lo = np.zeros(lat.shape)
    lo[:, 0] = 2.0 * (states[-1][:, 0] - target) * m0
    for s in reversed(range(50)):
        lo = o.step_adjoint(states[s], run.dts[s], lo)
    e = relerr_per_var(to_global(lam0, lat), to_global(lo, lat))
    go = prim_to_cons_vjp_plain(W0, lo) * mask
    eW = relerr_per_var(to_global(gW, lat), to_global(go, lat))
    report("gradient 256^2 x 50, conserved", e)
    report("gradient 256^2 x 50, primitive", eW)
    assert np.all(e[[0, 1, 2, 4]] <= TOL_GRAD), e
    assert np.all(eW[[0, 1, 2, 4]] <= TOL_GRAD), eW
    # w is identically zero in 2-D: its adjoint is round-off of the others'
    scale = np.max(np.abs(to_global(lo, lat)[[1, 2]]))
    assert np.max(np.abs(to_global(lam0, lat)[3] - to_global(lo, lat)[3])) <= TOL_GRAD * scale
