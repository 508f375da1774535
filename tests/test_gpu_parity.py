"""GPU parity: libgbhydro.so (through its C ABI) against the FP64 CPU oracle.

Bar: relative L-infinity <= 1e-11 per conserved variable after the stated
step counts (exact zero where the oracle's variable is identically zero), dt
sequences <= 1e-12 relative; <= 1e-13 for single stages / tiny grids; bitwise
for the guard-cell fill (a copy).
"""
import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle
from tests.gridutil import from_global, relerr_per_var, to_global

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_RUN = 1e-11
TOL_DT = 1e-12
TOL_TINY = 1e-13


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


def interior_err(Ug, Uo, lat):
    return relerr_per_var(to_global(Ug, lat), to_global(Uo, lat))


LATTICES = [
    wl.lattice_2d(3, 2, 16, 16, 4),
    wl.lattice_2d(4, 4, 8, 8, 4, bc="periodic"),
    wl.lattice_2d(3, 3, 4, 4, 2, bc=("periodic", "outflow")),
    wl.lattice_3d(2, 2, 2, 4, 4, 4, 4),
    wl.lattice_3d(2, 3, 2, 8, 8, 8, 4, bc=("outflow", "periodic", "outflow")),
    wl.lattice_3d(2, 2, 3, 16, 16, 16, 4, bc="periodic"),
    wl.lattice_3d(1, 1, 2, 16, 16, 16, 4),
]


@pytest.mark.parametrize("lat", LATTICES)
def test_fill_guardcells_bitwise(gb, lat):
    U = wl.random_state(lat, seed=1)
    U = wl.poison_guards(U, lat, np.nan)
    ref = U.copy()
    Oracle(lat).fill_guardcells(ref)
    h = gb.Hydro.from_lattice(lat)
    Ug = dev(U)
    h.fill_guardcells(Ug)
    out = host(Ug)
    # every guard the oracle defines must match bit for bit
    assert np.array_equal(np.isnan(out), np.isnan(ref))
    assert np.array_equal(np.nan_to_num(out), np.nan_to_num(ref))


@pytest.mark.parametrize("lat", LATTICES)
def test_compute_dt(gb, lat):
    U = wl.random_state(lat, seed=2)
    ref = Oracle(lat).compute_dt(U)
    h = gb.Hydro.from_lattice(lat)
    dt = float(host(h.compute_dt(dev(U)))[0])
    assert abs(dt / ref - 1) < 1e-14


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("ab", [(0.0, 1.0), (0.5, 0.5), (0.75, 0.25)])
@pytest.mark.parametrize("guarded", [False, True])
def test_single_stage(gb, lat, ab, guarded):
    a, b = ab
    rough = lat.n[0] != 16
    Uin = wl.random_state(lat, seed=3, rough=rough)
    Un = wl.random_state(lat, seed=4, rough=rough)
    o = Oracle(lat)
    filled = Uin.copy()
    o.fill_guardcells(filled)
    dt = 0.3 * o.compute_dt(Uin)
    ref = Un.copy()
    o.stage(filled, Un, ref, dt, a, b)
    h = gb.Hydro.from_lattice(lat)
    src = filled if guarded else wl.poison_guards(Uin, lat, np.nan)
    Ug = dev(src)
    Uo = dev(Un)
    h.stage(Ug, dev(Un), Uo, dt, a, b, guarded=guarded)
    err = interior_err(host(Uo), ref, lat)
    assert np.all(err <= TOL_TINY), err


def test_tiny_brute_one_step(gb):
    """nxb = 4, 2x2x2 blocks, random valid states, one full step."""
    lat = wl.lattice_3d(2, 2, 2, 4, 4, 4, 4)
    U = wl.random_state(lat, seed=6)
    ref = U.copy()
    o = Oracle(lat)
    dt = o.compute_dt(U)
    o.step(ref, dt)
    h = gb.Hydro.from_lattice(lat)
    Ug = dev(U)
    h.step(Ug, dt)
    assert np.all(interior_err(host(Ug), ref, lat) <= TOL_TINY)


def run_both(gb, lat, U0, nsteps, threads=0):
    from oracle import oracle as orc
    if threads:
        orc.set_threads(threads)
    ref = U0.copy()
    hist_o, hits_o = Oracle(lat).run(ref, nsteps)
    h = gb.Hydro.from_lattice(lat)
    Ug = dev(U0)
    dt = h.compute_dt(Ug)
    hist = torch.zeros(nsteps, dtype=torch.float64, device="cuda")
    h.advance(Ug, nsteps, dt, hist)
    return host(Ug), host(hist), ref, hist_o, h, hits_o


def test_sod_2d_128_100_steps(gb):
    """2-D Sod, 128^2 as 8x8 blocks of 16^2 + 4 guards, gamma 1.4, CFL 0.8, 100 steps."""
    lat = wl.lattice_2d(8, 8)
    Ug, hist, ref, hist_o, h, hits_o = run_both(gb, lat, wl.sod(lat), 100)
    err = interior_err(Ug, ref, lat)
    dterr = np.max(np.abs(hist / hist_o - 1))
    print("PARITY Sod 128^2 x 100: rel Linf per variable " + " ".join("%.2e" % x for x in err)
          + f"; dt history {dterr:.2e}")
    assert np.all(err <= TOL_RUN), err
    assert dterr <= TOL_DT
    G = to_global(Ug, lat)
    assert np.all(G[2] == 0) and np.all(G[3] == 0)
    assert np.all(G == G[:, :, :1, :]), "rows must stay identical"
    assert h.floor_hits() == hits_o == 0


def test_sedov_3d_128_trajectory_and_sampled_last_step(gb):
    """3-D Sedov, 128^3 as 512 blocks of 16^3 + 4 guards.  The whole
    trajectory is compared for the first 20 steps; at 200 steps the GPU's
    last step is compared with the oracle's step from the same state, the
    dt with the oracle's dt, and conservation / octant symmetry are checked."""
    lat = wl.lattice_3d(8, 8, 8)
    U0 = wl.sedov(lat)
    Ug, hist, ref, hist_o, h, _ = run_both(gb, lat, U0, 20)
    assert np.all(interior_err(Ug, ref, lat) <= TOL_RUN)
    assert np.max(np.abs(hist / hist_o - 1)) <= TOL_DT
    # continue on the GPU to step 199, then one step on both from the same state
    Ugd = dev(Ug)
    dt = h.compute_dt(Ugd)
    h.advance(Ugd, 179, dt)
    snap = host(Ugd)
    o = Oracle(lat)
    dt_o = o.compute_dt(snap)
    assert abs(float(host(dt)[0]) / dt_o - 1) <= TOL_DT
    ref = snap.copy()
    o.step(ref, dt_o)
    h.step(Ugd, dt_o)
    last = host(Ugd)
    assert np.all(interior_err(last, ref, lat) <= TOL_TINY)
    zs, ys, xs = lat.interior_slices()
    E0 = U0[:, 4, zs, ys, xs].sum()
    assert abs(last[:, 4, zs, ys, xs].sum() / E0 - 1) < 1e-12
    G = to_global(last, lat)
    sgn = np.array([1, -1, 1, 1, 1.0])[:, None, None, None]
    assert np.max(relerr_per_var(sgn * G[:, :, :, ::-1], G)) < 1e-10


@pytest.mark.slow
def test_sedov_3d_256_50_steps_sampled(gb):
    """3-D Sedov at 256^3 (4096 blocks of 16^3 + 4 guards) in the launch
    configuration the benchmark times (hydro_advance, device dt): step 50 is
    compared with the oracle's step from the GPU's state after 49 steps."""
    lat = wl.lattice_3d(16, 16, 16)
    U0 = wl.sedov(lat)
    h = gb.Hydro.from_lattice(lat)
    Ug = dev(U0)
    dt = h.compute_dt(Ug)
    dt_first = float(host(dt)[0])
    o = Oracle(lat)
    assert abs(dt_first / o.compute_dt(U0) - 1) <= TOL_DT
    h.advance(Ug, 49, dt)
    snap = host(Ug)
    dt_o = o.compute_dt(snap)
    assert abs(float(host(dt)[0]) / dt_o - 1) <= TOL_DT
    ref = snap.copy()
    o.step(ref, dt_o)
    h.step(Ug, dt_o)
    assert np.all(interior_err(host(Ug), ref, lat) <= TOL_TINY)
    assert h.floor_hits() == 0


@pytest.mark.slow
@pytest.mark.parametrize("ng,stages,tele", [(4, 2, True), (4, 3, False), (6, 3, True)])
def test_sedov_3d_256_variants_sampled(gb, ng, stages, tele):
    """The stepper variants bench.py times at 256^3 (telescoping two-stage,
    three-stage, telescoping three-stage on 6 guard cells), in that launch
    configuration: 19 steps with the device dt, then step 20 against the
    oracle's step of the same variant from the GPU's state."""
    lat = wl.lattice_3d(16, 16, 16, 16, 16, 16, ng)
    U0 = wl.sedov(lat)
    h = gb.Hydro.from_lattice(lat)
    h.set_rk_stages(stages)
    h.set_telescoping(tele)
    Ug = dev(U0)
    dt = h.compute_dt(Ug)
    h.advance(Ug, 19, dt)
    snap = host(Ug)
    o = Oracle(lat)
    dt_o = o.compute_dt(snap)
    assert abs(float(host(dt)[0]) / dt_o - 1) <= TOL_DT
    ref = snap.copy()
    o.step(ref, dt_o, telescoping=tele, stages=stages)
    h.step(Ug, dt_o)
    assert np.all(interior_err(host(Ug), ref, lat) <= TOL_TINY)
    assert h.floor_hits() == 0
    h.close()


def test_poisoned_guards_have_no_effect(gb):
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8, 4)
    U = wl.random_state(lat, seed=9)
    h = gb.Hydro.from_lattice(lat)
    outs = []
    for src in (U, wl.poison_guards(U, lat, np.nan)):
        Ug = dev(src)
        h.step(Ug, 1e-3)
        outs.append(to_global(host(Ug), lat))
    assert np.all(np.isfinite(outs[1]))
    assert np.array_equal(outs[0], outs[1])


def test_repeatable_and_step_variants_agree(gb):
    lat = wl.lattice_3d(2, 2, 2, 16, 16, 16, 4)
    U = wl.sedov(lat)
    h = gb.Hydro.from_lattice(lat)
    res = []
    for _ in range(2):
        Ug = dev(U)
        dt = h.compute_dt(Ug)
        h.advance(Ug, 5, dt)
        res.append(host(Ug))
    assert np.array_equal(res[0], res[1])
    # host-dt steps with the same dt sequence give the same bits
    Ug = dev(U)
    hist = torch.zeros(5, dtype=torch.float64, device="cuda")
    dt = h.compute_dt(Ug)
    h.advance(Ug, 5, dt, hist)
    hh = host(hist)
    Ug2 = dev(U)
    for s in range(5):
        h.step(Ug2, float(hh[s]))
    zs, ys, xs = lat.interior_slices()
    assert np.array_equal(host(Ug2)[:, :, zs, ys, xs], host(Ug)[:, :, zs, ys, xs])
    # host-buffer entry point gives the same bits as the device path
    Uh = U.copy()
    hist_h = np.zeros(5)
    h.advance_host(Uh, 5, hist_h)
    assert np.array_equal(Uh[:, :, zs, ys, xs], res[0][:, :, zs, ys, xs])
    assert np.array_equal(hist_h, hh)
    # and with a host state of the interior cells only (pageable, then pinned)
    for pinned in (False, True):
        Ui = np.ascontiguousarray(U[:, :, zs, ys, xs])
        Ui = torch.from_numpy(Ui).pin_memory() if pinned else Ui
        hist_i = np.zeros(5)
        h.advance_host(Ui, 5, hist_i, interior=True)
        got = Ui.numpy() if pinned else Ui
        assert np.array_equal(got, res[0][:, :, zs, ys, xs])
        assert np.array_equal(hist_i, hh)
    with pytest.raises(ValueError):
        h.advance_host(U.copy(), 5, None, interior=True)       # the padded shape is not that layout


def test_checkpoint_resume_bitwise(gb, tmp_path):
    """Checkpoint / resume: the state is plain tensors, so torch.save of U and
    the device dt after 10 steps, a fresh context and a load, then 10 more
    steps give the same bits as 20 uninterrupted steps (uniform and two-level)."""
    cases = [(wl.lattice_3d(2, 2, 2, 16, 16, 16, 4), None),
             (None, wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4), (1, 1, 1), (3, 3, 3)))]
    for lat, tl in cases:
        U0 = wl.sedov(lat) if tl is None else wl.sedov_two_level(tl)
        make = (lambda: gb.Hydro.from_lattice(lat)) if tl is None else (lambda: gb.Hydro.from_two_level(tl))
        h = make()
        A = dev(U0)
        if tl is not None:
            h.fill_guardcells(A)
        da = h.compute_dt(A)
        h.advance(A, 20, da)
        B = dev(U0)
        if tl is not None:
            h.fill_guardcells(B)
        db = h.compute_dt(B)
        h.advance(B, 10, db)
        path = tmp_path / "ckpt.pt"
        torch.save({"U": B.cpu(), "dt": db.cpu(), "step": 10}, path)
        h.close()
        del B, db
        ck = torch.load(path)
        h2 = make()
        C, dc = ck["U"].cuda(), ck["dt"].cuda()
        h2.advance(C, 20 - ck["step"], dc)
        assert torch.equal(A, C) and torch.equal(da, dc)


@pytest.mark.parametrize("kind", ["3d", "2d_many_chunks", "periodic_z", "batched", "telescoping"])
def test_step_host_equals_device_steps_bitwise(gb, kind):
    """hydro_step_host (copies overlapped with the stages, chunked by blocks)
    gives hydro_step_cfl's bits and dt, call after call."""
    if kind == "batched":
        probs = wl.ensemble(count=5, seed=4, choices=(64, 128))
        lats = [l for l, _ in probs]
        U0 = np.concatenate([u for _, u in probs])
        make = lambda: gb.Hydro.from_batch(lats)
        sl = lats[0].interior_slices()
    else:
        lat = {"3d": wl.lattice_3d(16, 8, 8, 8, 8, 8, 4),
               "2d_many_chunks": wl.lattice_2d(64, 64, 8, 8, 4),
               "periodic_z": wl.lattice_3d(8, 8, 16, 8, 8, 8, 4, bc=("outflow", "outflow", "periodic")),
               "telescoping": wl.lattice_3d(8, 8, 16, 8, 8, 8, 4)}[kind]
        U0 = wl.sedov(lat) if lat.ndim == 3 else wl.sod(lat)
        make = lambda: gb.Hydro.from_lattice(lat)
        sl = lat.interior_slices()
    hd, hh = make(), make()
    if kind == "telescoping":
        hd.set_telescoping(True)
        hh.set_telescoping(True)
    D = dev(U0)
    dt = hd.compute_dt(D)
    Uh = torch.from_numpy(U0.copy()).pin_memory()
    dth = np.zeros(hh.nproblems)
    zs, ys, xs = sl
    for _ in range(3):
        hd.step_cfl(D, dt)
        hh.step_host(Uh, dth)
        assert np.array_equal(host(D)[:, :, zs, ys, xs], Uh.numpy()[:, :, zs, ys, xs])
        assert np.array_equal(host(dt), dth)


@pytest.mark.parametrize("kind", ["3d", "2d_many_chunks", "periodic_z", "batched", "pageable", "telescoping",
                                  "three_stages", "two_level"])
def test_step_host_interior_equals_device_steps_bitwise(gb, kind):
    """hydro_step_host_interior (a host state of the interior cells only; staged,
    scattered into the padded device state and gathered back chunk by chunk)
    gives hydro_step_cfl's interior bits and dt, call after call, pipelined
    and in the step forms that run unpipelined (telescoping, three stages,
    two levels), from pinned and from pageable host memory."""
    if kind == "batched":
        probs = wl.ensemble(count=5, seed=4, choices=(64, 128))
        lats = [l for l, _ in probs]
        U0 = np.concatenate([u for _, u in probs])
        make = lambda: gb.Hydro.from_batch(lats)
    elif kind == "two_level":
        from tests.test_gpu_prim_carry import smooth_two_level
        tl = wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4), (1, 1, 1), (3, 3, 3))
        U0 = smooth_two_level(tl, 31)[tl.gpu_blocks]
        make = lambda: gb.Hydro.from_two_level(tl)
    else:
        lat = {"3d": wl.lattice_3d(16, 8, 8, 8, 8, 8, 4),
               "2d_many_chunks": wl.lattice_2d(64, 64, 8, 8, 4),
               "periodic_z": wl.lattice_3d(8, 8, 16, 8, 8, 8, 4, bc=("outflow", "outflow", "periodic")),
               "pageable": wl.lattice_3d(8, 8, 8, 16, 16, 16, 4),
               "telescoping": wl.lattice_3d(8, 8, 16, 8, 8, 8, 4),
               "three_stages": wl.lattice_3d(8, 8, 8, 8, 8, 8, 4)}[kind]
        U0 = wl.sedov(lat) if lat.ndim == 3 else wl.sod(lat)
        make = lambda: gb.Hydro.from_lattice(lat)
    hd, hh = make(), make()
    if kind == "telescoping":
        hd.set_telescoping(True)
        hh.set_telescoping(True)
    if kind == "three_stages":
        hd.set_rk_stages(3)
        hh.set_rk_stages(3)
    n = hh.interior_shape
    gz = hh.nguard if hh.ndim == 3 else 0
    g = hh.nguard
    interior = lambda A: A[:, :, gz:gz + n[2], g:g + n[3], g:g + n[4]]
    D = dev(U0)
    dt = hd.compute_dt(D)
    Ui = np.ascontiguousarray(interior(U0))
    Uh = Ui.copy() if kind == "pageable" else torch.from_numpy(Ui).pin_memory()
    dth = np.zeros(hh.nproblems)
    for _ in range(3):
        hd.step_cfl(D, dt)
        hh.step_host_interior(Uh, dth)
        got = Uh if kind == "pageable" else Uh.numpy()
        assert np.array_equal(interior(host(D)), got)
        assert np.array_equal(host(dt), dth)
    with pytest.raises(ValueError):
        hh.step_host_interior(np.zeros(hh.shape), dth)     # the padded shape is not this call's layout


@pytest.mark.parametrize("drift", [4.0, -4.0, 0.0])
def test_supersonic_faces(gb, drift):
    """Rough states with velocities drift + U(-3, 3) in every direction (Mach up
    to ~10): most faces have the whole wave fan on one side, the HLLC branch
    F = F_L (or F_R) that subsonic data never takes."""
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8, 4, bc="periodic")
    rng = np.random.default_rng(71)
    shape = (lat.nblocks,) + lat.padded
    rho, p = rng.uniform(0.5, 2.0, shape), rng.uniform(0.5, 2.0, shape)
    vel = drift + rng.uniform(-3.0, 3.0, (3,) + shape)
    U = wl._assemble(lat, rho, vel[0], vel[1], vel[2], p, 1.4)
    c = np.sqrt(1.4 * p / rho)
    if drift:
        assert np.mean(np.abs(vel[0]) > c) > 0.5
    o = Oracle(lat)
    dt = o.compute_dt(U)
    ref = U.copy()
    hits = o.step(ref, dt)
    h = gb.Hydro.from_lattice(lat)
    Ug = dev(U)
    h.step(Ug, dt)
    assert np.all(interior_err(host(Ug), ref, lat) <= TOL_TINY)
    assert h.floor_hits() == hits


@pytest.mark.slow
def test_state_beyond_2_31_elements(gb):
    """512^3 as 32768 blocks of 16^3 + 4 guards: 2.26e9 doubles per state, so
    every offset needs 64-bit arithmetic.  An x-only Sod problem must give
    bit-identical (y, z) rows equal to the 32 x 1 x 1-block lattice's result."""
    big = wl.lattice_3d(32, 32, 32, 16, 16, 16, 4)
    import dataclasses
    small = dataclasses.replace(wl.lattice_3d(32, 1, 1, 16, 16, 16, 4, bc=("outflow", "periodic", "periodic")),
                                extent=(1.0, 1.0 / 32, 1.0 / 32))
    assert small.dx == big.dx
    assert big.nblocks * 5 * np.prod(big.padded) > 2 ** 31
    Us = dev(wl.sod(small))
    hs = gb.Hydro.from_lattice(small)
    Ub = Us.index_select(0, torch.arange(32, device="cuda").repeat(32 * 32))
    hb = gb.Hydro.from_lattice(big)
    ds, db = hs.compute_dt(Us), hb.compute_dt(Ub)
    assert torch.equal(ds, db)
    hs.advance(Us, 3, ds)
    hb.advance(Ub, 3, db)
    assert torch.equal(ds, db)
    zs, ys, xs = big.interior_slices()
    got = Ub.view(32 * 32, 32, 5, *big.padded)[:, :, :, zs, ys, xs]
    ref = Us[:, :, zs, ys, xs]
    for r in range(0, 32 * 32, 64):
        assert torch.equal(got[r:r + 64], ref.expand(min(64, 32 * 32 - r), *ref.shape))
    del Ub, got
    torch.cuda.empty_cache()


def test_periodic_conservation(gb):
    lat = wl.lattice_3d(2, 2, 2, 16, 16, 16, 4, bc="periodic")
    U = wl.random_state(lat, seed=12, rough=True)
    zs, ys, xs = lat.interior_slices()
    before = U[:, :, zs, ys, xs].sum(axis=(0, 2, 3, 4))
    scale = np.abs(U[:, :, zs, ys, xs]).sum(axis=(0, 2, 3, 4))
    h = gb.Hydro.from_lattice(lat)
    Ug = dev(U)
    dt = h.compute_dt(Ug)
    h.advance(Ug, 20, dt)
    after = host(Ug)[:, :, zs, ys, xs].sum(axis=(0, 2, 3, 4))
    assert np.all(np.abs(after - before) <= 20 * 8 * np.finfo(float).eps * scale)


def test_errors_and_floors(gb):
    lat = wl.lattice_2d(2, 2, 8, 8, 4)
    U = wl.random_state(lat, seed=3)
    U[1, 4, 0, 6, 6] = -1.0
    h = gb.Hydro.from_lattice(lat)
    Ug = dev(U)
    assert h.check_state(Ug) == 1
    with pytest.raises(gb.GbhError) as ei:
        h.step(Ug, -1.0)
    assert ei.value.code == -1
    with pytest.raises(gb.GbhError):
        h.step(Ug, float("nan"))
    o = Oracle(lat)
    f = U.copy()
    o.fill_guardcells(f)
    out = f.copy()
    hits_o = o.stage(f, None, out, 1e-4, 0.0, 1.0)
    h.floor_hits()
    Uo = dev(U)
    h.stage(dev(U), None, Uo, 1e-4, 0.0, 1.0)
    assert h.floor_hits() == hits_o == 1
    assert h.check_state(dev(wl.random_state(lat, seed=4))) == 0


def test_fp64_probe_runs(gb):
    out = torch.zeros(152 * 4 * 256, dtype=torch.float64, device="cuda")
    for form in range(5):
        out.zero_()
        gb.fp64_probe(152 * 4, 256, 1000, out, 32, form)
        assert torch.isfinite(out).all() and bool((out != 0).all())
    with pytest.raises(Exception):
        gb.fp64_probe(152 * 4, 256, 1000, out, 32, 5)


def test_op_count_probe_runs(gb):
    """Every building block of the instruction-count probe runs and keeps its
    chained inputs finite (the chain only flips the last mantissa bit)."""
    from paper_2401_03378_gb300.probe import OP_COUNT, op_count, op_count_inputs
    for fn in OP_COUNT:
        io = op_count(fn, 4, 64, 16)
        ref = op_count_inputs(fn, 4 * 64)
        got = host(io)
        assert np.all(np.isfinite(got))
        rel = np.abs(got / ref.numpy() - 1)
        assert np.max(rel) <= 4 * np.finfo(float).eps
    with pytest.raises(Exception):
        op_count(8, 4, 64, 16)


def test_refined_reciprocal_and_roots_within_two_ulp(gb):
    """The kernels' reciprocal, 1/sqrt and sqrt (hardware seed + one
    third-order refinement) stay within 2 ulp of the IEEE results over the
    value ranges the scheme produces (and far beyond)."""
    import ctypes
    rng = np.random.default_rng(21)
    x = np.concatenate([10.0 ** rng.uniform(-14, 14, 400000), rng.uniform(0.5, 2.0, 100000),
                        np.array([1.0, 2.0, 0.5, 3.0, 1e-14, 1e14])])
    xd = dev(x)
    out = torch.empty(6 * len(x), dtype=torch.float64, device="cuda")
    lib = gb.load()
    assert lib.gbh_fastmath_selftest(xd.data_ptr(), out.data_ptr(), len(x),
                                     torch.cuda.current_stream().cuda_stream) == 0
    o = host(out).reshape(6, -1)
    for k in range(3):
        fast, ieee = o[2 * k], o[2 * k + 1]
        ulp = np.abs(fast - ieee) / np.spacing(np.abs(ieee))
        assert np.max(ulp) <= 2.0, (k, np.max(ulp))


@pytest.mark.parametrize("telescoping", [False, True])
@pytest.mark.parametrize("ndim,bc", [(3, "outflow"), (3, "periodic"), (2, "outflow"), (2, "periodic")])
def test_block_decomposition_invisible_bitwise(gb, ndim, bc, telescoping):
    """The same global state cut into blocks of 16, 8 or 4 cells per side gives the
    same state and dt history bit for bit (every face flux and every cell update
    is the same arithmetic on the same values, whichever block computes it)."""
    if ndim == 3:
        cuts = ((2, 16), (4, 8), (8, 4))
        mk = lambda nb, n: wl.lattice_3d(nb, nb, nb, n, n, n, 4, bc=bc)
    else:
        cuts = ((4, 16), (8, 8), (16, 4))
        mk = lambda nb, n: wl.lattice_2d(nb, nb, n, n, 4, bc=bc)
    Gl = to_global(wl.random_state(mk(*cuts[0]), seed=31, rough=True), mk(*cuts[0]))
    results = []
    for nb, n in cuts:
        lat = mk(nb, n)
        h = gb.Hydro.from_lattice(lat)
        h.set_telescoping(telescoping)
        U = dev(from_global(Gl, lat))
        dt = h.compute_dt(U)
        hist = torch.zeros(4, dtype=torch.float64, device="cuda")
        h.advance(U, 4, dt, hist)
        results.append((to_global(host(U), lat), host(hist)))
    for G, hh in results[1:]:
        assert np.array_equal(hh, results[0][1])
        assert np.array_equal(G, results[0][0])


def test_axis_permutation(gb):
    """Relabelling the axes (new x, y, z = old y, z, x, momenta alike) permutes the
    result up to the order of the x, y, z flux terms (<= 1e-14)."""
    lat = wl.lattice_3d(2, 2, 2, 16, 16, 16, 4)
    Gl = to_global(wl.random_state(lat, seed=8, rough=False), lat)

    def perm(A):
        return np.ascontiguousarray(A[[0, 2, 3, 1, 4]].transpose(0, 3, 1, 2))
    h = gb.Hydro.from_lattice(lat)
    out = []
    for G in (Gl, perm(Gl)):
        U = dev(from_global(G, lat))
        dt = h.compute_dt(U)
        hist = torch.zeros(4, dtype=torch.float64, device="cuda")
        h.advance(U, 4, dt, hist)
        out.append((to_global(host(U), lat), host(hist)))
    assert np.max(np.abs(out[0][1] - out[1][1]) / out[0][1]) < 1e-15
    assert np.max(relerr_per_var(out[1][0], perm(out[0][0]))) < 1e-14
