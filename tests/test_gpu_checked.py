"""The checked build (libgbhydro_check.so, -DGBH_CHECK): every computed index
of every kernel is compared with its buffer's length, out-of-range indices
are counted and redirected.  Every step path runs through it: the count must
stay 0 and the results must equal the normal build's bit for bit (the
checks change no arithmetic).  The self-test shows that a planted index past
a buffer is counted."""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2401_03378_gb300 as pkg
    pkg.load()
    pkg.load(checked=True)
    return pkg


def violations(gb):
    n = C.c_longlong(-1)
    assert gb.load(checked=True).gbh_check_violations(C.byref(n)) == 0
    return n.value


def dev(U):
    return torch.from_numpy(np.ascontiguousarray(U)).cuda()


def test_selftest_counts_a_planted_index(gb):
    n = C.c_longlong(-1)
    assert gb.load(checked=True).gbh_check_selftest(C.byref(n)) == 0
    assert n.value == 1
    assert violations(gb) == 0


def both(gb, make, run):
    """run(hydro) -> list of tensors, on the normal and the checked build"""
    out = []
    for checked in (False, True):
        h = make(checked)
        out.append([t.clone() for t in run(h)])
        h.close()
    for a, b in zip(*out):
        assert torch.equal(a, b)
    assert violations(gb) == 0


UNIFORM = [
    (wl.lattice_3d(2, 2, 2, 16, 16, 16, 4), 2, False),
    (wl.lattice_3d(2, 3, 2, 8, 8, 8, 4, bc=("periodic", "outflow", "periodic")), 2, False),
    (wl.lattice_3d(3, 2, 2, 4, 4, 4, 4, bc="periodic"), 2, False),
    (wl.lattice_2d(4, 3, 16, 16, 4), 2, False),
    (wl.lattice_2d(3, 3, 8, 8, 2, bc=("periodic", "outflow")), 2, False),
    (wl.lattice_3d(2, 2, 2, 16, 16, 16, 4), 2, True),
    (wl.lattice_3d(2, 2, 2, 8, 8, 8, 6, bc="periodic"), 3, True),
    (wl.lattice_2d(3, 2, 16, 16, 6), 3, True),
    (wl.lattice_3d(2, 2, 2, 8, 8, 8, 4), 3, False),
]


def split_tiles(h, split):
    """Row bands of the stage kernel's plane tile on every ring width."""
    for ring in (0, 2, 4):
        h.set_tile_split(ring, split)


# the row-band split (2) exists for blocks of at least 8 cells per side
@pytest.mark.parametrize("lat,stages,tele,split", [u + (s,) for u in UNIFORM for s in (1, 2)
                                                   if s == 1 or u[0].n[0] >= 8])
def test_uniform_paths(gb, lat, stages, tele, split):
    U0 = wl.random_state(lat, seed=61, rough=True)

    def make(checked):
        h = gb.Hydro.from_lattice(lat, checked=checked)
        h.set_rk_stages(stages)
        h.set_telescoping(tele)
        split_tiles(h, split)
        return h

    def run(h):
        U = dev(U0)
        h.fill_guardcells(U)
        dt = h.compute_dt(U)
        h.advance(U, 3, dt)
        V = dev(U0)
        out = torch.zeros_like(V)
        h.stage(V, V, out, 1e-3, 0.5, 0.5, guarded=True)
        W = dev(U0)
        h.stage(W, None, out, 1e-3, 0.0, 1.0)
        assert h.check_state(U) == 0
        return [U, dt, out]
    both(gb, make, run)


@pytest.mark.parametrize("kchunk,ipc", [(8, 3), (0, 5)])
def test_decompositions_and_graph(gb, kchunk, ipc):
    lat = wl.lattice_3d(3, 2, 2, 16, 16, 16, 4)
    U0 = wl.sedov(lat)

    def make(checked):
        h = gb.Hydro.from_lattice(lat, checked=checked)
        h.set_decomposition(kchunk, ipc)
        return h

    def run(h):
        U = dev(U0)
        dt = h.compute_dt(U)
        h.advance_graph(U, 3, dt)
        return [U, dt]
    both(gb, make, run)


@pytest.mark.parametrize("region", ["box", "tripod"])
@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("stages,tele,ng", [(2, False, 4), (2, True, 4), (3, False, 6), (3, True, 6)])
def test_two_level_paths(gb, stages, tele, ng, split, region):
    c = wl.lattice_3d(4, 4, 4, 8, 8, 8, ng)
    tl = (wl.two_level(c, (1, 1, 1), (3, 3, 3)) if region == "box" else
          wl.two_level_blocks(c, [(1, 1, 1), (2, 1, 1), (1, 2, 1), (1, 1, 2)]))
    U0 = wl.sedov_two_level(tl)[tl.gpu_blocks]

    def make(checked):
        h = gb.Hydro.from_two_level(tl, checked=checked)
        h.set_rk_stages(stages)
        h.set_telescoping(tele)
        split_tiles(h, split)
        return h

    def run(h):
        U = dev(U0)
        h.fill_guardcells(U)
        dt = h.compute_dt(U)
        h.advance(U, 3, dt)
        return [U, dt]
    both(gb, make, run)


def test_batched_and_host_step(gb):
    probs = wl.ensemble(count=4, seed=8, choices=(32, 64))
    lats = [l for l, _ in probs]
    U0 = np.concatenate([u for _, u in probs])
    lat2 = wl.lattice_2d(40, 40, 8, 8, 4)
    S0 = wl.sod(lat2)

    def make(checked):
        return (gb.Hydro.from_batch(lats, checked=checked), gb.Hydro.from_lattice(lat2, checked=checked))

    out = []
    for checked in (False, True):
        hb, hs = make(checked)
        U = dev(U0)
        dt = hb.compute_dt(U)
        hb.advance(U, 3, dt)
        Sh = torch.from_numpy(S0.copy()).pin_memory()
        dth = np.zeros(1)
        for _ in range(2):
            hs.step_host(Sh, dth)
        out.append((U.clone(), dt.clone(), Sh.clone(), dth.copy()))
        hb.close()
        hs.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2], out[1][2]) and np.array_equal(out[0][3], out[1][3])
    assert violations(gb) == 0


@pytest.mark.parametrize("tele,stages,ng", [(False, 2, 4), (True, 2, 4), (True, 3, 6)])
def test_adjoint(gb, tele, stages, ng):
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8, ng, bc=("periodic", "outflow", "outflow"))
    U0 = wl.random_state(lat, seed=62, rough=False)
    rng = np.random.default_rng(63)
    L0 = rng.normal(size=U0.shape)

    def make(checked):
        h = gb.Hydro.from_lattice(lat, checked=checked)
        h.set_rk_stages(stages)
        h.set_telescoping(tele)
        return h

    def run(h):
        U, lam = dev(U0), dev(L0)
        a = h.step_adjoint(U, 1e-3, lam)
        b = h.stage_vjp(U, lam, 1e-3)
        W = h.prim_to_cons(U)
        c = h.prim_to_cons_vjp(U, lam)
        return [a, b, W, c]
    both(gb, make, run)


def test_static_step(gb):
    from tests.test_zz_no_alloc import _params
    lat = wl.lattice_3d(2, 2, 2, 16, 16, 16, 4)
    U0 = wl.sedov(lat)
    res = []
    for checked in (False, True):
        lib = gb.load(checked=checked)
        keep = []
        p = _params(lat, keep)
        U = dev(U0)
        for _ in range(2):
            assert lib.hydro_step_static(C.byref(p), U.data_ptr(), 1e-4, torch.cuda.current_stream().cuda_stream) == 0
        torch.cuda.synchronize()
        res.append(U)
    assert torch.equal(res[0], res[1])
    assert violations(gb) == 0
