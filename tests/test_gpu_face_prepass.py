"""The face pre-pass (gbh_set_face_prepass): before each interior stage of a
uniform, batched or two-level context a kernel solves the flux through every
block face once, and the stage reads those fluxes instead of solving each shared face in
both blocks.  Every entry point gives the states, dt, dt histories and floor
counts of the pre-pass off, bit for bit: the same face states and HLLC
arithmetic on the same halo."""
import numpy as np
import pytest

import workloads as wl
from tests.test_gpu_prim_carry import LATTICES, paths, with_floors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2401_03378_gb300 as pkg
    pkg.load()
    return pkg


def on_and_off(make, U0, nsteps=4):
    res = []
    for pre in (True, False):
        h = make()
        h.set_face_prepass(pre)
        assert h.face_prepass() == pre
        res.append(paths(h, U0, nsteps))
        h.close()
    (a, ha), (b, hb) = res
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert ha == hb
    return ha


@pytest.mark.parametrize("stages", [2, 3])
@pytest.mark.parametrize("name", list(LATTICES))
def test_every_entry_point_bitwise(gb, name, stages):
    lat = LATTICES[name]
    U0 = wl.random_state(lat, seed=83, rough=True)

    def make():
        h = gb.Hydro.from_lattice(lat)
        h.set_rk_stages(stages)
        return h
    assert on_and_off(make, U0) == [0] * 6


@pytest.mark.parametrize("name", ["3d-16-outflow", "2d-16-outflow", "3d-4-periodic"])
def test_floor_counts_equal(gb, name):
    lat = LATTICES[name]
    hits = on_and_off(lambda: gb.Hydro.from_lattice(lat), with_floors(lat, 91), nsteps=3)
    assert all(x > 0 for x in hits), hits


@pytest.mark.parametrize("kchunk,ipc,split,carry", [(8, 1, 1, True), (0, 3, 1, True), (0, 1, 2, True),
                                                    (0, 1, 1, False), (8, 2, 1, False)])
def test_decompositions_bitwise(gb, kchunk, ipc, split, carry):
    """z-chunks (the pre-pass faces only at the block's own bottom and top),
    several items per CTA, the row-band tile (which solves its faces itself),
    with and without the primitive carry."""
    lat = wl.lattice_3d(3, 2, 2, 16, 16, 16, 4, bc=("periodic", "outflow", "periodic"))
    U0 = wl.random_state(lat, seed=84, rough=True)

    def make():
        h = gb.Hydro.from_lattice(lat)
        h.set_decomposition(kchunk, ipc)
        h.set_tile_split(0, split)
        h.set_prim_carry(carry)
        return h
    on_and_off(make, U0)


def test_batched_and_other_contexts(gb):
    probs = wl.ensemble(count=5, seed=4, choices=(32, 64, 128))
    lats = [l for l, _ in probs]
    U0 = np.concatenate([u for _, u in probs])
    on_and_off(lambda: gb.Hydro.from_batch(lats), U0)
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8, 4)

    def make():
        h = gb.Hydro.from_lattice(lat)
        h.set_telescoping(True)
        return h
    on_and_off(make, wl.random_state(lat, seed=85, rough=True))
    assert gb.Hydro.from_lattice(lat).face_prepass()                    # on by default in 3-D
    assert not gb.Hydro.from_lattice(wl.lattice_2d(2, 2, 8, 8, 4)).face_prepass()   # off in 2-D


TWO_LEVEL = [wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4), (1, 1, 1), (3, 3, 3)),
             wl.two_level_blocks(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4, bc="periodic"),
                                 [(1, 1, 1), (2, 1, 1), (1, 2, 1), (1, 1, 2)]),
             wl.two_level(wl.lattice_3d(4, 4, 3, 16, 16, 16, 4, bc=("periodic", "outflow", "outflow")),
                          (1, 1, 1), (3, 3, 2))]


@pytest.mark.parametrize("stages", [2, 3])
@pytest.mark.parametrize("ti", range(len(TWO_LEVEL)), ids=["box", "tripod-periodic", "16-mixed"])
def test_two_level_bitwise(gb, ti, stages):
    """All-levels two-level steps: same-level faces solved once, faces onto the
    coarser level by each side from its own halo (the fine block's prolonged
    guard cells), the flux registers filled from the pre-pass fluxes."""
    from tests.test_gpu_prim_carry import smooth_two_level
    tl = TWO_LEVEL[ti]

    def make():
        h = gb.Hydro.from_two_level(tl)
        h.set_rk_stages(stages)
        return h
    assert on_and_off(make, smooth_two_level(tl, 12)[tl.gpu_blocks]) == [0] * 6


def test_two_level_batched_bitwise(gb):
    from tests.test_gpu_prim_carry import smooth_two_level
    tls = [wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4), (1, 1, 1), (3, 3, 3))] * 3
    U0 = np.concatenate([smooth_two_level(t, 20 + i)[t.gpu_blocks] for i, t in enumerate(tls)])
    on_and_off(lambda: gb.Hydro.from_two_level_batch(tls), U0)


@pytest.mark.parametrize("chunks", [0, 3, 5, 64])
@pytest.mark.parametrize("interior", [False, True])
def test_host_pipeline_chunks_bitwise(gb, chunks, interior):
    """The pipelined host-buffer steps run the face pre-pass per chunk of
    consecutive blocks: a low face whose neighbour lies in a later chunk (here
    the periodic wraps in x, y and z) is solved by the block itself, a high
    face is written into the neighbour's slot only for a neighbour in this or
    a later chunk.  States and dt equal hydro_step_cfl's with the pre-pass off,
    for chunks of one block, uneven chunks and the default chunking."""
    lat = wl.lattice_3d(4, 4, 4, 8, 8, 8, 4, bc="periodic")
    U0 = wl.random_state(lat, seed=86, rough=True)
    hd, hh = gb.Hydro.from_lattice(lat), gb.Hydro.from_lattice(lat)
    hd.set_face_prepass(False)
    hh.set_host_pipeline(chunks)
    assert hh.face_prepass()
    sl = (slice(None), slice(None)) + tuple(lat.interior_slices())
    D = torch.from_numpy(U0.copy()).cuda()
    dt = hd.compute_dt(D)
    Uh = torch.from_numpy(np.ascontiguousarray(U0[sl]) if interior else U0.copy()).pin_memory()
    dth = np.zeros(1)
    for _ in range(3):
        hd.step_cfl(D, dt)
        (hh.step_host_interior if interior else hh.step_host)(Uh, dth)
        got = Uh.numpy() if interior else Uh.numpy()[sl]
        assert np.array_equal(D.cpu().numpy()[sl], got)
        assert np.array_equal(dt.cpu().numpy(), dth)
    hd.close()
    hh.close()
