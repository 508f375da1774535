"""The primitive carry (gbh_set_prim_carry): every stage's epilogue leaves the
primitive variables of its output for the next stage, which then reads them
instead of converting its input (calcEos once per stage, after updSoln, as in
Alg. "Intra stage calculations for Spark"); on two-level grids the restriction,
the prolongation and the flux correction add the primitives of the cells they
write.  With the carry on, every entry point gives the states, dt and dt
histories of the carry off bit for bit, and the same floor counts; telescoping
steps never carry."""
import numpy as np
import pytest

import workloads as wl
from oracle.oracle import Oracle

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


LATTICES = {
    "3d-16-outflow": wl.lattice_3d(2, 2, 2, 16, 16, 16, 4),
    "3d-8-mixed": wl.lattice_3d(3, 2, 2, 8, 8, 8, 4, bc=("periodic", "outflow", "periodic")),
    "3d-4-periodic": wl.lattice_3d(3, 3, 2, 4, 4, 4, 4, bc="periodic"),
    "3d-16x16x8": wl.lattice_3d(2, 2, 3, 16, 16, 8, 4),
    "3d-8x8x12-mixed": wl.lattice_3d(3, 2, 2, 8, 8, 12, 6, bc=("periodic", "outflow", "periodic")),
    "2d-16-outflow": wl.lattice_2d(4, 3, 16, 16, 4),
    "2d-8-mixed-ng2": wl.lattice_2d(3, 3, 8, 8, 2, bc=("periodic", "outflow")),
}


def with_floors(lat, seed):
    """A rough random state in which a few interior cells have E < |m|^2 / (2 rho):
    their pressure is floored by every conversion until the flow refills them."""
    U = wl.random_state(lat, seed=seed, rough=True)
    zs, ys, xs = lat.interior_slices()
    rng = np.random.default_rng(seed + 1)
    for _ in range(4):
        b = int(rng.integers(lat.nblocks))
        k = zs.start + int(rng.integers(zs.stop - zs.start))
        j = ys.start + int(rng.integers(ys.stop - ys.start))
        i = xs.start + int(rng.integers(xs.stop - xs.start))
        c = U[b, :, k, j, i]
        ke = 0.5 * (c[1] ** 2 + c[2] ** 2 + c[3] ** 2) / c[0]
        U[b, 4, k, j, i] = 0.5 * ke
    return U


def paths(h, U0, nsteps=4):
    """Every entry point that steps a state, on copies of U0: their states,
    dt and dt histories, and the floor count of each."""
    out, hits = [], []
    h.floor_hits()
    U = dev(U0)
    h.fill_guardcells(U)
    dt = h.compute_dt(U)
    d = float(host(dt)[0])
    A = U.clone()
    h.step(A, d)
    hits.append(h.floor_hits())
    B = U.clone()
    dB = dt.clone()
    h.step_cfl(B, dB)
    hits.append(h.floor_hits())
    C = U.clone()
    dC = dt.clone()
    hist = torch.zeros(nsteps * h.nproblems, dtype=torch.float64, device="cuda")
    h.advance(C, nsteps, dC, hist)
    hits.append(h.floor_hits())
    D = U.clone()
    dD = dt.clone()
    h.advance_graph(D, nsteps, dD)
    hits.append(h.floor_hits())
    Uh = torch.from_numpy(host(U)).pin_memory()
    dth = np.zeros(h.nproblems)
    for _ in range(2):
        h.step_host(Uh, dth)
    hits.append(h.floor_hits())
    Vh = torch.from_numpy(host(U)).pin_memory()
    hh = np.zeros(nsteps * h.nproblems)
    h.advance_host(Vh, nsteps, hh)
    hits.append(h.floor_hits())
    out += [A, B, dB, C, dC, hist, D, dD, Uh.cuda(), torch.from_numpy(dth).cuda(), Vh.cuda(),
            torch.from_numpy(hh).cuda()]
    return out, hits


def on_and_off(gb, make, U0, nsteps=4):
    res = []
    for carry in (True, False):
        h = make()
        h.set_prim_carry(carry)
        assert h.prim_carry() == carry
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
    U0 = wl.random_state(lat, seed=81, rough=True)

    def make():
        h = gb.Hydro.from_lattice(lat)
        h.set_rk_stages(stages)
        return h
    assert on_and_off(gb, make, U0) == [0] * 6


@pytest.mark.parametrize("name", ["3d-16-outflow", "2d-16-outflow", "3d-4-periodic"])
def test_floor_counts_equal_and_match_the_oracle(gb, name):
    lat = LATTICES[name]
    U0 = with_floors(lat, 90)
    hits = on_and_off(gb, lambda: gb.Hydro.from_lattice(lat), U0, nsteps=3)
    assert all(x > 0 for x in hits), hits
    # hydro_advance over 3 steps counts what the oracle's 3-step run counts
    ref = U0.copy()
    _, hits_o = Oracle(lat).run(ref, 3)
    assert hits[2] == hits_o


@pytest.mark.parametrize("kchunk,ipc,split", [(8, 1, 1), (0, 3, 1), (0, 1, 2), (8, 2, 2)])
def test_decompositions_bitwise(gb, kchunk, ipc, split):
    lat = wl.lattice_3d(3, 2, 2, 16, 16, 16, 4)
    U0 = wl.sedov(lat)

    def make():
        h = gb.Hydro.from_lattice(lat)
        h.set_decomposition(kchunk, ipc)
        h.set_tile_split(0, split)
        return h
    on_and_off(gb, make, U0)


def test_batched_ensemble_bitwise(gb):
    probs = wl.ensemble(count=5, seed=4, choices=(32, 64, 128))
    lats = [l for l, _ in probs]
    U0 = np.concatenate([u for _, u in probs])
    on_and_off(gb, lambda: gb.Hydro.from_batch(lats), U0)


TWO_LEVEL = {
    "box-3d": wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4), (1, 1, 1), (3, 3, 3)),
    "L-2d": wl.two_level_blocks(wl.lattice_2d(5, 5, 8, 8, 4), [(1, 1), (2, 1), (3, 1), (1, 2), (1, 3)]),
    "tripod-3d-periodic": wl.two_level_blocks(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4, bc="periodic"),
                                              [(1, 1, 1), (2, 1, 1), (1, 2, 1), (1, 1, 2)]),
    "box-2d-16": wl.two_level(wl.lattice_2d(4, 4, 16, 16, 4), (1, 1), (3, 3)),
}


def smooth_two_level(tl, seed):
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, 8)
    nd = tl.coarse.ndim

    def fn(X, Y, Z):
        s = np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1])
        if nd == 3:
            s = s * np.cos(2 * np.pi * Z + ph[2])
        return (1 + 0.4 * s, 0.5 * np.sin(2 * np.pi * Y + ph[3]) + 0 * X, 0.4 * np.cos(2 * np.pi * X + ph[4]),
                (0.3 * np.sin(2 * np.pi * X + ph[5]) if nd == 3 else 0 * X), 1 + 0.3 * s)
    return wl.two_level_state(tl, fn)


def floor_cells(tl, U, seed):
    """Plant E = |m|^2 / (4 rho) (a negative pressure, floored) in a few coarse
    leaf cells next to the refined region, whose flux correction changes them
    after every stage, and in a few fine cells at the coarse-fine boundary."""
    c = tl.coarse
    nd, n = c.ndim, c.n[0]
    zs, ys, xs = c.interior_slices()
    rng = np.random.default_rng(seed)
    picks = []
    for b in range(tl.n0):
        if tl.covered(b):
            continue
        bc = c.block_coords(b)
        for d in range(nd):
            for side in (0, 1):
                nbc = list(bc)
                nbc[d] += 1 if side else -1
                if not (0 <= nbc[d] < c.nb[d]):
                    continue
                nb = nbc[0] + c.nb[0] * (nbc[1] + c.nb[1] * nbc[2])
                if tl.covered(nb):
                    cell = [int(rng.integers(n)) for _ in range(3)]
                    if nd == 2:
                        cell[2] = 0
                    cell[d] = n - 1 if side else 0
                    picks.append((b, cell))
    for fb in [g for g in tl.gpu_blocks if g >= tl.n0][:3]:
        picks.append((fb, [0, 0, 0]))
    for b, (i, j, k) in picks[:6] + picks[-3:]:
        kk = zs.start + k
        cv = U[b, :, kk, ys.start + j, xs.start + i]
        ke = 0.5 * (cv[1] ** 2 + cv[2] ** 2 + cv[3] ** 2) / cv[0]
        U[b, 4, kk, ys.start + j, xs.start + i] = 0.5 * ke
    return U


@pytest.mark.parametrize("stages", [2, 3])
@pytest.mark.parametrize("name", list(TWO_LEVEL))
def test_two_level_every_entry_point_bitwise(gb, name, stages):
    tl = TWO_LEVEL[name]
    U0 = smooth_two_level(tl, 7)[tl.gpu_blocks]

    def make():
        h = gb.Hydro.from_two_level(tl)
        h.set_rk_stages(stages)
        return h
    assert on_and_off(gb, make, U0) == [0] * 6


@pytest.mark.parametrize("name", ["box-3d", "L-2d", "tripod-3d-periodic"])
def test_two_level_floor_counts_equal_with_corrected_cells(gb, name):
    """Floors planted in coarse cells that the flux correction changes: the
    carry counts the corrected value's floors, as the next stage's conversion
    would, so the counts of every entry point are those of the carry off."""
    tl = TWO_LEVEL[name]
    U = smooth_two_level(tl, 8)
    U = floor_cells(tl, U, 9)
    hits = on_and_off(gb, lambda: gb.Hydro.from_two_level(tl), U[tl.gpu_blocks], nsteps=3)
    assert all(x > 0 for x in hits), hits


def test_two_level_batched_bitwise(gb):
    tls = [wl.two_level(wl.lattice_2d(4, 4, 8, 8, 4, bc="periodic"), (1, 1), (3, 3)),
           wl.two_level(wl.lattice_3d(4, 4, 4, 8, 8, 8, 4), (1, 1, 1), (3, 3, 3))][:1] * 3
    U0 = np.concatenate([smooth_two_level(t, 10 + i)[t.gpu_blocks] for i, t in enumerate(tls)])
    on_and_off(gb, lambda: gb.Hydro.from_two_level_batch(tls), U0)


def test_telescoping_never_carries(gb):
    lat = wl.lattice_3d(2, 2, 2, 8, 8, 8, 4)
    U0 = wl.random_state(lat, seed=5, rough=True)

    def make():
        h = gb.Hydro.from_lattice(lat)
        h.set_telescoping(True)
        return h
    on_and_off(gb, make, U0)
    tl = TWO_LEVEL["box-3d"]

    def make2():
        h = gb.Hydro.from_two_level(tl)
        h.set_telescoping(True)
        return h
    on_and_off(gb, make2, smooth_two_level(tl, 11)[tl.gpu_blocks])


def test_toggle_and_default(gb):
    lat = wl.lattice_2d(2, 2, 8, 8, 4)
    h = gb.Hydro.from_lattice(lat)
    assert h.prim_carry()                       # on by default on a uniform context
    h.set_prim_carry(False)
    assert not h.prim_carry()
    h.set_prim_carry(True)
    assert h.prim_carry()
    h.close()
