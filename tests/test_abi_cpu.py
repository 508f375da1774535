"""CPU checks of the C ABI library: it builds, loads, exports every symbol the
header declares, and rejects invalid parameters before touching the GPU; plus
the host-side neighbour-table builder."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbhydro.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2401_03378_gb300 import build, _abi
    build.build()
    return _abi.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*([a-z_0-9]+)\s*\(", text, flags=re.M)))


def test_header_lists_the_abi():
    names = declared_functions()
    for required in ("hydro_fill_guardcells", "hydro_compute_dt", "hydro_step", "gbh_create"):
        assert required in names


@pytest.mark.parametrize("checked", [False, True])
def test_every_declared_symbol_is_exported(lib, checked):
    from paper_2401_03378_gb300 import _abi
    path = _abi.LIB_PATH_CHECK if checked else _abi.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in declared_functions():
        assert name in exported, name
        assert name in _abi.SIGNATURES, f"binding lacks {name}"


def test_normal_build_has_no_index_checks(lib):
    n = C.c_longlong(-1)
    assert lib.gbh_check_violations(C.byref(n)) == -5 and n.value == 0
    assert lib.gbh_check_selftest(C.byref(n)) == -5 and n.value == 0
    assert lib.gbh_check_violations(None) == -1


def _params(**over):
    from paper_2401_03378_gb300 import _abi, neighbour_table, uniform_widths
    nbr = neighbour_table(3, (2, 2, 2), (False, False, False))
    dx = uniform_widths(8, (0.1, 0.1, 0.1))
    p = _abi.GbhParams()
    p.ndim, p.nxb, p.nyb, p.nzb, p.nguard, p.nblocks = 3, 16, 16, 16, 4, 8
    p.gamma, p.cfl, p.small_rho, p.small_p = 1.4, 0.8, 1e-12, 1e-14
    for k, v in over.items():
        if k in ("nbr", "dx"):
            continue
        setattr(p, k, v)
    nbr = over.get("nbr", nbr)
    dx = over.get("dx", dx)
    keep = (np.ascontiguousarray(nbr, dtype=np.int32), np.ascontiguousarray(dx))
    p.nbr = keep[0].ctypes.data_as(C.POINTER(C.c_int32))
    p.dx = keep[1].ctypes.data_as(C.POINTER(C.c_double))
    return p, keep


@pytest.mark.parametrize("over,code", [
    (dict(ndim=4), -1),
    (dict(nguard=1), -1),
    (dict(nguard=17), -1),
    (dict(gamma=1.0), -1),
    (dict(cfl=0.0), -1),
    (dict(nblocks=0), -1),
    (dict(nzb=1), -1),
    (dict(nxb=12, nyb=12), -5),
    (dict(nxb=16, nyb=8, nguard=4), -5),
    (dict(small_rho=1e-200), -1),   # 1/sqrt(rho_L rho_R) in the HLLC flux must stay normal
])
def test_create_rejects_invalid_params_without_gpu(lib, over, code):
    p, keep = _params(**over)
    ctx = C.c_void_p()
    assert lib.gbh_create(C.byref(p), C.byref(ctx)) == code
    assert ctx.value is None
    assert lib.gbh_last_error(None)


def test_create_rejects_bad_tables_without_gpu(lib):
    from paper_2401_03378_gb300 import neighbour_table
    nbr = neighbour_table(3, (2, 2, 2), (False, False, False)).copy()
    nbr[3, 5] = 99
    p, keep = _params(nbr=nbr)
    ctx = C.c_void_p()
    assert lib.gbh_create(C.byref(p), C.byref(ctx)) == -1
    nbr = neighbour_table(3, (2, 2, 2), (False, False, False)).copy()
    nbr[2, 13] = 1
    p, keep = _params(nbr=nbr)
    assert lib.gbh_create(C.byref(p), C.byref(ctx)) == -1
    dx = np.full((8, 3), 0.1)
    dx[4, 1] = -0.1
    p, keep = _params(dx=dx)
    assert lib.gbh_create(C.byref(p), C.byref(ctx)) == -1


def test_null_context_calls_fail_cleanly(lib):
    assert lib.hydro_step(None, None, 1.0, None) == -1
    assert lib.gbh_destroy(None) == 0
    # the host-buffer entry points check the context before any CUDA call
    dt = (C.c_double * 1)(0.0)
    assert lib.hydro_step_host(None, None, dt, None) == -1
    assert lib.hydro_step_host_interior(None, None, dt, None) == -1
    assert lib.hydro_advance_host(None, None, 1, None, None) == -1
    assert lib.hydro_advance_host_interior(None, None, 1, None, None) == -1
    assert b"null context" in lib.gbh_last_error(None)


@pytest.mark.parametrize("ndim,nb,per", [
    (2, (3, 2, 1), (False, False, False)),
    (2, (4, 3, 1), (True, False, False)),
    (3, (3, 2, 2), (False, True, True)),
    (3, (1, 2, 3), (True, True, True)),
])
def test_neighbour_table_geometry(ndim, nb, per):
    """Every entry is the block whose lattice coordinates differ by the offset
    (wrapped when periodic); the table is symmetric under offset negation."""
    from paper_2401_03378_gb300 import neighbour_table
    tab = neighbour_table(ndim, nb, per)
    nbz = nb[2] if ndim == 3 else 1
    nblk = nb[0] * nb[1] * nbz
    assert tab.shape == (nblk, 27 if ndim == 3 else 9)
    offs = [(ox, oy, oz) for oz in ((-1, 0, 1) if ndim == 3 else (0,)) for oy in (-1, 0, 1) for ox in (-1, 0, 1)]
    coords = [(b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])) for b in range(nblk)]
    dims = (nb[0], nb[1], nbz)
    for b in range(nblk):
        for e, o in enumerate(offs):
            target = []
            inside = True
            for d in range(3):
                x = coords[b][d] + o[d]
                if not 0 <= x < dims[d]:
                    if per[d]:
                        x %= dims[d]
                    else:
                        inside = False
                target.append(x)
            if inside:
                assert coords[tab[b, e]] == tuple(target)
                back = offs.index(tuple(-x for x in o))
                assert tab[tab[b, e], back] == b or any(
                    dims[d] <= 2 and per[d] for d in range(3))
            else:
                assert tab[b, e] == -1


def test_two_level_tables_structure():
    from paper_2401_03378_gb300.grid import two_level_tables
    nbr, dx, parent, children = two_level_tables(3, (4, 4, 4), (8, 8, 8), (1, 1, 1), (3, 3, 3),
                                                 (False, False, False), (1 / 32, 1 / 32, 1 / 32))
    n0 = 64
    assert nbr.shape == (128, 27)
    # every covered coarse block has 8 children whose parent is it, at the right offsets
    for b in range(n0):
        ch = children[b]
        c = (b % 4, (b // 4) % 4, b // 16)
        inside = all(1 <= c[d] < 3 for d in range(3))
        assert (ch >= 0).all() == inside and ((ch < 0).all() or inside)
        for o, f in enumerate(ch if inside else []):
            assert parent[f, 0] == b
            assert tuple(parent[f, 1:]) == tuple(((o >> d) & 1) * 4 for d in range(3))
    # fine blocks: GBH_NBR_COARSER exactly where the fine lattice ends
    fine_faces = nbr[n0:][:, [12, 14, 10, 16, 4, 22]]
    assert (fine_faces == -2).sum() == 6 * 16
    assert np.all(dx[n0:] == dx[:n0][0] * 0.5)


def test_create_refined_rejects_bad_tables_without_gpu(lib):
    from paper_2401_03378_gb300 import _abi
    from paper_2401_03378_gb300.grid import two_level_tables
    nbr, dx, parent, children = two_level_tables(3, (4, 4, 4), (8, 8, 8), (1, 1, 1), (3, 3, 3),
                                                 (False, False, False), (1 / 32,) * 3)
    def attempt(nbr_, dx_, parent_, children_):
        keep = [np.ascontiguousarray(x) for x in (nbr_, dx_, parent_, children_)]
        p = _abi.GbhParams()
        p.ndim, p.nxb, p.nyb, p.nzb, p.nguard, p.nblocks = 3, 8, 8, 8, 4, keep[0].shape[0]
        p.gamma, p.cfl, p.small_rho, p.small_p = 1.4, 0.8, 1e-12, 1e-14
        p.nbr = keep[0].ctypes.data_as(C.POINTER(C.c_int32))
        p.dx = keep[1].ctypes.data_as(C.POINTER(C.c_double))
        r = _abi.GbhRefinement()
        r.parent = keep[2].ctypes.data_as(C.POINTER(C.c_int32))
        r.children = keep[3].ctypes.data_as(C.POINTER(C.c_int32))
        ctx = C.c_void_p()
        return lib.gbh_create_refined(C.byref(p), C.byref(r), C.byref(ctx))
    bad = children.copy(); bad[21, 3] = 7
    assert attempt(nbr, dx, parent, bad) == -1
    bad = parent.copy(); bad[70, 1] = 3
    assert attempt(nbr, dx, bad, children) == -1
    bad = dx.copy(); bad[90, 0] *= 1.5
    assert attempt(nbr, bad, parent, children) == -1
    bad = nbr.copy(); bad[5, 13 + 1] = -2
    assert attempt(bad, dx, parent, children) == -1
    bad = nbr.copy(); bad[64][bad[64] == -2] = -1   # a fine block claims an outflow edge
    assert attempt(bad, dx, parent, children) == -1


def test_create_batched_rejects_cross_problem_neighbours_without_gpu(lib):
    from paper_2401_03378_gb300 import _abi
    from paper_2401_03378_gb300.grid import batched_tables
    nbr, dx, prob = batched_tables([(2, (2, 2, 1), (True, True, False), (0.1, 0.1, 0.1)),
                                    (2, (3, 3, 1), (True, True, False), (0.05, 0.05, 0.1))])
    assert nbr.shape == (13, 9) and list(prob) == [0] * 4 + [1] * 9
    assert nbr[:4].max() < 4 and nbr[4:].min() >= 4
    bad = nbr.copy()
    bad[1, 5] = 7
    keep = [np.ascontiguousarray(bad), np.ascontiguousarray(dx), np.ascontiguousarray(prob)]
    p = _abi.GbhParams()
    p.ndim, p.nxb, p.nyb, p.nzb, p.nguard, p.nblocks = 2, 16, 16, 1, 4, 13
    p.gamma, p.cfl, p.small_rho, p.small_p = 1.4, 0.8, 1e-12, 1e-14
    p.nbr = keep[0].ctypes.data_as(C.POINTER(C.c_int32))
    p.dx = keep[1].ctypes.data_as(C.POINTER(C.c_double))
    ctx = C.c_void_p()
    rc = lib.gbh_create_batched(C.byref(p), keep[2].ctypes.data_as(C.POINTER(C.c_int32)), 2, C.byref(ctx))
    assert rc == -1 and b"different problems" in lib.gbh_last_error(None)


def test_batched_two_level_tables_and_checks_without_gpu(lib):
    from paper_2401_03378_gb300 import _abi
    from paper_2401_03378_gb300.grid import batched_two_level_tables, two_level_tables
    grids = [(2, (4, 4, 1), (8, 8, 1), (1, 1), (3, 3), (True, True, False), (1 / 32, 1 / 32, 1.0)),
             (2, (5, 4, 1), (8, 8, 1), (1, 1), (4, 3), (False, False, False), (1 / 40, 1 / 32, 1.0))]
    nbr, dx, parent, children, prob = batched_two_level_tables(grids)
    one = [two_level_tables(*g) for g in grids]
    n = [t[0].shape[0] for t in one]
    assert nbr.shape == (sum(n), 9) and list(prob) == [0] * n[0] + [1] * n[1]
    # the second grid's tables, shifted by the first grid's block count
    nb2, dx2, par2, ch2 = one[1]
    assert np.array_equal(nbr[n[0]:], np.where(nb2 >= 0, nb2 + n[0], nb2))
    assert np.array_equal(dx[n[0]:], dx2)
    assert np.array_equal(parent[n[0]:, 0], np.where(par2[:, 0] >= 0, par2[:, 0] + n[0], -1))
    assert np.array_equal(parent[n[0]:, 1:], par2[:, 1:])
    assert np.array_equal(children[n[0]:], np.where(ch2 >= 0, ch2 + n[0], -1))
    assert np.array_equal(nbr[:n[0]], one[0][0]) and np.array_equal(children[:n[0]], one[0][3])

    def attempt(prob_, parent_=parent, nproblems=2):
        keep = [np.ascontiguousarray(x) for x in (nbr, dx, parent_, children, prob_)]
        p = _abi.GbhParams()
        p.ndim, p.nxb, p.nyb, p.nzb, p.nguard, p.nblocks = 2, 8, 8, 1, 4, keep[0].shape[0]
        p.gamma, p.cfl, p.small_rho, p.small_p = 1.4, 0.8, 1e-12, 1e-14
        p.nbr = keep[0].ctypes.data_as(C.POINTER(C.c_int32))
        p.dx = keep[1].ctypes.data_as(C.POINTER(C.c_double))
        r = _abi.GbhRefinement()
        r.parent = keep[2].ctypes.data_as(C.POINTER(C.c_int32))
        r.children = keep[3].ctypes.data_as(C.POINTER(C.c_int32))
        ctx = C.c_void_p()
        return lib.gbh_create_refined_batched(C.byref(p), C.byref(r), keep[4].ctypes.data_as(C.POINTER(C.c_int32)),
                                              nproblems, C.byref(ctx))
    # a fine block of grid 0 whose own same-level neighbours stay in problem 0 but
    # whose parent is then in another problem: move its whole fine lattice
    bad = prob.copy()
    f0 = 16
    bad[f0:n[0]] = 1
    assert attempt(bad) == -1 and b"different problems" in lib.gbh_last_error(None)
    bad = prob.copy(); bad[3] = 2
    assert attempt(bad) == -1 and b"out of range" in lib.gbh_last_error(None)
    assert attempt(prob, nproblems=0) == -1


def refined_tables(ndim, nb0, n, refined, dx0):
    """Two-level tables for any set of refined coarse blocks (coarse lattice
    coordinates), non-periodic: fine blocks in lexicographic order of the fine
    lattice, GBH_NBR_COARSER where a fine block's neighbour lies on the coarse
    level.  For a box this is two_level_tables' layout."""
    from paper_2401_03378_gb300.grid import GBH_BC_OUTFLOW, GBH_NBR_COARSER, neighbour_table
    nd = ndim
    nb0 = tuple(nb0) + (1,) * (3 - len(nb0))
    ref = {tuple(c) + (0,) * (3 - len(c)) for c in refined}
    n0 = nb0[0] * nb0[1] * nb0[2]
    fdim = tuple(2 * nb0[d] if d < nd else 1 for d in range(3))
    fine = [(fx, fy, fz) for fz in range(fdim[2]) for fy in range(fdim[1]) for fx in range(fdim[0])
            if tuple(c // 2 if d < nd else 0 for d, c in enumerate((fx, fy, fz))) in ref]
    fid = {fc: n0 + i for i, fc in enumerate(fine)}
    offs = [(ox, oy, oz) for oz in ((-1, 0, 1) if nd == 3 else (0,)) for oy in (-1, 0, 1) for ox in (-1, 0, 1)]
    nbr = np.concatenate([neighbour_table(nd, nb0, (False,) * 3),
                          np.empty((len(fine), len(offs)), dtype=np.int32)])
    parent = np.zeros((n0 + len(fine), 4), dtype=np.int32)
    parent[:n0, 0] = -1
    children = np.full((n0 + len(fine), 8), -1, dtype=np.int32)
    for i, fc in enumerate(fine):
        for e, o in enumerate(offs):
            q = tuple(fc[d] + o[d] for d in range(3))
            inside = all(0 <= q[d] < fdim[d] for d in range(3))
            nbr[n0 + i, e] = fid.get(q, GBH_NBR_COARSER if inside else GBH_BC_OUTFLOW)
        pc = tuple(fc[d] // 2 if d < nd else 0 for d in range(3))
        pid = pc[0] + nb0[0] * (pc[1] + nb0[1] * pc[2])
        parent[n0 + i] = (pid, *((fc[d] % 2) * (n[d] // 2) if d < nd else 0 for d in range(3)))
        children[pid, sum((fc[d] % 2) << d for d in range(nd))] = n0 + i
    dx = np.empty((n0 + len(fine), 3))
    dx[:n0] = dx0
    dx[n0:] = np.asarray(dx0) * 0.5
    return nbr, dx, parent, children


def test_create_refined_takes_any_region_without_gpu(lib):
    """The tables of any set of refined coarse blocks (a box, an L whose inner
    coarse block borders the fine region through two faces, a notch with three,
    two boxes one coarse block apart) built by two_level_tables equal this
    test's own construction, and they pass the context's table checks: without
    a GPU the context allocation then fails, not the tables."""
    from paper_2401_03378_gb300 import _abi
    from paper_2401_03378_gb300.grid import two_level_tables

    def attempt(tables):
        keep = [np.ascontiguousarray(x) for x in tables]
        p = _abi.GbhParams()
        p.ndim, p.nxb, p.nyb, p.nzb, p.nguard, p.nblocks = 2, 8, 8, 1, 4, keep[0].shape[0]
        p.gamma, p.cfl, p.small_rho, p.small_p = 1.4, 0.8, 1e-12, 1e-14
        p.nbr = keep[0].ctypes.data_as(C.POINTER(C.c_int32))
        p.dx = keep[1].ctypes.data_as(C.POINTER(C.c_double))
        r = _abi.GbhRefinement()
        r.parent = keep[2].ctypes.data_as(C.POINTER(C.c_int32))
        r.children = keep[3].ctypes.data_as(C.POINTER(C.c_int32))
        ctx = C.c_void_p()
        rc = lib.gbh_create_refined(C.byref(p), C.byref(r), C.byref(ctx))
        if rc == 0:
            lib.gbh_destroy(ctx)
        return rc, lib.gbh_last_error(None)

    regions = [((4, 4), [(x, y) for y in (1, 2) for x in (1, 2)]),            # box
               ((4, 4), [(1, 1), (2, 1), (1, 2)]),                          # L
               ((5, 4), [(1, 1), (2, 1), (3, 1), (1, 2), (3, 2)]),          # notch
               ((5, 4), [(1, 1), (1, 2), (3, 1), (3, 2)]),                  # two boxes, one block apart
               ((5, 5), [(1, 1), (3, 3)])]                                  # separate blocks
    for nb0, blocks in regions:
        dx0 = (1 / (8 * nb0[0]), 1 / (8 * nb0[1]), 1.0)
        mine = refined_tables(2, nb0, (8, 8), blocks, dx0)
        lo = (min(b[0] for b in blocks), min(b[1] for b in blocks))
        hi = (max(b[0] for b in blocks) + 1, max(b[1] for b in blocks) + 1)
        ref = two_level_tables(2, nb0 + (1,), (8, 8, 1), lo, hi, (False, False, False), dx0, blocks)
        for x, y in zip(mine, ref):
            assert np.array_equal(x, y)
        rc, msg = attempt(mine)
        assert rc in (0, -2, -4) and b"faces" not in msg, msg


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: loading a library that is not there raises, and a
    context cannot be created without a CUDA device (the error names CUDA)."""
    from paper_2401_03378_gb300 import _abi
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _abi.load(str(tmp_path / "libgbhydro.so"))


def test_hydro_binding_without_a_device_raises(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2401_03378_gb300 import Hydro, _abi
    with pytest.raises(_abi.GbhError):
        Hydro(3, (8, 8, 8), 4, nb=(2, 2, 2))
