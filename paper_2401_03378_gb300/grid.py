"""Host-side description of a uniform block lattice -> the C ABI's tables.

Sec. 2.2 of the paper: the domain is divided into blocks with identical cell
counts, each with a halo of guard cells.  The library takes the block
adjacency as an explicit table; this module builds it for a rectangular
lattice of blocks numbered lexicographically (x fastest) with outflow or
periodic domain boundaries.
"""
from __future__ import annotations

import numpy as np

GBH_BC_OUTFLOW = -1
GBH_NBR_COARSER = -2


def neighbour_table(ndim: int, nb, periodic) -> np.ndarray:
    """int32 [nblocks][3^ndim]: entry (oz+1)*9 + (oy+1)*3 + (ox+1) (2-D: (oy+1)*3 + (ox+1))
    holds the block at lattice offset (ox, oy, oz), wrapped across periodic
    boundaries, or GBH_BC_OUTFLOW outside a non-periodic one."""
    nbx, nby, nbz = (int(nb[0]), int(nb[1]), int(nb[2]) if ndim == 3 else 1)
    per = [bool(periodic[d]) for d in range(3)]
    nblk = nbx * nby * nbz
    offs = [(ox, oy, oz) for oz in ((-1, 0, 1) if ndim == 3 else (0,))
            for oy in (-1, 0, 1) for ox in (-1, 0, 1)]
    tab = np.empty((nblk, len(offs)), dtype=np.int32)
    dims = (nbx, nby, nbz)
    for b in range(nblk):
        c = (b % nbx, (b // nbx) % nby, b // (nbx * nby))
        for e, o in enumerate(offs):
            q = []
            ok = True
            for d in range(3):
                x = c[d] + o[d]
                if x < 0 or x >= dims[d]:
                    if not per[d]:
                        ok = False
                        break
                    x %= dims[d]
                q.append(x)
            tab[b, e] = q[0] + nbx * (q[1] + nby * q[2]) if ok else GBH_BC_OUTFLOW
    return tab


def uniform_widths(nblocks: int, dx) -> np.ndarray:
    w = np.empty((nblocks, 3), dtype=np.float64)
    w[:] = np.asarray(dx, dtype=np.float64)
    return w


def two_level_tables(ndim: int, nb0, n, lo, hi, periodic, dx0, refined=None):
    """Tables of a two-level composite grid: the complete coarse lattice nb0
    (blocks 0..n0-1) plus a fine level at half the cell width over refined
    coarse blocks: every block of [lo, hi), or, if `refined` lists coarse block
    coordinates, those blocks ([lo, hi) is then their bounding box).  The fine
    blocks (n0..) are the children of the refined blocks, numbered in the order
    of the fine lattice over [lo, hi) (x fastest), the children of blocks that
    are not refined left out.  A fine face or edge with no fine block beyond it
    faces the coarser level (GBH_NBR_COARSER).

    Returns (nbr, dx, parent, children) in the layout gbh_create_refined takes.
    """
    nd = int(ndim)
    nb0 = tuple(int(x) for x in nb0) + (1,) * (3 - len(nb0))
    lo = tuple(int(x) for x in lo) + (0,) * (3 - len(lo))
    hi = tuple(int(x) for x in hi) + (1,) * (3 - len(hi))
    n = tuple(int(x) for x in n) + (1,) * (3 - len(n))
    nb1 = tuple(2 * (hi[d] - lo[d]) if d < nd else 1 for d in range(3))
    n0 = nb0[0] * nb0[1] * nb0[2]
    nlat = nb1[0] * nb1[1] * nb1[2]
    ref = None if refined is None else {tuple(int(x) for x in c) + (0,) * (3 - len(c)) for c in refined}

    def fine_coords(f):
        return (f % nb1[0], (f // nb1[0]) % nb1[1], f // (nb1[0] * nb1[1]))

    def parent_coords(f):
        fc = fine_coords(f)
        return tuple(lo[d] + fc[d] // 2 if d < nd else 0 for d in range(3))

    exists = np.array([ref is None or parent_coords(f) in ref for f in range(nlat)], dtype=bool)
    rank = np.full(nlat, -1, dtype=np.int64)
    rank[exists] = np.arange(int(exists.sum()))
    n1 = int(exists.sum())
    cnbr = neighbour_table(nd, nb0, periodic)
    lat = neighbour_table(nd, nb1, (False, False, False)).astype(np.int64)[exists]
    safe = np.where(lat >= 0, lat, 0)
    fnbr = np.where((lat >= 0) & exists[safe], n0 + rank[safe], GBH_NBR_COARSER).astype(np.int32)
    nbr = np.concatenate([cnbr, fnbr], axis=0)
    dx = np.empty((n0 + n1, 3))
    dx[:n0] = np.asarray(dx0, dtype=np.float64)
    dx[n0:] = np.asarray(dx0, dtype=np.float64) * 0.5
    parent = np.zeros((n0 + n1, 4), dtype=np.int32)
    parent[:n0, 0] = -1
    children = np.full((n0 + n1, 8), -1, dtype=np.int32)
    for f in np.flatnonzero(exists):
        fc = fine_coords(f)
        pc = parent_coords(f)
        pid = pc[0] + nb0[0] * (pc[1] + nb0[1] * pc[2])
        off = tuple((fc[d] % 2) * (n[d] // 2) if d < nd else 0 for d in range(3))
        parent[n0 + rank[f]] = (pid, *off)
        oct_ = sum((fc[d] % 2) << d for d in range(nd))
        children[pid, oct_] = n0 + rank[f]
    return nbr, dx, parent, children


def batched_two_level_tables(grids):
    """Tables of independent two-level composite grids in one state array.

    grids: sequence of (ndim, nb0, n, lo, hi, periodic, dx0[, refined]), the
    arguments of two_level_tables (same block shape).  The blocks of grid i (its coarse
    blocks, then its fine blocks) follow those of grid i-1.  Returns
    (nbr, dx, parent, children, problem) for gbh_create_refined_batched.
    """
    nbrs, dxs, pars, chls, ids = [], [], [], [], []
    off = 0
    for i, g in enumerate(grids):
        nbr, dx, parent, children = two_level_tables(*g)
        nbr = nbr.astype(np.int64)
        nbrs.append(np.where(nbr >= 0, nbr + off, nbr).astype(np.int32))
        dxs.append(dx)
        parent = parent.astype(np.int64)
        parent[:, 0] = np.where(parent[:, 0] >= 0, parent[:, 0] + off, parent[:, 0])
        pars.append(parent.astype(np.int32))
        children = children.astype(np.int64)
        chls.append(np.where(children >= 0, children + off, children).astype(np.int32))
        ids.append(np.full(nbr.shape[0], i, dtype=np.int32))
        off += nbr.shape[0]
    return (np.concatenate(nbrs), np.concatenate(dxs), np.concatenate(pars), np.concatenate(chls),
            np.concatenate(ids))


def batched_tables(problems):
    """Tables of independent problems in one state array.

    problems: sequence of (ndim, nb, periodic, dx) uniform lattices (same block
    shape).  Blocks of problem i follow those of problem i-1.  Returns
    (nbr, dx, problem) for gbh_create_batched.
    """
    nbrs, dxs, ids = [], [], []
    off = 0
    for i, (ndim, nb, periodic, dx) in enumerate(problems):
        t = neighbour_table(ndim, nb, periodic).astype(np.int64)
        t = np.where(t >= 0, t + off, t).astype(np.int32)
        nbrs.append(t)
        dxs.append(uniform_widths(t.shape[0], dx))
        ids.append(np.full(t.shape[0], i, dtype=np.int32))
        off += t.shape[0]
    return np.concatenate(nbrs), np.concatenate(dxs), np.concatenate(ids)
