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
