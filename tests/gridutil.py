"""Test helpers: move between the block layout and one global array."""
import numpy as np


def to_global(U, lat):
    """Interior cells of every block -> (5, NZ, NY, NX) global array."""
    NX, NY, NZ = lat.global_cells
    out = np.empty((5, NZ, NY, NX))
    zs, ys, xs = lat.interior_slices()
    nx, ny, nz = lat.n
    for b in range(lat.nblocks):
        bi, bj, bk = lat.block_coords(b)
        out[:, bk * nz:(bk + 1) * nz, bj * ny:(bj + 1) * ny, bi * nx:(bi + 1) * nx] = U[b][:, zs, ys, xs]
    return out


def from_global(Gl, lat, guard_value=0.0):
    """(5, NZ, NY, NX) global array -> block layout with guards set to guard_value."""
    U = np.full(lat.shape, guard_value)
    zs, ys, xs = lat.interior_slices()
    nx, ny, nz = lat.n
    for b in range(lat.nblocks):
        bi, bj, bk = lat.block_coords(b)
        U[b][:, zs, ys, xs] = Gl[:, bk * nz:(bk + 1) * nz, bj * ny:(bj + 1) * ny, bi * nx:(bi + 1) * nx]
    return np.ascontiguousarray(U)


def padded_global(Gl, lat):
    """Global array padded by the guard width: 'edge' for outflow, 'wrap' for periodic,
    applied axis by axis in the order x, y, z."""
    P = Gl
    g = lat.ng
    for d, ax in ((0, 3), (1, 2), (2, 1)):
        if d >= lat.ndim:
            continue
        pad = [(0, 0)] * 4
        pad[ax] = (g, g)
        P = np.pad(P, pad, mode="wrap" if lat.bc[d] == "periodic" else "edge")
    return P


def relerr_per_var(A, B):
    """max|A-B| / max|B| per conserved variable (exact zero required where max|B| = 0)."""
    out = []
    for v in range(5):
        m = np.max(np.abs(B[v]))
        d = np.max(np.abs(A[v] - B[v]))
        out.append(d / m if m > 0 else (0.0 if d == 0 else np.inf))
    return np.array(out)
