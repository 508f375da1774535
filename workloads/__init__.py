"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *describes* problems: the block lattice (sizes, spacing,
boundary kinds, block numbering) and initial conditions given as primitive
states (rho, u, v, w, p) turned into conserved arrays.  It contains none of the
hydrodynamics method (no reconstruction, no Riemann solver, no update, no
time-step rule), and it imports neither the product package nor ``oracle/``.

Block storage layout (the layout both sides consume):
    U[nblocks][5][nz + 2*gz][ny + 2*g][nx + 2*g]   float64, x fastest
with variables (rho, rho*u, rho*v, rho*w, E); gz = g in 3-D and 0 in 2-D.
Block ids are lexicographic over the lattice, x fastest:
    b = bi + nbx * (bj + nby * bk).
The domain is the unit square / cube; cell widths are 1/(nb_d * n_d).

The problems follow the workloads of the block-structured hydrodynamics runs
the paper generates code for (Sec. 4.2: equal-size blocks with a halo of
guard cells, Sec. 2.2): a 2-D Sod shock tube, a 3-D Sedov blast, periodic
Sod / Kelvin-Helmholtz ensembles with log-normal density noise, and random
valid states for brute-force checks.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

OUTFLOW = "outflow"
PERIODIC = "periodic"


@dataclass(frozen=True)
class Lattice:
    """A uniform lattice of equal blocks covering [0,1]^ndim."""

    ndim: int
    nb: Tuple[int, int, int]          # blocks per dimension (nb[2] == 1 in 2-D)
    n: Tuple[int, int, int]           # interior cells per block (n[2] == 1 in 2-D)
    ng: int = 4                       # guard cells per side (x, y; z too in 3-D)
    bc: Tuple[str, str, str] = (OUTFLOW, OUTFLOW, OUTFLOW)
    extent: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)

    def __post_init__(self):
        if self.ndim not in (2, 3):
            raise ValueError("ndim must be 2 or 3")
        if self.ndim == 2 and (self.nb[2] != 1 or self.n[2] != 1):
            raise ValueError("2-D lattices have nb[2] == n[2] == 1")
        for b in self.bc:
            if b not in (OUTFLOW, PERIODIC):
                raise ValueError(f"unknown boundary kind {b!r}")

    @property
    def gz(self) -> int:
        return self.ng if self.ndim == 3 else 0

    @property
    def nblocks(self) -> int:
        return self.nb[0] * self.nb[1] * self.nb[2]

    @property
    def padded(self) -> Tuple[int, int, int]:
        """(nz_pad, ny_pad, nx_pad)."""
        return (self.n[2] + 2 * self.gz, self.n[1] + 2 * self.ng, self.n[0] + 2 * self.ng)

    @property
    def shape(self) -> Tuple[int, int, int, int, int]:
        return (self.nblocks, 5) + self.padded

    @property
    def global_cells(self) -> Tuple[int, int, int]:
        return tuple(self.nb[d] * self.n[d] for d in range(3))

    @property
    def dx(self) -> Tuple[float, float, float]:
        return tuple(self.extent[d] / (self.nb[d] * self.n[d]) for d in range(3))

    @property
    def interior_cells(self) -> int:
        g = self.global_cells
        return g[0] * g[1] * g[2]

    def block_coords(self, b: int) -> Tuple[int, int, int]:
        bi = b % self.nb[0]
        bj = (b // self.nb[0]) % self.nb[1]
        bk = b // (self.nb[0] * self.nb[1])
        return bi, bj, bk

    def interior_slices(self):
        """Index of the interior cells inside a padded block (z, y, x)."""
        gz, g = self.gz, self.ng
        return (slice(gz, gz + self.n[2]), slice(g, g + self.n[1]), slice(g, g + self.n[0]))


def lattice_2d(nbx, nby, nxb=16, nyb=16, ng=4, bc=OUTFLOW) -> Lattice:
    bcs = (bc, bc, OUTFLOW) if isinstance(bc, str) else tuple(bc) + (OUTFLOW,)
    return Lattice(2, (nbx, nby, 1), (nxb, nyb, 1), ng, bcs)


def lattice_3d(nbx, nby, nbz, nxb=16, nyb=16, nzb=16, ng=4, bc=OUTFLOW) -> Lattice:
    bcs = (bc, bc, bc) if isinstance(bc, str) else tuple(bc)
    return Lattice(3, (nbx, nby, nbz), (nxb, nyb, nzb), ng, bcs)


def cell_centers(lat: Lattice):
    """Cell-centre coordinates X, Y, Z of every padded cell, shape (nblk, nz, ny, nx)."""
    nzp, nyp, nxp = lat.padded
    dx = lat.dx
    X = np.empty((lat.nblocks, nzp, nyp, nxp))
    Y = np.empty_like(X)
    Z = np.empty_like(X)
    ii = np.arange(nxp) - lat.ng
    jj = np.arange(nyp) - lat.ng
    kk = np.arange(nzp) - lat.gz
    for b in range(lat.nblocks):
        bi, bj, bk = lat.block_coords(b)
        x = lat.origin[0] + (bi * lat.n[0] + ii + 0.5) * dx[0]
        y = lat.origin[1] + (bj * lat.n[1] + jj + 0.5) * dx[1]
        z = (lat.origin[2] + (bk * lat.n[2] + kk + 0.5) * dx[2]) if lat.ndim == 3 else np.full(nzp, 0.5 * dx[2])
        Z[b], Y[b], X[b] = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def conserved(rho, u, v, w, p, gamma):
    """Conserved (rho, rho u, rho v, rho w, E) of a primitive ideal-gas state.

    This is the definition of the initial data (total energy of the stated
    state), not part of the method being tested.
    """
    rho = np.asarray(rho, dtype=np.float64)
    U = np.empty((5,) + rho.shape)
    U[0] = rho
    U[1] = rho * u
    U[2] = rho * v
    U[3] = rho * w
    U[4] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return U


def _assemble(lat: Lattice, rho, u, v, w, p, gamma):
    U = conserved(rho, u, v, w, p, gamma)          # (5, nblk, nz, ny, nx)
    return np.ascontiguousarray(np.moveaxis(U, 0, 1))


# ----------------------------------------------------------------------------
# Initial conditions
# ----------------------------------------------------------------------------

SOD_LEFT = (1.0, 0.0, 1.0)      # (rho, u, p) for x < 1/2
SOD_RIGHT = (0.125, 0.0, 0.1)


def sod(lat: Lattice, gamma: float = 1.4, x0: float = 0.5, axis: int = 0):
    """Sod shock tube along ``axis``: (rho,p) = (1,1) left of x0, (0.125,0.1) right."""
    X, Y, Z = cell_centers(lat)
    s = (X, Y, Z)[axis]
    left = s < x0
    rho = np.where(left, SOD_LEFT[0], SOD_RIGHT[0])
    p = np.where(left, SOD_LEFT[2], SOD_RIGHT[2])
    zero = np.zeros_like(rho)
    return _assemble(lat, rho, zero, zero, zero, p, gamma)


def sedov_cells(lat: Lattice, r_cells: float = 3.5):
    """Mask of the cells whose centres lie within r_cells cell widths of the centre."""
    X, Y, Z = cell_centers(lat)
    dx = lat.dx[0]
    c = [lat.origin[d] + 0.5 * lat.extent[d] for d in range(3)]
    r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2
    if lat.ndim == 3:
        r2 = r2 + (Z - c[2]) ** 2
    mask = r2 <= (r_cells * dx) ** 2
    # only interior cells carry the deposit
    inner = np.zeros_like(mask)
    zs, ys, xs = lat.interior_slices()
    inner[:, zs, ys, xs] = True
    return mask & inner


def sedov(lat: Lattice, gamma: float = 1.4, energy: float = 1.0, r_cells: float = 3.5,
          p_ambient: float = 1e-5, rho_ambient: float = 1.0):
    """Sedov blast: energy deposited as uniform pressure in the cells within r_cells.

    The deposit pressure is p = (gamma-1) * energy / (n_dep * cell_volume), so the
    deposited internal energy equals ``energy`` exactly; elsewhere p = p_ambient.
    """
    mask = sedov_cells(lat, r_cells)
    ndep = int(mask.sum())
    vol = float(np.prod(lat.dx[: lat.ndim]))
    p_dep = (gamma - 1.0) * energy / (ndep * vol)
    rho = np.full(mask.shape, rho_ambient)
    p = np.where(mask, p_dep, p_ambient)
    zero = np.zeros_like(rho)
    return _assemble(lat, rho, zero, zero, zero, p, gamma)


def kelvin_helmholtz(lat: Lattice, gamma: float = 1.4, seed: int = 0, sigma: float = 0.1):
    """2-D Kelvin-Helmholtz shear layer with log-normal density noise (periodic)."""
    X, Y, _ = cell_centers(lat)
    rng = np.random.Generator(np.random.PCG64(seed))
    inner = np.abs(Y - 0.5) < 0.25
    rho = np.where(inner, 2.0, 1.0)
    u = np.where(inner, 0.5, -0.5)
    v = 0.01 * np.sin(4.0 * np.pi * X)
    p = np.full(rho.shape, 2.5)
    rho = rho * np.exp(sigma * rng.standard_normal(rho.shape))
    return _assemble(lat, rho, u, v, np.zeros_like(rho), p, gamma)


def sod_periodic(lat: Lattice, gamma: float = 1.4, seed: int = 0, sigma: float = 0.1):
    """Sod layout on a periodic domain (two interfaces) with log-normal density noise."""
    X, _, _ = cell_centers(lat)
    rng = np.random.Generator(np.random.PCG64(seed))
    left = X < 0.5
    rho = np.where(left, SOD_LEFT[0], SOD_RIGHT[0]) * np.exp(sigma * rng.standard_normal(X.shape))
    p = np.where(left, SOD_LEFT[2], SOD_RIGHT[2])
    zero = np.zeros_like(rho)
    return _assemble(lat, rho, zero, zero, zero, p, gamma)


def random_state(lat: Lattice, seed: int, gamma: float = 1.4, rough: bool = True,
                 mach: float = 0.8):
    """Random valid state: positive density/pressure, velocities up to ~mach.

    rough=True draws independent values per cell (discontinuous everywhere);
    rough=False draws a few random Fourier modes (smooth).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (lat.nblocks,) + lat.padded
    if rough:
        rho = rng.uniform(0.5, 2.0, shape)
        p = rng.uniform(0.5, 2.0, shape)
        vel = rng.uniform(-mach, mach, (3,) + shape)
    else:
        X, Y, Z = cell_centers(lat)
        def field(lo, hi):
            f = np.zeros(shape)
            for _ in range(3):
                kx, ky, kz = rng.integers(1, 4, 3)
                ph = rng.uniform(0, 2 * np.pi)
                f += np.sin(2 * np.pi * (kx * X + ky * Y + (kz * Z if lat.ndim == 3 else 0)) + ph)
            return lo + (hi - lo) * (f / 6.0 + 0.5)
        rho = field(0.5, 2.0)
        p = field(0.5, 2.0)
        vel = np.stack([field(-mach, mach) for _ in range(3)])
    if lat.ndim == 2:
        vel[2] = 0.0
    return _assemble(lat, rho, vel[0], vel[1], vel[2], p, gamma)


def poison_guards(U: np.ndarray, lat: Lattice, value: float = np.nan, corners_only: bool = False):
    """Overwrite guard cells (all, or only edge/corner regions) with ``value``."""
    U = U.copy()
    nzp, nyp, nxp = lat.padded
    g, gz = lat.ng, lat.gz
    k = np.arange(nzp)
    j = np.arange(nyp)
    i = np.arange(nxp)
    ox = (i < g).astype(int) + (i >= g + lat.n[0]).astype(int)
    oy = (j < g).astype(int) + (j >= g + lat.n[1]).astype(int)
    oz = ((k < gz).astype(int) + (k >= gz + lat.n[2]).astype(int)) if lat.ndim == 3 else np.zeros(nzp, int)
    nout = oz[:, None, None] + oy[None, :, None] + ox[None, None, :]
    sel = nout >= 2 if corners_only else nout >= 1
    U[:, :, sel] = value
    return U


# ----------------------------------------------------------------------------
# Two-level composite grids (refinement ratio 2)
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class TwoLevel:
    """A complete coarse lattice plus a fine level at twice the resolution over
    a set of whole coarse blocks, each at least one block from the domain edge:
    the box [lo, hi) of coarse blocks, or, when `refined` lists coarse block
    coordinates, those blocks (an L shape, separate boxes, ...), of which
    [lo, hi) is then the bounding box.

    Composite arrays hold the coarse blocks first, then the fine lattice over
    [lo, hi) block by block; fine blocks whose parent is not refined have slots
    there too (the oracle's layout), and `gpu_blocks` lists the blocks of the
    library's layout, which has no such slots."""

    coarse: Lattice
    lo: Tuple[int, int, int]
    hi: Tuple[int, int, int]
    refined: Optional[Tuple[Tuple[int, int, int], ...]] = None

    def __post_init__(self):
        for d in range(self.coarse.ndim):
            if not (1 <= self.lo[d] < self.hi[d] <= self.coarse.nb[d] - 1):
                raise ValueError("the fine region must be made of coarse blocks away from the domain edge")
        if self.refined is not None:
            for c in self.refined:
                if not all(self.lo[d] <= c[d] < self.hi[d] for d in range(3)):
                    raise ValueError("refined blocks must lie in [lo, hi)")

    @property
    def fine(self) -> Lattice:
        c = self.coarse
        nd = c.ndim
        dx = c.dx
        nb = tuple(2 * (self.hi[d] - self.lo[d]) if d < nd else 1 for d in range(3))
        origin = tuple(self.lo[d] * c.n[d] * dx[d] if d < nd else 0.0 for d in range(3))
        extent = tuple((self.hi[d] - self.lo[d]) * c.n[d] * dx[d] if d < nd else c.extent[d] for d in range(3))
        return Lattice(nd, nb, c.n, c.ng, (OUTFLOW, OUTFLOW, OUTFLOW), extent, origin)

    @property
    def n0(self) -> int:
        return self.coarse.nblocks

    @property
    def n1(self) -> int:
        return self.fine.nblocks

    @property
    def nblocks(self) -> int:
        return self.n0 + self.n1

    @property
    def shape(self):
        return (self.nblocks, 5) + self.coarse.padded

    def covered(self, b: int) -> bool:
        c = self.coarse.block_coords(b)
        if not all(self.lo[d] <= c[d] < self.hi[d] for d in range(3)):
            return False
        return self.refined is None or tuple(c) in self.refined

    def refined_mask(self) -> np.ndarray:
        """uint8 [n0]: 1 for every refined (covered) coarse block."""
        return np.array([1 if self.covered(b) else 0 for b in range(self.n0)], dtype=np.uint8)

    def fine_exists(self, f: int) -> bool:
        """Fine lattice block f exists: its parent coarse block is refined."""
        c = self.fine.block_coords(f)
        nd = self.coarse.ndim
        p = tuple(self.lo[d] + c[d] // 2 if d < nd else 0 for d in range(3))
        return self.covered(p[0] + self.coarse.nb[0] * (p[1] + self.coarse.nb[1] * p[2]))

    @property
    def gpu_blocks(self) -> np.ndarray:
        """Composite-array indices of the library's blocks: every coarse block,
        then the fine blocks that exist, in fine-lattice order."""
        fine = [self.n0 + f for f in range(self.n1) if self.fine_exists(f)]
        return np.array(list(range(self.n0)) + fine, dtype=np.int64)

    @property
    def leaf_cells(self) -> int:
        c = self.coarse
        per = c.n[0] * c.n[1] * c.n[2]
        ncov = sum(1 for b in range(self.n0) if self.covered(b))
        nfine = sum(1 for f in range(self.n1) if self.fine_exists(f))
        return (self.n0 - ncov + nfine) * per


def two_level(coarse: Lattice, lo, hi) -> TwoLevel:
    lo = tuple(lo) + (0,) * (3 - len(lo))
    hi = tuple(hi) + (1,) * (3 - len(hi))
    return TwoLevel(coarse, lo, hi)


def two_level_blocks(coarse: Lattice, blocks) -> TwoLevel:
    """Two-level grid refining the listed coarse blocks (coordinates (i, j[, k]))."""
    cs = sorted({tuple(b) + (0,) * (3 - len(b)) for b in blocks})
    lo = tuple(min(c[d] for c in cs) for d in range(3))
    hi = tuple(max(c[d] for c in cs) + 1 for d in range(3))
    return TwoLevel(coarse, lo, hi, tuple(cs))


def two_level_state(tl: TwoLevel, prim_fn, gamma: float = 1.4):
    """Composite conserved array from a primitive-state function of (X, Y, Z)."""
    parts = []
    for lat in (tl.coarse, tl.fine):
        X, Y, Z = cell_centers(lat)
        rho, u, v, w, p = prim_fn(X, Y, Z)
        parts.append(_assemble(lat, rho, u, v, w, p, gamma))
    return np.ascontiguousarray(np.concatenate(parts, axis=0))


def sedov_two_level(tl: TwoLevel, gamma: float = 1.4, energy: float = 1.0, r_cells: float = 3.5,
                    p_ambient: float = 1e-5):
    """Sedov blast on a composite grid: the energy sits in the fine cells within
    r_cells FINE cell widths of the centre (which the fine region must contain);
    every other cell is ambient (covered coarse cells are restricted by the solver)."""
    fine = tl.fine
    mask = sedov_cells(fine, r_cells)
    ndep = int(mask.sum())
    vol = float(np.prod(fine.dx[: fine.ndim]))
    p_dep = (gamma - 1.0) * energy / (ndep * vol)
    shape_c = (tl.coarse.nblocks,) + tl.coarse.padded
    zc = np.zeros(shape_c)
    Uc = _assemble(tl.coarse, np.ones(shape_c), zc, zc, zc, np.full(shape_c, p_ambient), gamma)
    rho = np.ones(mask.shape)
    p = np.where(mask, p_dep, p_ambient)
    zero = np.zeros_like(rho)
    Uf = _assemble(fine, rho, zero, zero, zero, p, gamma)
    return np.ascontiguousarray(np.concatenate([Uc, Uf], axis=0))


def sod_smooth(lat: Lattice, gamma: float = 1.4, width_cells: float = 2.0, amp: float = 0.05,
               primitive: bool = False):
    """Sod-like 2-D data for gradient checks: the Sod jump at x = 1/2 smoothed by
    tanh over `width_cells` cells, with smooth 2-D modulations of every field
    (amplitude `amp`) so that no field is locally constant (the MC limiter is
    not differentiable where both one-sided differences vanish).  Returns the
    conserved array, or with primitive=True the (rho, u, v, w, p) array in the
    same layout."""
    X, Y, _ = cell_centers(lat)
    dx = lat.dx[0]
    s = 0.5 * (1.0 - np.tanh((X - 0.5) / (width_cells * dx)))      # 1 left, 0 right
    mod = 1.0 + amp * np.sin(2 * np.pi * X + 0.3) * np.sin(2 * np.pi * Y + 0.7)
    rho = (SOD_RIGHT[0] + (SOD_LEFT[0] - SOD_RIGHT[0]) * s) * mod
    p = (SOD_RIGHT[2] + (SOD_LEFT[2] - SOD_RIGHT[2]) * s) * (2.0 - mod)
    u = amp * np.sin(2 * np.pi * Y + 0.2) * np.cos(np.pi * X + 0.1)
    v = amp * np.cos(2 * np.pi * X + 0.4) * np.sin(2 * np.pi * Y + 0.9)
    zero = np.zeros_like(rho)
    if primitive:
        return np.ascontiguousarray(np.stack([rho, u, v, zero, p], axis=1))
    return _assemble(lat, rho, u, v, zero, p, gamma)


def ensemble_sizes(count: int = 96, seed: int = 0, choices=(64, 128, 256, 512)):
    """Problem sizes for the batched-ensemble workload (uniform draw, seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(choices[i]) for i in rng.integers(0, len(choices), count)]


def ensemble(count: int = 96, seed: int = 0, nxb: int = 16, ng: int = 4, choices=(64, 128, 256, 512)):
    """Batched-ensemble workload: `count` independent periodic 2-D problems of
    sizes drawn from `choices` (seed `seed`) in nxb^2 blocks; problem i starts
    from the periodic Sod layout (i even) or the Kelvin-Helmholtz layer (i odd),
    each with log-normal density noise of sigma 0.1 drawn with seed 1000 + i.
    Returns a list of (Lattice, U)."""
    out = []
    for i, size in enumerate(ensemble_sizes(count, seed, choices)):
        nb = size // nxb
        lat = lattice_2d(nb, nb, nxb, nxb, ng, bc=PERIODIC)
        U = sod_periodic(lat, seed=1000 + i) if i % 2 == 0 else kelvin_helmholtz(lat, seed=1000 + i)
        out.append((lat, U))
    return out


def two_level_ensemble(count: int = 8, seed: int = 0, ndim: int = 3, nxb: int = 16, ng: int = 4,
                       choices=(4, 6, 8)):
    """Ensemble of independent two-level Sedov problems of uneven sizes: problem
    i has a coarse lattice of c^ndim blocks (c drawn from `choices` with seed
    `seed`, outflow boundaries) refined over its central c/2 blocks per
    dimension, with the Sedov blast of sedov_two_level in the fine region.
    Returns a list of (TwoLevel, U)."""
    out = []
    for c in ensemble_sizes(count, seed, choices):
        lat = lattice_3d(c, c, c, nxb, nxb, nxb, ng) if ndim == 3 else lattice_2d(c, c, nxb, nxb, ng)
        lo, hi = (c // 4,) * ndim, (c - c // 4,) * ndim
        tl = two_level(lat, lo, hi)
        out.append((tl, sedov_two_level(tl)))
    return out
