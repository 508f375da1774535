"""Index maps of the kernels, restated on the CPU: the thread -> column map and the
face lists of the stage kernel's unsplit ring-2 tile, the face pre-pass's
thread -> face-cell map and its slots against the stage kernel's reads
(gbh_stage.cu), the guard-cell enumeration of the fill kernel and the cell map
of the interior scatter / gather (gbh_aux.cu).

The telescoping variant's first stage (Sec. 4.2) updates the interior widened
by 2 cells; the next stage reads that output in its own box and in the 2-deep
slabs across its faces, never in the 2 x 2 corner columns.  The kernel
launches N (N + 8) threads (no thread for a corner column) and, in the inner
planes, forms only the faces the update of those columns reads: every face of
the N interior lines, the faces at positions [2, N + 2] of the 4 slab lines.
These tests check that the maps are one-to-one, cover exactly what the update
reads, and give whole warps and exactly two passes of the face list."""
import pytest

E = 2


def thread_columns(N):
    """(tx, ty) tile position of each thread: rows above the interior (interior
    columns only), the interior rows (all columns), the rows below."""
    M = N + 2 * E
    out = []
    for tid in range(N * (N + 4 * E)):
        if tid < E * N:
            ty, tx = tid // N, E + tid % N
        elif tid < E * N + N * M:
            r = tid - E * N
            ty, tx = E + r // M, r % M
        else:
            r = tid - E * N - N * M
            ty, tx = E + N + r // N, E + r % N
        out.append((tx, ty))
    return out


def face_list_c(N):
    """Faces of phase (C) in the inner planes: ('x', i, j) is the x face
    i - 1/2 of row j, ('y', i, j) the y face j - 1/2 of column i."""
    M = N + 2 * E
    nper = N * (N + 8)
    out = []
    for f in range(2 * nper):
        xf = f < nper
        g = f if xf else f - nper
        if g < N * M:
            line = 2 + g // M
            pos = g - (line - 2) * M
        else:
            h = g - N * M
            sl = h // N
            line = sl if sl < 2 else N + sl
            pos = 2 + h - sl * N
        out.append(("x", pos, line) if xf else ("y", line, pos))
    return out


def boundary_faces_b(N):
    """The faces the slope phase (B) solves: the tile's upper boundary face of
    every line, or, on a slab line, the face at position N + 2."""
    M = N + 2 * E
    out = []
    for f in range(2 * M):
        xf = f < M
        line = f if xf else f - M
        pos = M - 2 if (line < 2 or line >= M - 2) else M
        out.append(("x", pos, line) if xf else ("y", line, pos))
    return out


@pytest.mark.parametrize("N", [4, 8, 16])
def test_threads_cover_the_columns_but_the_corners(N):
    M = N + 2 * E
    cols = thread_columns(N)
    assert len(set(cols)) == len(cols) == N * (N + 8)
    corner = {(x, y) for x in range(M) for y in range(M)
              if not (E <= x < E + N) and not (E <= y < E + N)}
    assert len(corner) == 4 * E * E
    assert set(cols) == {(x, y) for x in range(M) for y in range(M)} - corner
    if N == 16:
        assert len(cols) == 384 and len(cols) % 32 == 0


@pytest.mark.parametrize("N", [4, 8, 16])
def test_face_lists_are_exactly_what_the_update_reads(N):
    M = N + 2 * E
    c, b = face_list_c(N), boundary_faces_b(N)
    assert len(set(c)) == len(c) and len(set(b)) == len(b) and not set(c) & set(b)
    for d, i, j in c + b:
        assert 0 <= i <= M and 0 <= j <= M
    need = set()
    for tx, ty in thread_columns(N):
        need |= {("x", tx, ty), ("x", tx + 1, ty), ("y", tx, ty), ("y", tx, ty + 1)}
    assert set(c) | set(b) == need
    # two full passes of the threads, against 2 M^2 faces (a third, partial pass) untrimmed
    assert len(c) == 2 * len(thread_columns(N))
    assert 2 * M * M > len(c)


def fill_plane_cells(n, g, nd, kk):
    """Cells (jj, ii) the fill kernel's threads take in padded plane kk."""
    nxp = n + 2 * g
    gz = g if nd == 3 else 0
    nz = n if nd == 3 else 1
    cz = kk - gz
    zguard = cz < 0 or cz >= nz
    full = 2 * g * nxp
    out = []
    for q in range(nxp * nxp if zguard else full + n * 2 * g):
        if zguard:
            jj, ii = divmod(q, nxp)
        elif q < full:
            r = q // nxp
            jj, ii = (r if r < g else n + r), q - r * nxp
        else:
            row, side = divmod(q - full, 2 * g)
            jj, ii = g + row, (side if side < g else n + side)
        out.append((jj, ii))
    return out


@pytest.mark.parametrize("nd", [2, 3])
@pytest.mark.parametrize("n,g", [(4, 2), (8, 3), (16, 4), (8, 6)])
def test_fill_enumeration_covers_each_guard_cell_once(nd, n, g):
    """The guard fill (Sec. 4.2) takes, per (block, padded z plane), exactly the
    plane's guard cells: the whole plane outside the interior z range, else the
    g full rows below and above the interior rows and the g-cell x guards."""
    nxp = n + 2 * g
    gz = g if nd == 3 else 0
    nzp = n + 2 * gz if nd == 3 else 1
    got = [(kk,) + c for kk in range(nzp) for c in fill_plane_cells(n, g, nd, kk)]
    assert len(got) == len(set(got))
    inside = lambda x: g <= x < g + n
    want = {(kk, jj, ii) for kk in range(nzp) for jj in range(nxp) for ii in range(nxp)
            if not (inside(ii) and inside(jj) and (kk - gz >= 0 and kk - gz < (n if nd == 3 else 1)))}
    assert set(got) == want


def interior_copy_launches(nblocks, n, g, nd, b0, nb):
    """The launcher's split of blocks [b0, b0 + nb) (at most 2^30 cells per
    launch) and, per launch, the kernel's map from the cell index t to the
    offset in the padded blocks and in the interior-only blocks."""
    nx = ny = n
    nz = n if nd == 3 else 1
    gz = g if nd == 3 else 0
    nxp, nyp, nzp = nx + 2 * g, ny + 2 * g, nz + 2 * gz
    vstride = nxp * nyp * nzp
    bstride = 5 * vstride
    per = nx * ny * nz
    cells = 5 * per
    per_launch = max((1 << 30) // cells, 1)
    out = []
    b = b0
    while b < b0 + nb:
        cnt = min(per_launch, b0 + nb - b)
        total = cells * cnt
        assert total < (1 << 30) + cells and total + 152 * 16 * 256 < (1 << 32)
        for t in range(total):
            bl, r = divmod(t, cells)
            v, r = divmod(r, per)
            i, r = r % nx, r // nx
            j, k = r % ny, r // ny
            o = bl * bstride + v * vstride + ((k + gz) * nyp + (j + g)) * nxp + (i + g)
            assert 0 <= o < cnt * bstride
            out.append((b * bstride + o, b * cells + t))
        b += cnt
    return out, (nxp, nyp, nzp, bstride, cells)


@pytest.mark.parametrize("nd,n,g,nblocks,b0,nb", [(3, 4, 2, 5, 1, 3), (3, 8, 4, 3, 0, 3), (2, 16, 4, 7, 2, 4),
                                                   (2, 4, 3, 6, 5, 1)])
def test_interior_copy_maps_each_interior_cell_once(nd, n, g, nblocks, b0, nb):
    """hydro_step_host_interior's scatter / gather: every interior cell of the
    chunk's blocks once, no guard cell, the interior-only index in layout
    order [block][var][z][y][x] and inside the chunk's range on both sides."""
    pairs, (nxp, nyp, nzp, bstride, cells) = interior_copy_launches(nblocks, n, g, nd, b0, nb)
    gz = g if nd == 3 else 0
    nz = n if nd == 3 else 1
    pads = [p for p, _ in pairs]
    ints = [c for _, c in pairs]
    assert ints == list(range(b0 * cells, (b0 + nb) * cells))
    assert len(set(pads)) == len(pads)
    want = set()
    for b in range(b0, b0 + nb):
        for v in range(5):
            for k in range(nz):
                for j in range(n):
                    for i in range(n):
                        want.add(b * bstride + v * nxp * nyp * nzp + ((k + gz) * nyp + j + g) * nxp + i + g)
    assert set(pads) == want
    # consecutive cells along x are consecutive on both sides (whole rows)
    for (p0, c0), (p1, c1) in zip(pairs, pairs[1:]):
        if c1 % n:
            assert p1 == p0 + 1 and c1 == c0 + 1


def prepass_thread_cells(N, nz, nblocks, lo, hi):
    """The face pre-pass's thread map over blocks [lo, hi) (face_flux_kernel,
    3-D): (block, face, cell coordinates i, j, k of the face's cell index, slot
    index tt) per thread that solves a face, before the neighbour rules."""
    NF = N * max(N, nz)
    out = []
    for t in range((hi - lo) * 6 * NF):
        bl, r = divmod(t, 6 * NF)
        b = lo + bl
        face, tt = divmod(r, NF)
        d = face >> 1
        if tt // N >= (N if d == 2 else nz):
            continue
        t1, t2 = tt % N, tt // N
        ijk = {0: ("-", t1, t2), 1: (t1, "-", t2), 2: (t1, t2, "-")}[d]
        out.append((b, face, ijk, tt))
    return out, NF


def stage_read_slot(N, face, i, j, k):
    """Slot index the stage kernel reads for a face cell: x faces row j of plane
    k (j + N k), y faces column i of plane k (i + N k), z faces (i + N j)."""
    d = face >> 1
    return {0: j + N * k, 1: i + N * k, 2: i + N * j}[d]


@pytest.mark.parametrize("N,nz,nblocks,lo,hi", [(16, 16, 3, 0, 3), (16, 8, 4, 1, 3), (8, 12, 5, 2, 5), (4, 4, 2, 0, 1)])
def test_prepass_slots_match_the_stage_reads(N, nz, nblocks, lo, hi):
    """Every face cell of the range's blocks has one thread, its slot is the
    one the stage kernel reads for that cell, and slots stay inside
    [nblocks][6][5][N max(N, nz)] (non-cubic blocks too)."""
    cells, NF = prepass_thread_cells(N, nz, nblocks, lo, hi)
    keys = [(b, f, ijk) for b, f, ijk, _ in cells]
    assert len(keys) == len(set(keys))
    want = set()
    for b in range(lo, hi):
        for f in range(6):
            d = f >> 1
            ext = {0: (N, nz), 1: (N, nz), 2: (N, N)}[d]
            for t2 in range(ext[1]):
                for t1 in range(ext[0]):
                    want.add((b, f, {0: ("-", t1, t2), 1: (t1, "-", t2), 2: (t1, t2, "-")}[d]))
    assert set(keys) == want
    total = nblocks * 6 * 5 * NF
    for b, f, (i, j, k), tt in cells:
        ii = 0 if i == "-" else i
        jj = 0 if j == "-" else j
        kk = 0 if k == "-" else k
        assert stage_read_slot(N, f, ii, jj, kk) == tt
        for v in range(5):
            assert 0 <= ((b * 6 + f) * 5 + v) * NF + tt < total
