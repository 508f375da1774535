// gbh_stage.cu -- the fused RK-stage kernel (one launch per stage).
//
// One stage of the non-telescoping SSP-RK method (Sec. 4.2): for every block,
// the intra-stage calculations calcLims -> calcFlux -> updSoln -> calcEos
// (Alg. "Intra stage calculations for Spark") followed by the Shu-Osher RK
// combine Uout = a*Un + b*(Uin + dt*L(Uin)); initSoln (Alg. "Block
// initializations for Spark") is the caller keeping Un.  The guard-cell fill
// that precedes every stage is fused: the halo cells the face stencil reads
// (a 2-deep slab across each face) are gathered straight from the neighbour
// blocks' interiors through the face-neighbour table, or, at an outflow
// domain edge, from the nearest interior cell.
//
// Work decomposition (one CTA = one block, or a z-chunk of one, N*N threads):
//  - the CTA marches through the z planes of its chunk; thread (i, j) keeps
//    the primitive variables of its own column at planes k, k+1 and the z
//    face state / z flux of the previous plane in registers, so each z face
//    is reconstructed and solved exactly once;
//  - per plane, the primitives of the plane plus its 2-deep x/y rims go to
//    shared memory; MC face states of the (N+2)*N x-slope cells and
//    N*(N+2) y-slope cells (with the 2N faces on the block's upper x and y
//    boundaries, which form their own face states), then the remaining N*N x
//    faces and N*N y faces are processed as flat work lists over all threads
//    (full warps, two passes of the CTA for the faces);
//  - all FP64 arithmetic is register FMAs (gbh_fastmath.cuh);
//  - the update of the plane reads its x/y fluxes from shared memory and its
//    z fluxes from registers and writes Uout.
// Optional epilogue: calcEos of Uout (the conversion to primitive variables),
// which the next stage of the call reads from a.Wout instead of converting
// its input again; at the last RK stage, the max over the CTA of the CFL
// signal speed of Uout from the same conversion, one 64-bit atomicMax per CTA
// on the bit pattern of the non-negative double (on two-level grids without
// the cells the flux correction changes afterwards).
//
// Telescoping mode (Sec. 4.2): the earlier stages also update a ring of E
// guard cells around the interior (E = 2 (S - s) for stage s of S), from the
// block's own guard cells.  The same kernel does it with an (N+2E)^2 plane
// tile shifted by -E and z planes -E .. nz+E-1; tile position (u, v) is cell
// (u-E, v-E).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbh_device.cuh"
#include "gbh_gather.cuh"
#include "gbh_internal.h"

namespace gbh {
namespace {

// Two-level grids: a cell that the flux correction changes after this stage,
// next to a face of a coarse block whose face neighbour is refined (a
// flux-register slot and a block neighbour; the slotted faces of a fine block
// face the coarser level instead).  The correction adds the CFL speed of these
// cells itself.
template <int N, bool DIM3>
__device__ __forceinline__ bool corrected_cell(const StageArgs& a, int b, int i, int j, int k, int nz) {
  if (!a.flux_slot) return false;
  const int* fs = a.flux_slot + 6 * b;
  const int* fn = a.face_nbr + 6 * b;
  auto on = [&](int f) { return __ldg(fs + f) >= 0 && __ldg(fn + f) >= 0; };
  return (i == 0 && on(FACE_XM)) || (i == N - 1 && on(FACE_XP)) || (j == 0 && on(FACE_YM)) ||
         (j == N - 1 && on(FACE_YP)) || (DIM3 && k == 0 && on(FACE_ZM)) || (DIM3 && k == nz - 1 && on(FACE_ZP));
}

// Primitives of a cell of the stage's input, in load_prim's addressing: read
// from a.Win, where the epilogue of the stage that produced Uin left them
// (calcEos of Alg. "Intra stage calculations for Spark" runs once per stage,
// after updSoln; that stage also counted their floors), or converted from Uin
// when the input comes from outside the stage sequence.  Ring stages read
// guard cells, which carry no primitives, and always convert.
template <int N, int E>
__device__ __forceinline__ int stage_prim(const StageArgs& a, const Eos& e, int b, int i, int j, int k, double W[5]) {
  if (E == 0 && a.Win) {
    const long long o = cell_offset<N>(a, b, i, j, k);
#pragma unroll
    for (int v = 0; v < 5; ++v) W[v] = __ldg(a.Win + o + v * a.lay.vstride);
    return 0;
  }
  return load_prim<N>(a, e, b, i, j, k, W);
}

// Hint: fetch the line holding *p into L1 (PTX prefetch; no register, no wait).
__device__ __forceinline__ void prefetch_l1(const double* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// Threads of a stage CTA: one per column of the band, except the 2 x 2
// corner columns of an unsplit ring-2 tile (N (N + 8), 384 = 12 whole warps at
// N = 16, against 400 = 12.5).
template <int N, int E, int S>
constexpr int stage_threads() {
  return E == 2 && S == 1 ? N * (N + 4 * E) : (N + 2 * E) * (N + 2 * E) / S;
}

// One work item: block `b` of the list (or of the lattice), z-chunk `chunk`
// and row band `band` of the plane tile.  The (N+2E)-wide plane tile is cut
// into S bands of MY = (N+2E)/S rows; a CTA of M*MY threads updates one band
// (S = 1: the whole tile).  Uses the caller's shared memory; ends with the
// per-item atomics.
template <int N, bool DIM3, int E, int S, bool BF = false>
__device__ __forceinline__ void stage_item(const StageArgs& a, int item, double* smem, double* s_red,
                                           double* s_dt) {
  constexpr int M = N + 2 * E;              // plane tile width (the interior when E = 0)
  constexpr int MY = M / S;                 // rows of one band
  constexpr int NT = stage_threads<N, E, S>();   // threads: one per updated column
  constexpr int PX = M + 4, PY = MY + 4;    // band with 2-deep x/y rims
  constexpr int QXS = MY * (M + 2);         // x face states of a band, per variable and side
  constexpr int QYS = (MY + 2) * M;         // y face states
  constexpr int FXS = MY * (M + 1);         // x fluxes per variable
  constexpr int FYS = (MY + 1) * M;         // y fluxes per variable
  double* sW = smem;                        // [5][PY][PX] primitives of the band
  double* sQx = sW + 5 * PY * PX;           // [2][5][MY][M+2] x face states (minus, plus)
  double* sQy = sQx + 2 * 5 * QXS;          // [2][5][MY+2][M] y face states
  double* sFx = sQy + 2 * 5 * QYS;          // [5][MY][M+1] x fluxes
  double* sFy = sFx + 5 * FXS;              // [5][MY+1][M] y fluxes

  const Layout& L = a.lay;
  const int tid = threadIdx.x;
  const int band = S == 1 ? 0 : item % S;
  const int rest = S == 1 ? item : item / S;
  const int y0 = band * MY;                 // first tile row of the band
  // The next stage reads a ring stage's output only in its own box (ring
  // width E - 2) and the 2-deep face slabs around it, so the 2 x 2 columns at
  // the corners of the tile, outside that box in both x and y, are never read.
  // The ring-2 stage on the whole tile (S = 1) has no thread for them (its
  // corners are exactly those 2 x 2 squares): they are not updated, and the
  // primitives of their cells, which the slopes of the neighbouring rim cells
  // need, are loaded with the rims.  The other columns are numbered row by
  // row: the rows above the interior (its columns only), the interior rows
  // (all columns), the rows below.  (At ring 4 the same 16 corner columns of
  // 576 would leave 560 threads, not a whole number of warps; that tile keeps
  // one thread per column.)
  int tx, ty;                               // band position; cell (tx - E, y0 + ty - E)
  if constexpr (E == 2 && S == 1) {
    if (tid < E * N) {
      ty = tid / N; tx = E + tid % N;
    } else if (tid < E * N + N * M) {
      const int r = tid - E * N;
      ty = E + r / M; tx = r % M;
    } else {
      const int r = tid - E * N - N * M;
      ty = E + N + r / N; tx = E + r % N;
    }
  } else {
    tx = tid % M; ty = tid / M;
  }
  const int ci = tx - E, cj = y0 + ty - E;
  const int slot_idx = rest / a.nchunks;
  const int chunk = rest - slot_idx * a.nchunks;
  const int b = a.block_list ? __ldg(a.block_list + slot_idx) : slot_idx;
  const int prob = a.problem ? __ldg(a.problem + b) : 0;
  const int k0 = DIM3 ? chunk * a.kchunk - E : 0;
  const int k1 = DIM3 ? min(L.nz + E, k0 + a.kchunk) : 1;
  // floor hits are counted on interior cells only (plane kk of this column)
  const bool col_in = E == 0 || (ci >= 0 && ci < N && cj >= 0 && cj < N);
  auto counted = [&](int kk) { return E == 0 ? kk < k1 : (col_in && kk >= 0 && kk < L.nz && kk < k1); };
  const double dt = a.dt_dev ? a.dt_dev[prob] : a.dt;
  const double idx = __ldg(a.inv_dx + 3 * b), idy = __ldg(a.inv_dx + 3 * b + 1);
  const double idz = DIM3 ? __ldg(a.inv_dx + 3 * b + 2) : 0.0;
  // FP64 constants in per-thread registers (gbh_fastmath.cuh)
  const long long zt = thread_zero(a.eos);
  const Eos e = reg_eos(a.eos, zt);
  const Rk& rk = e.k;
  // dt/dx, dt/dy, dt/dz: formed once per item by thread 0 and read back in
  // the update, after the plane's barriers (three FP64 multiplies per thread
  // otherwise, which an item of one 2-D plane pays per cell)
  if (tid == 0) {
    s_dt[0] = dt * idx;
    s_dt[1] = dt * idy;
    s_dt[2] = DIM3 ? dt * idz : 0.0;
  }

  int hits = 0;
  double smax = 0.0;
  double W0[5], Wp1[5], qpz[5], Fzm[5];     // column state carried along z
  double dz1[5];                            // Wp1 - W0 (the next z slope's left difference)

  // the face pre-pass solved the block's faces (the interior stage on whole
  // blocks: the host takes this kernel only for items of one whole block, so
  // the z march starts at the block's bottom face and ends at its top face)
  constexpr bool bf = BF && E == 0 && S == 1;
  // faces per block face in the buffer: N max(N, nz) in 3-D (x and y faces
  // have N nz, z faces N N), N in 2-D
  const int NF = DIM3 ? N * (L.nz > N ? L.nz : N) : N;
  const double* bfb = bf ? a.bflux + (long long)b * 6 * 5 * NF : nullptr;
  if (DIM3) {
    double Wm2[5], Wm1[5], qpm1[5], qm0[5];
    constexpr bool bottom = bf;                // the z face -1/2 comes from the pre-pass
    if (!bottom) stage_prim<N, E>(a, e, b, ci, cj, k0 - 2, Wm2);
    stage_prim<N, E>(a, e, b, ci, cj, k0 - 1, Wm1);
    const int h0 = stage_prim<N, E>(a, e, b, ci, cj, k0, W0);
    if (counted(k0)) hits += h0;
    const int h1 = stage_prim<N, E>(a, e, b, ci, cj, k0 + 1, Wp1);
    if (counted(k0 + 1)) hits += h1;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double d0 = sub(W0[v], Wm1[v], rk);
      if (!bottom) qpm1[v] = add(Wm1[v], mc_half_slope_d(sub(Wm1[v], Wm2[v], rk), d0, rk), rk);
      dz1[v] = sub(Wp1[v], W0[v], rk);
      const double t = mc_half_slope_d(d0, dz1[v], rk);
      qm0[v] = sub(W0[v], t, rk);
      qpz[v] = add(W0[v], t, rk);
    }
    if (bottom) {
#pragma unroll
      for (int v = 0; v < 5; ++v) Fzm[v] = bfb[(FACE_ZM * 5 + v) * NF + cj * N + ci];
    } else {
      // z face k0 - 1/2; rotated order (rho, w, u, v, p)
      double wl[5] = {qpm1[0], qpm1[3], qpm1[1], qpm1[2], qpm1[4]};
      double wr[5] = {qm0[0], qm0[3], qm0[1], qm0[2], qm0[4]};
      double f[5];
      hllc_flux(wl, wr, e, f);
      Fzm[0] = f[0]; Fzm[1] = f[2]; Fzm[2] = f[3]; Fzm[3] = f[1]; Fzm[4] = f[4];
    }
  } else {
    const int h0 = stage_prim<N, E>(a, e, b, ci, cj, 0, W0);
    if (col_in) hits += h0;
  }

  for (int k = k0; k < k1; ++k) {
    double Fzp[5], Wn[5], qpn[5];
    if constexpr (E == 0) {
      // Into L1 ahead of their use: the conserved operands of this plane's
      // update (D), which nothing else reads when the primitives come from
      // a.Win, and the z march's cell of the next iteration (plane k + 3 of
      // this column, while it lies in the block): -0.7% per step.  (A ring
      // stage reads its update operands two planes earlier with its
      // primitives; the hint there measured 0.4% slower.)
      const long long pb =
          (long long)b * L.bstride + ((long long)(k + L.gz) * L.nyp + (cj + L.g)) * L.nxp + (ci + L.g);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        prefetch_l1(a.Uin + pb + v * L.vstride);
        if (a.combine) prefetch_l1(a.Un + pb + v * L.vstride);
      }
      if (DIM3 && k + 3 < L.nz) {
        const double* src = a.Win ? a.Win : a.Uin;
#pragma unroll
        for (int v = 0; v < 5; ++v) prefetch_l1(src + pb + 3LL * L.nyp * L.nxp + v * L.vstride);
      }
    }
    if (DIM3 && bf && k == L.nz - 1) {
      // the z face nz - 1/2 comes from the pre-pass
#pragma unroll
      for (int v = 0; v < 5; ++v) Fzp[v] = bfb[(FACE_ZP * 5 + v) * NF + cj * N + ci];
    } else if (DIM3) {
      // own column: primitives at k+2, face states of k+1, z flux at k + 1/2
      const int hn = stage_prim<N, E>(a, e, b, ci, cj, k + 2, Wn);
      if (counted(k + 2)) hits += hn;
      double qmz[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double dn = sub(Wn[v], Wp1[v], rk);
        const double t = mc_half_slope_d(dz1[v], dn, rk);
        dz1[v] = dn;
        qmz[v] = sub(Wp1[v], t, rk);
        qpn[v] = add(Wp1[v], t, rk);
      }
      double wl[5] = {qpz[0], qpz[3], qpz[1], qpz[2], qpz[4]};
      double wr[5] = {qmz[0], qmz[3], qmz[1], qmz[2], qmz[4]};
      double f[5];
      hllc_flux(wl, wr, e, f);
      Fzp[0] = f[0]; Fzp[1] = f[2]; Fzp[2] = f[3]; Fzp[3] = f[1]; Fzp[4] = f[4];
    }

    // Ring stages (E > 0): the next stage reads this stage's output only in
    // its own box (ring width E - 2) and in 2-deep slabs across its faces.
    // So in the outer z planes, outside that box, only the columns of the box
    // are read: the window [2, M - 2)^2 of the tile.  There the x/y work
    // (slopes, faces, update) is done on the window alone, and rims are read
    // only where the window's slopes reach beyond the band (at a cut between
    // bands).  Elsewhere the window is the whole band.  Window bounds are in
    // band positions: columns [wx0, wx1), rows [wy0, wy1).
    const bool outer = E > 0 && (k < 2 - E || k >= L.nz + E - 2);
    const int ow = outer ? 2 : 0;
    const int wx0 = ow, wx1 = M - ow;
    // (written out for S = 1, where the band is the tile, so that the bounds
    // are compile-time constants of the interior kernel: with the clamped
    // bounds and the band's rim loop below it took 0.7% longer)
    const int wy0 = S == 1 ? ow : max(ow - y0, 0), wy1 = S == 1 ? M - ow : min(M - ow - y0, MY);
    const int Wx = wx1 - wx0, Wy = wy1 - wy0;
    // slope cells reach one position beyond the window, their stencils two
    const bool rim_xlo = wx0 <= 1, rim_xhi = wx1 >= M - 1, rim_ylo = wy0 <= 1, rim_yhi = wy1 >= MY - 1;

    // (A) primitives of plane k in the band and its 2-deep x/y rims -> shared
    //     memory (i, j: band positions)
#pragma unroll
    for (int v = 0; v < 5; ++v) sW[GBH_IX((v * PY + ty + 2) * PX + tx + 2, 5 * PY * PX)] = W0[v];
    if constexpr (S == 1) {
      // the whole tile: all four rims (and at ring 2 the 16 cells of the
      // corner columns, which have no thread) on every plane except the
      // outer planes of a ring stage, which read none (their window lies 2
      // cells inside)
      constexpr int NC = E == 2 ? 16 : 0;
      for (int r = tid; r < (outer ? 0 : 8 * M + NC); r += NT) {
        const int q = r / (2 * M), t = r - q * 2 * M;
        const int depth = t / M, pos = t - depth * M;
        int i, j;
        if (q == 0) { i = -1 - depth; j = pos; }
        else if (q == 1) { i = M + depth; j = pos; }
        else if (q == 2) { i = pos; j = -1 - depth; }
        else if (q == 3) { i = pos; j = M + depth; }
        else {
          const int c = r - 8 * M, cx = c % (2 * E), cy = c / (2 * E);
          i = cx < E ? cx : N + cx;
          j = cy < E ? cy : N + cy;
        }
        double W[5];
        stage_prim<N, E>(a, e, b, i - E, j - E, k, W);
#pragma unroll
        for (int v = 0; v < 5; ++v) sW[GBH_IX((v * PY + j + 2) * PX + i + 2, 5 * PY * PX)] = W[v];
      }
    } else {
      // a band: each rim side only where the window's slopes reach it
      for (int r = tid; r < 4 * MY + 4 * M; r += NT) {
        int i, j;
        bool need;
        if (r < 4 * MY) {
          const int side = r / (2 * MY), t = r - side * 2 * MY;
          const int depth = t / MY, pos = t - depth * MY;
          i = side == 0 ? -1 - depth : M + depth;
          j = pos;
          need = side == 0 ? rim_xlo : rim_xhi;
        } else {
          const int r2 = r - 4 * MY;
          const int side = r2 / (2 * M), t = r2 - side * 2 * M;
          const int depth = t / M, pos = t - depth * M;
          i = pos;
          j = side == 0 ? -1 - depth : MY + depth;
          need = side == 0 ? rim_ylo : rim_yhi;
        }
        if (!need) continue;
        double W[5];
        stage_prim<N, E>(a, e, b, i - E, y0 + j - E, k, W);
#pragma unroll
        for (int v = 0; v < 5; ++v) sW[GBH_IX((v * PY + j + 2) * PX + i + 2, 5 * PY * PX)] = W[v];
      }
    }
    __syncthreads();

    // Work-list rotation: the item -> thread map of (B) is shifted by
    // 32 * rot threads, rot = (k + CTA) mod 4, so the warps left without an
    // item (7 warp passes for 8 warps at N = 16) are not always the same ones;
    // the items and their arithmetic are unchanged.
    const int rtid = NT % 128 == 0 ? (tid + 32 * ((k + (int)blockIdx.x) & 3)) % NT : tid;

    // (B) MC face states: x-slope cells i in [wx0 - 1, wx1] of the window's
    //     rows, y-slope cells j in [wy0 - 1, wy1] of its columns, three
    //     consecutive cells per work item, so the two inner differences are
    //     formed once for two slopes (the last triple of a line may be
    //     partial: its reads are clamped to the line and its extra slopes not
    //     stored).  The list ends with the window's upper boundary faces x =
    //     wx1 - 1/2 and y = wy1 - 1/2, each forming the two face states it
    //     needs from the primitives (the same arithmetic as the slope items):
    //     so (C) is exactly 2 Wx Wy faces (two full passes of an unsplit CTA).
    //     In the inner planes of the unsplit ring-2 tile the next stage reads
    //     the slab lines (the 2 + 2 rows and columns outside the interior)
    //     only at the N interior positions, so these lines need no face past
    //     position N + 2 (the face between tile cells N + 1 and N + 2, which
    //     the list takes instead of their boundary face) and (C) skips their
    //     faces outside [2, N + 2): (C) is then 2 N (N + 8) faces, exactly
    //     two passes of the N (N + 8) threads.
    const bool trim = E == 2 && S == 1 && !outer;
    const int TRX = (Wx + 4) / 3, TRY = (Wy + 4) / 3;   // triples per line (W + 2 slope cells)
    const int NSX = TRX * Wy, NSY = TRY * Wx;
    for (int s = rtid; s < NSX + NSY + (bf ? 2 : 1) * (Wy + Wx); s += NT) {
      if (bf && s >= NSX + NSY) {
        // the block's boundary faces from the pre-pass: x faces 0 and N of
        // each row, y faces 0 and N of each column (plane k)
        const int f = s - NSX - NSY;
        const bool xf = f < 2 * N;
        const int side = (xf ? f : f - 2 * N) / N, line = (xf ? f : f - 2 * N) % N;
        const int face = xf ? FACE_XM + side : FACE_YM + side;
        const double* src = bfb + face * 5 * NF + line + (DIM3 ? N * k : 0);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if (xf) sFx[GBH_IX((v * MY + line) * (M + 1) + side * N, 5 * FXS)] = src[v * NF];
          else sFy[GBH_IX((v * (MY + 1) + side * N) * M + line, 5 * FYS)] = src[v * NF];
        }
        continue;
      }
      if (s >= NSX + NSY) {
        const int f = s - NSX - NSY;
        const bool xf = f < Wy;
        const int line = xf ? f : f - Wy;                       // window row (x face) or column (y face)
        const int step = xf ? 1 : PX;
        const bool slab = trim && (line < 2 || line >= M - 2);
        const int pos = xf ? (slab ? M - 2 : wx1) : (slab ? M - 2 : wy1);   // the face pos - 1/2
        // positions pos - 2 .. pos + 1 along x (or y)
        const int first = xf ? (wy0 + line + 2) * PX + pos : pos * PX + wx0 + line + 2;
        double ql[5], qr[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const double* q = sW + GBH_IX(v * PY * PX + first, 5 * PY * PX - 3 * step);
          const double a0 = q[0], a1 = q[step], a2 = q[2 * step], a3 = q[3 * step];
          const double d0 = sub(a1, a0, rk), d1 = sub(a2, a1, rk), d2 = sub(a3, a2, rk);
          ql[v] = add(a1, mc_half_slope_d(d0, d1, rk), rk);   // plus state of the last window cell
          qr[v] = sub(a2, mc_half_slope_d(d1, d2, rk), rk);   // minus state of the next cell
        }
        const int vn = xf ? 1 : 2, vt = xf ? 2 : 1;
        double wl[5] = {ql[0], ql[vn], ql[vt], ql[3], ql[4]};
        double wr[5] = {qr[0], qr[vn], qr[vt], qr[3], qr[4]};
        double F[5];
        hllc_flux(wl, wr, e, F);
        const int fs = xf ? FXS : FYS;
        double* o = xf ? sFx + GBH_IX((wy0 + line) * (M + 1) + pos, FXS)
                       : sFy + GBH_IX(pos * M + wx0 + line, FYS);
        o[0] = F[0]; o[vn * fs] = F[1]; o[vt * fs] = F[2]; o[3 * fs] = F[3]; o[4 * fs] = F[4];
        continue;
      }
      const bool xs = s < NSX;
      const int s2 = xs ? s : s - NSX;
      const int TR = xs ? TRX : TRY, Wl = xs ? Wx : Wy;
      const int line = s2 / TR, c0 = 3 * (s2 - line * TR);   // window row (x) or column (y); first slope cell + 1
      const int step = xs ? 1 : PX;
      const int first = xs ? (wy0 + line + 2) * PX + wx0 + c0 : (wy0 + c0) * PX + wx0 + line + 2;
      const int last = Wl + 3 - c0;                   // positions c0 .. Wl + 3 exist
      const int k3 = 3 < last ? 3 : last, k4 = 4 < last ? 4 : last;
      const bool two = c0 + 1 < Wl + 2, three = c0 + 2 < Wl + 2;
#pragma unroll 1
      for (int v = 0; v < 5; ++v) {
        const int os = xs ? 1 : M;                    // next slope cell
        const int op = xs ? 5 * QXS : 5 * QYS;        // plus states follow the minus states
        const double* q = sW + v * PY * PX + first;
        const double q1 = q[step], q2 = q[2 * step], q3 = q[k3 * step];
        const double d0 = sub(q1, q[0], rk), d1 = sub(q2, q1, rk), d2 = sub(q3, q2, rk);
        const double d3 = sub(q[k4 * step], q3, rk);
        const double t0 = mc_half_slope_d(d0, d1, rk), t1 = mc_half_slope_d(d1, d2, rk);
        const double t2 = mc_half_slope_d(d2, d3, rk);
        // the base slot lies in the minus half; a partial triple stores no slot past its line
        double* qm = xs ? sQx + GBH_IX((v * MY + wy0 + line) * (M + 2) + wx0 + c0, 5 * QXS)
                        : sQy + GBH_IX((v * (MY + 2) + wy0 + c0) * M + wx0 + line, 5 * QYS);
        qm[0] = sub(q1, t0, rk);
        qm[op] = add(q1, t0, rk);
        if (two) {
          qm[os] = sub(q2, t1, rk);
          qm[os + op] = add(q2, t1, rk);
        }
        if (three) {
          qm[2 * os] = sub(q3, t2, rk);
          qm[2 * os + op] = add(q3, t2, rk);
        }
      }
    }
    __syncthreads();

    // (C) HLLC on the x faces (i - 1/2, i in [wx0, wx1)) and y faces (j - 1/2,
    //     j in [wy0, wy1)) of the window; the faces at wx1 - 1/2 and wy1 - 1/2
    //     came with (B)
    // (in the inner planes of the ring-2 tile: N full lines of M faces, then
    //     the 4 slab lines at positions [2, N + 2), per direction)
    // (with the pre-pass: the N - 1 inner faces of each line only)
    const int nper = trim ? N * (N + 8) : bf ? (N - 1) * N : Wx * Wy;
    for (int f = tid; f < 2 * nper; f += NT) {
      const bool xf = f < nper;
      int i, j;                    // band positions
      const double *ql, *qr;       // minus/plus state arrays, var stride vs
      int vs, ol, orr;
      int line = 0, pos = 0;       // trimmed mapping: face pos - 1/2 of line
      if (trim) {
        const int g = xf ? f : f - nper;
        if (g < N * M) {
          line = 2 + g / M; pos = g - (line - 2) * M;
        } else {
          const int h = g - N * M, sl = h / N;
          line = sl < 2 ? sl : N + sl; pos = 2 + h - sl * N;
        }
      }
      if (xf) {
        if (trim) { i = pos; j = line; }
        else if (bf) { i = f % (N - 1) + 1; j = f / (N - 1); }
        else { i = f % Wx + wx0; j = f / Wx + wy0; }
        vs = QXS;
        ol = 5 * vs + j * (M + 2) + i;        // plus state of cell i-1 (slot i)
        orr = j * (M + 2) + i + 1;            // minus state of cell i (slot i+1)
        ql = sQx; qr = sQx;
      } else {
        const int f2 = f - nper;
        if (trim) { i = line; j = pos; }
        else if (bf) { i = f2 % N; j = f2 / N + 1; }
        else { i = f2 % Wx + wx0; j = f2 / Wx + wy0; }
        vs = QYS;
        ol = 5 * vs + j * M + i;              // plus state of cell j-1 (slot j)
        orr = (j + 1) * M + i;                // minus state of cell j (slot j+1)
        ql = sQy; qr = sQy;
      }
      const int vn = xf ? 1 : 2, vt = xf ? 2 : 1;   // normal and first tangential momentum
      double wl[5] = {ql[ol], ql[ol + vn * vs], ql[ol + vt * vs], ql[ol + 3 * vs], ql[ol + 4 * vs]};
      double wr[5] = {qr[orr], qr[orr + vn * vs], qr[orr + vt * vs], qr[orr + 3 * vs], qr[orr + 4 * vs]};
      double F[5];
      hllc_flux(wl, wr, e, F);
      if (xf) {
        double* o = sFx + GBH_IX(j * (M + 1) + i, FXS);
        o[0] = F[0]; o[vn * FXS] = F[1]; o[vt * FXS] = F[2]; o[3 * FXS] = F[3]; o[4 * FXS] = F[4];
      } else {
        double* o = sFy + GBH_IX(j * M + i, FYS);
        o[0] = F[0]; o[vn * FYS] = F[1]; o[vt * FYS] = F[2]; o[3 * FYS] = F[3]; o[4 * FYS] = F[4];
      }
    }
    __syncthreads();

    // (D) updSoln + RK combine for cell (ci, cj, k):
    //     Uin + dt L = Uin - dt/dx dFx - dt/dy dFy - dt/dz dFz
    const long long base =
        (long long)b * L.bstride + ((long long)(k + L.gz) * L.nyp + (cj + L.g)) * L.nxp + (ci + L.g);
    // in an outer plane of a ring stage only the window's cells are updated
    // (the others are never read again and their fluxes were not formed)
    const bool upd = !outer || (tx >= wx0 && tx < wx1 && ty >= wy0 && ty < wy1);
    double out[5];
    const double dtx = reg_const(s_dt[0], zt), dty = reg_const(s_dt[1], zt), dtz = reg_const(s_dt[2], zt);
#pragma unroll
    for (int v = 0; v < 5 && upd; ++v) {
      const double fx = sub(sFx[GBH_IX((v * MY + ty) * (M + 1) + tx + 1, 5 * FXS)], sFx[(v * MY + ty) * (M + 1) + tx], rk);
      const double fy = sub(sFy[GBH_IX((v * (MY + 1) + ty + 1) * M + tx, 5 * FYS)], sFy[(v * (MY + 1) + ty) * M + tx], rk);
      const long long o = GBH_IX(base + v * L.vstride, (long long)L.nblocks * L.bstride);
      double r = fma(-dtx, fx, __ldg(a.Uin + o));
      r = fma(-dty, fy, r);
      if (DIM3) r = fma(-dtz, sub(Fzp[v], Fzm[v], rk), r);
      // combine 2: a = b = 1/2 (second SSP-RK2 stage), one FP64 add
      out[v] = a.combine == 2 ? half_any(add(a.Un[o], r, rk))
               : a.combine ? fma(reg_const(a.a, zt), a.Un[o], mul(reg_const(a.b, zt), r, rk)) : r;
      a.Uout[o] = out[v];
    }
    if (a.flux_slot && col_in && (E == 0 || (k >= 0 && k < L.nz))) {
      // fluxBuff: fluxes through the block's faces on a coarse-fine boundary,
      // for the correction (interior cells next to the face write them)
      const long long n2 = DIM3 ? N : 1;
      const long long ss = 5 * n2 * N;
      const int* fsl = a.flux_slot + 6 * b;
      const int t2k = DIM3 ? k : 0;
      if (ci == 0 && fsl[FACE_XM] >= 0)
        for (int v = 0; v < 5; ++v)
          a.flux_reg[GBH_IX(fsl[FACE_XM] * ss + (v * n2 + t2k) * N + cj, a.flux_reg_len)] = sFx[(v * MY + ty) * (M + 1) + tx];
      if (ci == N - 1 && fsl[FACE_XP] >= 0)
        for (int v = 0; v < 5; ++v)
          a.flux_reg[GBH_IX(fsl[FACE_XP] * ss + (v * n2 + t2k) * N + cj, a.flux_reg_len)] = sFx[(v * MY + ty) * (M + 1) + tx + 1];
      if (cj == 0 && fsl[FACE_YM] >= 0)
        for (int v = 0; v < 5; ++v)
          a.flux_reg[GBH_IX(fsl[FACE_YM] * ss + (v * n2 + t2k) * N + ci, a.flux_reg_len)] = sFy[(v * (MY + 1) + ty) * M + tx];
      if (cj == N - 1 && fsl[FACE_YP] >= 0)
        for (int v = 0; v < 5; ++v)
          a.flux_reg[GBH_IX(fsl[FACE_YP] * ss + (v * n2 + t2k) * N + ci, a.flux_reg_len)] = sFy[(v * (MY + 1) + ty + 1) * M + tx];
      if (DIM3 && k == 0 && fsl[FACE_ZM] >= 0)
        for (int v = 0; v < 5; ++v) a.flux_reg[GBH_IX(fsl[FACE_ZM] * ss + (v * n2 + cj) * N + ci, a.flux_reg_len)] = Fzm[v];
      if (DIM3 && k == L.nz - 1 && fsl[FACE_ZP] >= 0)
        for (int v = 0; v < 5; ++v) a.flux_reg[GBH_IX(fsl[FACE_ZP] * ss + (v * n2 + cj) * N + ci, a.flux_reg_len)] = Fzp[v];
    }
    if (E == 0 && (a.smax_acc || a.Wout)) {
      // calcEos of the new state: the CFL speed, and the next stage's primitives
      double W[5], ir;
      const int h = cons_to_prim_ir(out, W, e, ir);
      if (a.Wout) {
#pragma unroll
        for (int v = 0; v < 5; ++v) a.Wout[GBH_IX(base + v * L.vstride, (long long)L.nblocks * L.bstride)] = W[v];
        hits += h;
      }
      if (a.smax_acc) {
        const double sp = signal_speed_ir(W, ir, e, reg_const(idx, zt), reg_const(idy, zt), reg_const(idz, zt), DIM3);
        if (!corrected_cell<N, DIM3>(a, b, ci, cj, k, L.nz)) smax = max_nonneg(smax, sp);
      }
    }

    if (DIM3) {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        W0[v] = Wp1[v];
        Wp1[v] = Wn[v];
        qpz[v] = qpn[v];
        Fzm[v] = Fzp[v];
      }
    }
  }

  if (hits) atomicAdd(a.floor_count, (unsigned long long)hits);
  if (E == 0 && a.smax_acc) {
    const double m = block_max<NT>(smax, s_red);   // warp shuffles, then across warps
    if (tid == 0) atomicMax(a.smax_acc + prob, (unsigned long long)__double_as_longlong(m));
  }
}

// The face pre-pass: one thread per (block, face, face cell) over blocks
// [lo, hi).  The flux through a face is solved once: by the block on its high
// side (x = N - 1/2, y = N - 1/2, z = nz - 1/2, which also writes it into the
// neighbour's slot for that neighbour's low face), and, where a block has no
// face neighbour on a low side (an outflow edge, or on a two-level grid a face
// whose halo is the block's own prolonged guard cells), by that block.  When
// the stage runs over consecutive block ranges in order (the host-buffer
// pipeline), a low face whose neighbour lies in a later range (a periodic
// wrap) is solved by the block itself, and a high face is written into the
// neighbour's slot only when the neighbour is in this range or a later one
// (an earlier range's stage has already read its slots).  Face states as the stage
// kernel forms them (the plus state of the cell below the face, the minus
// state of the cell above, MC slopes of the primitives, the same arithmetic
// and halo addressing), the same HLLC, the same rotations: the stage reads
// the same bits it would have formed.
template <int N, bool DIM3>
__global__ void __launch_bounds__(256) face_flux_kernel(const StageArgs a, double* __restrict__ out, int lo,
                                                        int hi) {
  const int nz = a.lay.nz;
  const int NF = DIM3 ? N * (nz > N ? nz : N) : N;   // slots per block face (x, y faces: N nz; z faces: N N)
  constexpr int NFACES = DIM3 ? 6 : 4;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)(hi - lo) * NFACES * NF) return;
  const int bl = (int)(t / (NFACES * NF));
  const int r = (int)(t - (long long)bl * NFACES * NF);
  const int b = lo + bl;
  const int face = r / NF, tt = r - face * NF;
  const int d = face >> 1, side = face & 1;
  if (DIM3 && tt / N >= (d == 2 ? N : nz)) return;  // past the face's extent
  const int nb = __ldg(a.face_nbr + 6 * b + face);
  if (side == 0 && nb >= 0 && nb < hi) return;  // solved by the neighbour, as its high face
  const long long zt = thread_zero(a.eos);
  const Eos e = reg_eos(a.eos, zt);
  const Rk& rk = e.k;
  // the cell coordinates along the normal: two below the face, two above
  const int p0 = side ? (d == 2 ? nz : N) - 2 : -2;
  const int t1 = tt % N, t2 = DIM3 ? tt / N : 0;
  double Q[4][5];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int i, j, k;
    if (d == 0) { i = p0 + c; j = t1; k = t2; }
    else if (d == 1) { i = t1; j = p0 + c; k = t2; }
    else { i = t1; j = t2; k = p0 + c; }
    stage_prim<N, 0>(a, e, b, i, j, k, Q[c]);
  }
  double ql[5], qr[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double d0 = sub(Q[1][v], Q[0][v], rk), d1 = sub(Q[2][v], Q[1][v], rk), d2 = sub(Q[3][v], Q[2][v], rk);
    ql[v] = add(Q[1][v], mc_half_slope_d(d0, d1, rk), rk);   // plus state of the cell below
    qr[v] = sub(Q[2][v], mc_half_slope_d(d1, d2, rk), rk);   // minus state of the cell above
  }
  // rotated order: the normal momentum second (x: rho u v w p; y: rho v u w p; z: rho w u v p)
  const int vn = d + 1, va = d == 0 ? 2 : 1, vb = d == 2 ? 2 : 3;
  double wl[5] = {ql[0], ql[vn], ql[va], ql[vb], ql[4]};
  double wr[5] = {qr[0], qr[vn], qr[va], qr[vb], qr[4]};
  double F[5];
  hllc_flux(wl, wr, e, F);
  double G[5];
  G[0] = F[0]; G[vn] = F[1]; G[va] = F[2]; G[vb] = F[3]; G[4] = F[4];
  double* o = out + ((long long)b * 6 + face) * 5 * NF + tt;
#pragma unroll
  for (int v = 0; v < 5; ++v) o[v * NF] = G[v];
  if (side == 1 && nb >= lo) {
    double* on = out + ((long long)nb * 6 + (face - 1)) * 5 * NF + tt;
#pragma unroll
    for (int v = 0; v < 5; ++v) on[v * NF] = G[v];
  }
}

// CTAs per SM the register budget is sized for: an unsplit interior tile
// (256 threads at N = 16) two, a band of it four; a ring tile one, a band
// of it two.
template <int E, int S>
constexpr int min_ctas() { return (E == 0 ? 2 : 1) * S; }

// Work list: items (block, z-chunk, band) in order; each CTA processes
// `items_per_cta` consecutive items (1 = one CTA per item; a machine-sized
// grid makes the kernel persistent).  No CTA waits on another.
template <int N, bool DIM3, int E, int S, bool BF = false>
__global__ void __launch_bounds__(stage_threads<N, E, S>(), min_ctas<E, S>()) stage_kernel(const StageArgs a) {
  constexpr int NT = stage_threads<N, E, S>();
  extern __shared__ double smem[];
  __shared__ double s_red[E == 0 && NT > 32 ? NT / 32 : 1];
  __shared__ double s_dt[3];
  const int nitems = (a.block_list ? a.nlist : a.lay.nblocks) * a.nchunks * S;
  const int first = blockIdx.x * a.items_per_cta;
  const int last = min(nitems, first + a.items_per_cta);
  for (int item = first; item < last; ++item) {
    stage_item<N, DIM3, E, S, BF>(a, item, smem, s_red, s_dt);
    __syncthreads();
  }
}

template <int N, int E, int S>
constexpr size_t smem_for() {
  constexpr int M = N + 2 * E;
  constexpr int MY = M / S;
  return sizeof(double) * (5 * (MY + 4) * (M + 4) + 2 * 5 * MY * (M + 2) + 2 * 5 * (MY + 2) * M +
                           5 * MY * (M + 1) + 5 * (MY + 1) * M);
}

template <int N, bool D3, int E, int S, bool BF = false>
cudaError_t launch_t(const StageArgs& a, cudaStream_t s) {
  const long long nitems = (long long)(a.block_list ? a.nlist : a.lay.nblocks) * a.nchunks * S;
  const int per = a.items_per_cta > 0 ? a.items_per_cta : 1;
  const unsigned grid = (unsigned)((nitems + per - 1) / per);
  stage_kernel<N, D3, E, S, BF><<<grid, stage_threads<N, E, S>(), smem_for<N, E, S>(), s>>>(a);
  return cudaGetLastError();
}

template <int N, bool D3, int E, int S, bool BF = false>
cudaError_t prepare_one() {
  return cudaFuncSetAttribute(stage_kernel<N, D3, E, S, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_for<N, E, S>());
}

// The row-band split (S = 2) exists for N >= 8 (a band of at least 4 rows).
template <int N, bool D3>
cudaError_t prepare_t() {
  cudaError_t e = prepare_one<N, D3, 0, 1>();
  if (e == cudaSuccess) e = prepare_one<N, D3, 0, 1, true>();
  if (e == cudaSuccess) e = prepare_one<N, D3, 2, 1>();
  if (e == cudaSuccess) e = prepare_one<N, D3, 4, 1>();
  if constexpr (N >= 8) {
    if (e == cudaSuccess) e = prepare_one<N, D3, 0, 2>();
    if (e == cudaSuccess) e = prepare_one<N, D3, 2, 2>();
    if (e == cudaSuccess) e = prepare_one<N, D3, 4, 2>();
  }
  return e;
}

template <int N, bool D3, int E>
cudaError_t launch_s(const StageArgs& a, cudaStream_t s) {
  if constexpr (N >= 8) {
    if (a.ysplit == 2) return launch_t<N, D3, E, 2>(a, s);
  }
  if (a.ysplit != 1) return cudaErrorInvalidValue;
  if constexpr (E == 0) {
    if (a.bflux) return launch_t<N, D3, 0, 1, true>(a, s);
  }
  return launch_t<N, D3, E, 1>(a, s);
}

template <int E>
cudaError_t launch_e(const StageArgs& a, cudaStream_t s) {
  const bool d3 = a.lay.ndim == 3;
  switch (a.lay.nx) {
    case 4: return d3 ? launch_s<4, true, E>(a, s) : launch_s<4, false, E>(a, s);
    case 8: return d3 ? launch_s<8, true, E>(a, s) : launch_s<8, false, E>(a, s);
    case 16: return d3 ? launch_s<16, true, E>(a, s) : launch_s<16, false, E>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

GBH_CHECK_TAKE(check_take_stage)

size_t stage_smem_bytes(int nx) {
  switch (nx) {
    case 4: return smem_for<4, 0, 1>();
    case 8: return smem_for<8, 0, 1>();
    case 16: return smem_for<16, 0, 1>();
    default: return 0;
  }
}

cudaError_t stage_prepare(int nx, int ndim) {
  const bool d3 = ndim == 3;
  switch (nx) {
    case 4: return d3 ? prepare_t<4, true>() : prepare_t<4, false>();
    case 8: return d3 ? prepare_t<8, true>() : prepare_t<8, false>();
    case 16: return d3 ? prepare_t<16, true>() : prepare_t<16, false>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stage(const StageArgs& a, cudaStream_t s) { return launch_e<0>(a, s); }

cudaError_t launch_face_fluxes(const StageArgs& a, double* out, cudaStream_t s, int lo, int hi) {
  const bool d3 = a.lay.ndim == 3;
  if (hi < 0) hi = a.lay.nblocks;
  if (lo < 0 || lo > hi || hi > a.lay.nblocks) return cudaErrorInvalidValue;
  if (lo == hi) return cudaSuccess;
  const long long total =
      (long long)(hi - lo) * (d3 ? 6 : 4) * a.lay.nx * (d3 ? (a.lay.nz > a.lay.nx ? a.lay.nz : a.lay.nx) : 1);
  const unsigned grid = (unsigned)((total + 255) / 256);
  switch (a.lay.nx) {
    case 4: d3 ? face_flux_kernel<4, true><<<grid, 256, 0, s>>>(a, out, lo, hi) : face_flux_kernel<4, false><<<grid, 256, 0, s>>>(a, out, lo, hi); break;
    case 8: d3 ? face_flux_kernel<8, true><<<grid, 256, 0, s>>>(a, out, lo, hi) : face_flux_kernel<8, false><<<grid, 256, 0, s>>>(a, out, lo, hi); break;
    case 16: d3 ? face_flux_kernel<16, true><<<grid, 256, 0, s>>>(a, out, lo, hi) : face_flux_kernel<16, false><<<grid, 256, 0, s>>>(a, out, lo, hi); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_stage_ring(const StageArgs& a, int ring, cudaStream_t s) {
  if (a.gather || a.smax_acc || a.lay.g < ring + 2) return cudaErrorInvalidValue;
  switch (ring) {
    case 0: return launch_e<0>(a, s);
    case 2: return launch_e<2>(a, s);
    case 4: return launch_e<4>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gbh
