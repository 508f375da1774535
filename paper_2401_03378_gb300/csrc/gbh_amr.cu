// gbh_amr.cu -- two-level composite grid: restriction, prolongation into fine
// guard cells, and the coarse-side flux correction.
//
// Sec. 4.2 of the paper (all-levels listing): every leaf block of every level
// is advanced in one sweep; then the fluxes through coarse-fine boundaries are
// communicated and the coarse side corrected; Sec. 2.2: blocks of all levels
// hold the same number of cells, only the cell width differs.  The formulas
// are not in the paper; the readings used (refinement ratio 2, one dt):
//  - restriction: a covered coarse cell = mean of its 2^d children, summed in
//    the order (z, y, x) of the child offsets;
//  - prolongation: a fine guard cell whose region lies on the coarser level =
//    u_c + sum_d s_d sigma_d / 4 (s_d = -1 for the lower child, +1 for the
//    upper), sigma_d the MC slope of the conserved coarse variable;
//  - flux correction: the coarse flux through a face on the boundary of the
//    fine region is replaced by the mean of the fine fluxes through it:
//    U += b dt (F_c - mean F_f) / dx (low side of the face; opposite sign on
//    the high side), b = the stage's weight of L.
// With a primitive array W (the primitive carry between the stages of an
// all-levels step), each kernel also writes the primitive variables of the
// cells it writes, so that the next stage reads them for every cell of its
// stencil: restricted covered cells, prolonged fine guard cells, corrected
// coarse cells (the conversion of the stage kernel, no floor counted: these
// cells are read as halo or were counted by the stage that produced them).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbh_check.cuh"
#include "gbh_device.cuh"
#include "gbh_internal.h"

namespace gbh {
namespace {

constexpr int kThreads = 256;

int grid_for(long long work) {
  long long g = (work + kThreads - 1) / kThreads;
  if (g > 152LL * 16) g = 152LL * 16;
  return (int)(g < 1 ? 1 : g);
}

__device__ __forceinline__ long long at(const Layout& L, int b, int v, int i, int j, int k) {
  return GBH_IX((long long)b * L.bstride + v * L.vstride + ((long long)(k + L.gz) * L.nyp + (j + L.g)) * L.nxp + (i + L.g),
                (long long)L.nblocks * L.bstride);
}

// Primitives of the conserved vector Uc at state offset o (cell offset, variable 0).
__device__ __forceinline__ void write_prim(double* W, const Layout& L, long long o, const double Uc[5], const Eos& e) {
  double Wp[5];
  cons_to_prim(Uc, Wp, e);
  for (int v = 0; v < 5; ++v) W[GBH_IX(o + v * L.vstride, (long long)L.nblocks * L.bstride)] = Wp[v];
}

// Restriction: one thread per (covered block, interior cell); 5 variables.
__global__ void restrict_kernel(double* U, const AmrArgs a, double* W) {
  const Layout& L = a.lay;
  const Eos e = reg_eos(a.eos, thread_zero(a.eos));
  const int n[3] = {L.nx, L.ny, L.nz};
  const int h[3] = {L.nx / 2, L.ny / 2, L.ndim == 3 ? L.nz / 2 : 1};
  const long long per = (long long)L.nx * L.ny * L.nz;
  const long long total = per * a.ncovered;
  const double w = L.ndim == 3 ? 0.125 : 0.25;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int cb = __ldg(a.covered + t / per);
    long long r = t % per;
    const int i = (int)(r % n[0]);
    r /= n[0];
    const int j = (int)(r % n[1]);
    const int k = (int)(r / n[1]);
    const int oct = (i / h[0]) + 2 * (j / h[1]) + (L.ndim == 3 ? 4 * (k / h[2]) : 0);
    const int child = __ldg(a.children + 8 * cb + oct);
    const int fi = 2 * (i % h[0]), fj = 2 * (j % h[1]), fk = L.ndim == 3 ? 2 * (k % h[2]) : 0;
    double Uc[5];
    for (int v = 0; v < 5; ++v) {
      double s = 0.0;
      for (int dz = 0; dz < (L.ndim == 3 ? 2 : 1); ++dz)
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx) s = __dadd_rn(s, U[at(L, child, v, fi + dx, fj + dy, fk + dz)]);
      Uc[v] = __dmul_rn(s, w);
      U[at(L, cb, v, i, j, k)] = Uc[v];
    }
    if (W) write_prim(W, L, at(L, cb, 0, i, j, k), Uc, e);
  }
}

// Coarse cell at parent-local coordinates (x, y, z), which may lie outside
// the parent block in any direction by at most one block: resolved through
// the parent's 27-entry neighbour table (clamped at an outflow edge).
__device__ __forceinline__ long long coarse_offset(const AmrArgs& a, int parent, int x, int y, int z) {
  const Layout& L = a.lay;
  const int n[3] = {L.nx, L.ny, L.nz};
  int c[3] = {x, y, z};
  int o[3];
  for (int d = 0; d < 3; ++d) o[d] = c[d] < 0 ? -1 : (c[d] >= n[d] ? 1 : 0);
  int blk = parent;
  if (o[0] | o[1] | o[2]) {
    const int e = L.ndim == 3 ? (o[2] + 1) * 9 + (o[1] + 1) * 3 + (o[0] + 1) : (o[1] + 1) * 3 + (o[0] + 1);
    const int nb = __ldg(a.nbr + (long long)(L.ndim == 3 ? 27 : 9) * parent + e);
    if (nb >= 0) {
      blk = nb;
      for (int d = 0; d < 3; ++d) c[d] -= o[d] * n[d];
    } else {
      for (int d = 0; d < 3; ++d) c[d] = c[d] < 0 ? 0 : (c[d] >= n[d] ? n[d] - 1 : c[d]);
    }
  }
  return GBH_IX((long long)blk * L.bstride + ((long long)(c[2] + L.gz) * L.nyp + (c[1] + L.g)) * L.nxp + (c[0] + L.g),
                (long long)L.nblocks * L.bstride - 4 * L.vstride);
}

__device__ __forceinline__ int floor_div2(int x) { return x >= 0 ? x / 2 : -((1 - x) / 2); }

// Prolongation into the guard cells of fine blocks whose region lies on the
// coarser level (neighbour code GBH_NBR_COARSER).  One thread per (task,
// cell): a task is one fine block; `depth` limits the guard depth and
// `faces_only` restricts to the face slabs (what the stage kernel reads).
__global__ void prolong_kernel(double* U, const AmrArgs a, int depth, int faces_only, double* W) {
  const Layout& L = a.lay;
  const Eos eo = reg_eos(a.eos, thread_zero(a.eos));
  const int n[3] = {L.nx, L.ny, L.nz};
  const int gg[3] = {depth, depth, L.ndim == 3 ? depth : 0};
  const int ex[3] = {n[0] + 2 * gg[0], n[1] + 2 * gg[1], n[2] + 2 * gg[2]};
  const long long per = (long long)ex[0] * ex[1] * ex[2];
  const long long total = per * a.nfine;
  const int nn = L.ndim == 3 ? 27 : 9;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int fb = __ldg(a.fine + t / per);
    long long r = t % per;
    int c[3];
    c[0] = (int)(r % ex[0]) - gg[0];
    r /= ex[0];
    c[1] = (int)(r % ex[1]) - gg[1];
    c[2] = (int)(r / ex[1]) - gg[2];
    int o[3], nout = 0;
    for (int d = 0; d < 3; ++d) {
      o[d] = c[d] < 0 ? -1 : (c[d] >= n[d] ? 1 : 0);
      nout += o[d] != 0;
    }
    if (nout == 0 || (faces_only && nout != 1)) continue;
    const int e = L.ndim == 3 ? (o[2] + 1) * 9 + (o[1] + 1) * 3 + (o[0] + 1) : (o[1] + 1) * 3 + (o[0] + 1);
    if (__ldg(a.nbr + (long long)nn * fb + e) != GBH_NBR_COARSER) continue;
    const int parent = __ldg(a.parent + 4 * fb);
    int P[3], s[3];
    for (int d = 0; d < 3; ++d) {
      if (d < L.ndim) {
        const int hh = floor_div2(c[d]);
        P[d] = __ldg(a.parent + 4 * fb + 1 + d) + hh;
        s[d] = (c[d] - 2 * hh) == 0 ? -1 : 1;
      } else {
        P[d] = 0;
        s[d] = 0;
      }
    }
    const long long oc = coarse_offset(a, parent, P[0], P[1], P[2]);
    long long om[3], op[3];
    for (int d = 0; d < L.ndim; ++d) {
      int Pm[3] = {P[0], P[1], P[2]}, Pp[3] = {P[0], P[1], P[2]};
      Pm[d] -= 1;
      Pp[d] += 1;
      om[d] = coarse_offset(a, parent, Pm[0], Pm[1], Pm[2]);
      op[d] = coarse_offset(a, parent, Pp[0], Pp[1], Pp[2]);
    }
    double Uf[5];
    for (int v = 0; v < 5; ++v) {
      const long long vo = v * L.vstride;
      const double q0 = U[oc + vo];
      double val = q0;
      for (int d = 0; d < L.ndim; ++d) {
        const double h = mc_half_slope(U[om[d] + vo], q0, U[op[d] + vo]);   // sigma / 2
        val = __dadd_rn(val, __dmul_rn(0.5 * h, (double)s[d]));
      }
      Uf[v] = val;
      U[at(L, fb, v, c[0], c[1], c[2])] = val;
    }
    if (W) write_prim(W, L, at(L, fb, 0, c[0], c[1], c[2]), Uf, eo);
  }
}

// Prolongation into the 2-deep face slabs that the stage kernel reads, for a
// list of (fine block, face) pairs whose face neighbour lies on the coarser
// level: one thread per (pair, slab cell).
__global__ void prolong_faces_kernel(double* U, const AmrArgs a, double* W) {
  const Layout& L = a.lay;
  const Eos eo = reg_eos(a.eos, thread_zero(a.eos));
  const int N = L.nx;
  const int n2 = L.ndim == 3 ? N : 1;
  const long long per = 2LL * N * n2;
  const long long total = per * a.ncf_faces;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int2 ff = a.cf_faces[t / per];
    const int fb = ff.x, d = ff.y >> 1, side = ff.y & 1;
    const int r = (int)(t % per);
    const int depth = r % 2, t1 = (r / 2) % N, t2 = r / (2 * N);
    const int t1d = d == 0 ? 1 : 0, t2d = d == 2 ? 1 : 2;
    int c[3];
    c[d] = side ? N + depth : -1 - depth;
    c[t1d] = t1;
    c[t2d] = L.ndim == 3 ? t2 : 0;
    const int parent = __ldg(a.parent + 4 * fb);
    int P[3], sg[3];
    for (int e = 0; e < 3; ++e) {
      if (e < L.ndim) {
        const int hh = floor_div2(c[e]);
        P[e] = __ldg(a.parent + 4 * fb + 1 + e) + hh;
        sg[e] = (c[e] - 2 * hh) == 0 ? -1 : 1;
      } else {
        P[e] = 0;
        sg[e] = 0;
      }
    }
    const long long oc = coarse_offset(a, parent, P[0], P[1], P[2]);
    long long om[3], op[3];
    for (int e = 0; e < L.ndim; ++e) {
      int Pm[3] = {P[0], P[1], P[2]}, Pp[3] = {P[0], P[1], P[2]};
      Pm[e] -= 1;
      Pp[e] += 1;
      om[e] = coarse_offset(a, parent, Pm[0], Pm[1], Pm[2]);
      op[e] = coarse_offset(a, parent, Pp[0], Pp[1], Pp[2]);
    }
    double Uf[5];
    for (int v = 0; v < 5; ++v) {
      const long long vo = v * L.vstride;
      const double q0 = U[oc + vo];
      double val = q0;
      for (int e = 0; e < L.ndim; ++e) {
        const double h = mc_half_slope(U[om[e] + vo], q0, U[op[e] + vo]);
        val = __dadd_rn(val, __dmul_rn(0.5 * h, (double)sg[e]));
      }
      Uf[v] = val;
      U[at(L, fb, v, c[0], c[1], c[2])] = val;
    }
    if (W) write_prim(W, L, at(L, fb, 0, c[0], c[1], c[2]), Uf, eo);
  }
}

// Flux correction on the coarse side of the fine-region boundary.  One
// thread per (interface face, face cell).  A coarse cell next to several
// corrected faces of its block (a block bordering the refined region through
// two or three faces) is handled by the thread of the lowest of those faces,
// which adds every face's correction in the order x-, x+, y-, y+, z-, z+ (one
// writer per cell); the other threads leave it.  With smax_acc (the last
// correction of a step), the thread then forms the corrected cell's CFL
// signal-speed sum, which the stage kernel's epilogue left out, and adds it
// to the step's max.
__global__ void __launch_bounds__(kThreads) reflux_kernel(double* U, const AmrArgs a, const double* dt_dev,
                                                          double dt_val, double coef, unsigned long long* smax_acc,
                                                          double* W) {
  const Layout& L = a.lay;
  const long long zt = thread_zero(a.eos);
  const Eos e = reg_eos(a.eos, zt);   // FP64 constants in per-thread registers (gbh_fastmath.cuh)
  double smax = 0.0;
  const int N = L.nx;
  const int n2 = L.ndim == 3 ? N : 1;
  const int half = N / 2;
  const long long per = (long long)N * n2;
  const long long total = per * a.nreflux;
  const long long sstride = 5LL * N * n2;
  const double nfine = L.ndim == 3 ? 0.25 : 0.5;
  const int nfaces = 2 * L.ndim;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const RefluxEntry en = a.reflux[t / per];
    const int* of = a.reflux_of + 6LL * en.block;
    // the coarse cell next to this entry's face at face cell (t1, t2)
    const int r = (int)(t % per);
    int x[3];
    {
      const int d = en.face >> 1, side = en.face & 1;
      const int t1d = d == 0 ? 1 : 0, t2d = d == 2 ? 1 : 2;
      x[d] = side ? N - 1 : 0;
      x[t1d] = r % N;
      x[t2d] = L.ndim == 3 ? r / N : 0;
    }
    auto touches = [&](int f) {   // the cell lies next to face f of the block and f is corrected
      const int d = f >> 1;
      return __ldg(of + f) >= 0 && x[d] == ((f & 1) ? N - 1 : 0);
    };
    int owner = -1;
    for (int f = 0; f < nfaces && owner < 0; ++f)
      if (touches(f)) owner = f;
    if (owner != en.face) continue;
    // the time step of the block's problem (one entry unless batched)
    const double dt = dt_dev ? dt_dev[a.problem ? __ldg(a.problem + en.block) : 0] : dt_val;
    double Uc[5], U0[5];   // corrected, and as the stage left it
    for (int v = 0; v < 5; ++v) U0[v] = Uc[v] = U[at(L, en.block, v, x[0], x[1], x[2])];
    for (int f = 0; f < nfaces; ++f) {
      if (!touches(f)) continue;
      const RefluxEntry& eg = a.reflux[__ldg(of + f)];
      const int d = f >> 1, side = f & 1;
      const int t1d = d == 0 ? 1 : 0, t2d = d == 2 ? 1 : 2;
      const int t1 = x[t1d], t2 = L.ndim == 3 ? x[t2d] : 0;
      const int q1 = t1 / half, q2 = L.ndim == 3 ? t2 / half : 0;
      const int fs = eg.fine_slot[q1 + 2 * q2];
      const int f1 = 2 * (t1 % half), f2 = L.ndim == 3 ? 2 * (t2 % half) : 0;
      const double* Fc = a.flux_reg + (long long)eg.coarse_slot * sstride;
      const double* Ff = a.flux_reg + (long long)fs * sstride;
      const double idx = __ldg(a.inv_dx + 3 * en.block + d);
      for (int v = 0; v < 5; ++v) {
        double fsum = 0.0;
        for (int b2 = 0; b2 < (L.ndim == 3 ? 2 : 1); ++b2)
          for (int b1 = 0; b1 < 2; ++b1)
            fsum = __dadd_rn(fsum, Ff[GBH_IX((long long)fs * sstride + ((long long)v * n2 + f2 + b2) * N + f1 + b1,
                                             a.flux_reg_len) - (long long)fs * sstride]);
        const double fmean = __dmul_rn(fsum, nfine);
        const double fc = Fc[GBH_IX((long long)eg.coarse_slot * sstride + ((long long)v * n2 + t2) * N + t1,
                                    a.flux_reg_len) - (long long)eg.coarse_slot * sstride];
        const double corr = side ? __dsub_rn(fc, fmean) : __dsub_rn(fmean, fc);
        Uc[v] = __dadd_rn(Uc[v], __dmul_rn(__dmul_rn(__dmul_rn(coef, dt), corr), idx));
      }
    }
    for (int v = 0; v < 5; ++v) U[at(L, en.block, v, x[0], x[1], x[2])] = Uc[v];
    if (W) {
      // the stage's epilogue converted (and counted) the uncorrected value
      // for the next stage; replace it, and count the corrected value's floors
      // instead, as a conversion of this cell by the next stage would
      double W0[5], Wc[5];
      const long long o = at(L, en.block, 0, x[0], x[1], x[2]);
      const int h0 = cons_to_prim(U0, W0, e), h1 = cons_to_prim(Uc, Wc, e);
      for (int v = 0; v < 5; ++v) W[GBH_IX(o + v * L.vstride, (long long)L.nblocks * L.bstride)] = Wc[v];
      if (h1 != h0) atomicAdd(a.floor_count, (unsigned long long)(long long)(h1 - h0));
    }
    if (smax_acc) {
      double W[5], ir;
      cons_to_prim_ir(Uc, W, e, ir);
      const double sp = signal_speed_ir(W, ir, e, reg_const(__ldg(a.inv_dx + 3 * en.block), zt),
                                        reg_const(__ldg(a.inv_dx + 3 * en.block + 1), zt),
                                        reg_const(__ldg(a.inv_dx + 3 * en.block + 2), zt), L.ndim == 3);
      if (a.problem)
        atomicMax(smax_acc + __ldg(a.problem + en.block), (unsigned long long)__double_as_longlong(sp));
      else
        smax = max_nonneg(smax, sp);
    }
  }
  if (smax_acc && !a.problem) {
    // one accumulator: warp max, one atomic per warp (every lane of the warp
    // reaches this point: the block size is a multiple of 32)
    for (int o = 16; o > 0; o >>= 1) smax = max_nonneg(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(smax_acc, (unsigned long long)__double_as_longlong(smax));
  }
}

}  // namespace

GBH_CHECK_TAKE(check_take_amr)

cudaError_t launch_restrict(double* U, const AmrArgs& a, cudaStream_t s, double* W) {
  if (a.ncovered == 0) return cudaSuccess;
  restrict_kernel<<<grid_for((long long)a.ncovered * a.lay.nx * a.lay.ny * a.lay.nz), kThreads, 0, s>>>(U, a, W);
  return cudaGetLastError();
}

cudaError_t launch_prolong(double* U, const AmrArgs& a, int depth, bool faces_only, cudaStream_t s, double* W) {
  if (a.nfine == 0) return cudaSuccess;
  if (faces_only && depth == 2 && a.cf_faces) {
    const long long per = 2LL * a.lay.nx * (a.lay.ndim == 3 ? a.lay.nx : 1);
    prolong_faces_kernel<<<grid_for(per * a.ncf_faces), kThreads, 0, s>>>(U, a, W);
    return cudaGetLastError();
  }
  const Layout& L = a.lay;
  const long long per = (long long)(L.nx + 2 * depth) * (L.ny + 2 * depth) * (L.ndim == 3 ? L.nz + 2 * depth : 1);
  prolong_kernel<<<grid_for(per * a.nfine), kThreads, 0, s>>>(U, a, depth, faces_only ? 1 : 0, W);
  return cudaGetLastError();
}

cudaError_t launch_reflux(double* U, const AmrArgs& a, const double* dt_dev, double dt, double coef,
                          unsigned long long* smax_acc, cudaStream_t s, double* W) {
  if (a.nreflux == 0) return cudaSuccess;
  const long long per = (long long)a.lay.nx * (a.lay.ndim == 3 ? a.lay.nx : 1);
  reflux_kernel<<<grid_for(per * a.nreflux), kThreads, 0, s>>>(U, a, dt_dev, dt, coef, smax_acc, W);
  return cudaGetLastError();
}

}  // namespace gbh
