// gbh_aux.cu -- guard-cell fill, CFL time-step reduction, state check and the
// FP64 throughput probe.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbh_check.cuh"
#include "gbh_device.cuh"
#include "gbh_internal.h"

namespace gbh {
namespace {

constexpr int kThreads = 256;

// fill_guardcells (Sec. 4.2).  Work items are (block, padded z plane), a CTA
// each in turn; the CTA's threads take the plane's guard cells only: the whole
// plane in a z guard plane, else the g rows below and above the interior rows
// and the g-cell x guards of the interior rows (32-bit index arithmetic; rows
// are contiguous in x, so the copies are coalesced).  The value of a guard
// cell is resolved directly, without passes that depend on one another:
//  1. for each dimension d in which the cell lies outside the block and the
//     block's face in that direction is an outflow edge, its coordinate is
//     clamped to the nearest interior index (outflow is applied in the order
//     x, then y, then z; clamps in different dimensions commute);
//  2. the remaining outside dimensions give a lattice offset; the cell is the
//     interior cell of the neighbour block at that offset (full table).
// Every source is an interior cell, so the in-place fill has no read/write
// overlap.  An offset with no neighbour and no outflow face is left untouched.
__global__ void __launch_bounds__(kThreads) fill_kernel(const FillArgs a) {
  const Layout& L = a.lay;
  const int nn = L.ndim == 3 ? 27 : 9;
  const int n[3] = {L.nx, L.ny, L.nz};
  const int nitems = L.nblocks * L.nzp;
  const int full = 2 * L.g * L.nxp;            // cells of the 2g full rows of an interior plane
  const long long lim = (long long)L.nblocks * L.bstride - 4 * L.vstride;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int b = item / L.nzp, kk = item - b * L.nzp;
    const int cz = kk - L.gz;
    const bool zguard = cz < 0 || cz >= n[2];
    const int ncell = zguard ? L.nyp * L.nxp : full + L.ny * 2 * L.g;
    for (int q = threadIdx.x; q < ncell; q += blockDim.x) {
      int ii, jj;
      if (zguard) {
        jj = q / L.nxp;
        ii = q - jj * L.nxp;
      } else if (q < full) {
        const int r = q / L.nxp;
        jj = r < L.g ? r : L.ny + r;
        ii = q - r * L.nxp;
      } else {
        const int r = q - full, row = r / (2 * L.g), side = r - row * 2 * L.g;
        jj = L.g + row;
        ii = side < L.g ? side : L.nx + side;
      }
      int c[3] = {ii - L.g, jj - L.g, cz};
      int o[3];
      for (int d = 0; d < 3; ++d) o[d] = c[d] < 0 ? -1 : (c[d] >= n[d] ? 1 : 0);
      for (int d = 0; d < L.ndim; ++d) {
        if (o[d] == 0) continue;
        const int f = 2 * d + (o[d] > 0 ? 1 : 0);
        if (__ldg(a.face_nbr + 6 * b + f) == -1) {   // outflow face
          c[d] = o[d] < 0 ? 0 : n[d] - 1;
          o[d] = 0;
        }
      }
      int src = b;
      if (o[0] != 0 || o[1] != 0 || o[2] != 0) {
        const int e = L.ndim == 3 ? (o[2] + 1) * 9 + (o[1] + 1) * 3 + (o[0] + 1) : (o[1] + 1) * 3 + (o[0] + 1);
        src = __ldg(a.nbr + nn * b + e);
        if (src < 0) continue;
        for (int d = 0; d < 3; ++d) c[d] -= o[d] * n[d];
      }
      const long long so = GBH_IX(
          (long long)src * L.bstride + ((c[2] + L.gz) * L.nyp + (c[1] + L.g)) * L.nxp + (c[0] + L.g), lim);
      const long long dof = GBH_IX((long long)b * L.bstride + (kk * L.nyp + jj) * L.nxp + ii, lim);
#pragma unroll
      for (int v = 0; v < 5; ++v) a.U[dof + v * L.vstride] = a.U[so + v * L.vstride];
    }
  }
}

// CFL reduction: max over interior cells of the signal-speed sum, one
// atomicMax per CTA on the bit pattern (order-preserving for doubles >= 0).
__global__ void __launch_bounds__(kThreads) dt_reduce_kernel(const DtArgs a) {
  const Layout& L = a.lay;
  const long long per = (long long)L.nx * L.ny * L.nz;
  const long long total = per * (a.block_list ? a.nlist : L.nblocks);
  const bool d3 = L.ndim == 3;
  const long long zt = thread_zero(a.eos);
  const Eos e = reg_eos(a.eos, zt);   // FP64 constants in per-thread registers (gbh_fastmath.cuh)
  double smax = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = a.block_list ? __ldg(a.block_list + t / per) : (int)(t / per);
    long long r = t % per;
    const int i = (int)(r % L.nx);
    r /= L.nx;
    const int j = (int)(r % L.ny);
    const int k = (int)(r / L.ny);
    const long long o = GBH_IX((long long)b * L.bstride + ((long long)(k + L.gz) * L.nyp + (j + L.g)) * L.nxp + (i + L.g),
                               (long long)L.nblocks * L.bstride - 4 * L.vstride);
    double U[5], W[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = __ldg(a.U + o + v * L.vstride);
    double ir;
    cons_to_prim_ir(U, W, e, ir);
    const double s = signal_speed_ir(W, ir, e, reg_const(__ldg(a.inv_dx + 3 * b), zt),
                                     reg_const(__ldg(a.inv_dx + 3 * b + 1), zt),
                                     reg_const(__ldg(a.inv_dx + 3 * b + 2), zt), d3);
    smax = max_nonneg(smax, s);
  }
  __shared__ double red[kThreads / 32];
  const double m = block_max<kThreads>(smax, red);
  if (threadIdx.x == 0) atomicMax(a.smax_acc, (unsigned long long)__double_as_longlong(m));
}

// dt = cfl / smax per problem; also records it and clears the accumulator for
// its next use.
__global__ void dt_finalize_kernel(unsigned long long* acc, double cfl, double* dt_out, double* hist, int n) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const double smax = __longlong_as_double((long long)acc[p]);
    const double dt = cfl / smax;
    dt_out[p] = dt;
    if (hist) hist[p] = dt;
    acc[p] = 0ull;
  }
}

// Segmented CFL reduction for batched ensembles: one CTA per block at a time
// (grid-stride over blocks), one atomicMax into the block's problem slot.
__global__ void __launch_bounds__(kThreads) dt_reduce_blocks_kernel(const DtArgs a, const int* problem) {
  const Layout& L = a.lay;
  const int per = L.nx * L.ny * L.nz;
  const bool d3 = L.ndim == 3;
  const long long zt = thread_zero(a.eos);
  const Eos e = reg_eos(a.eos, zt);   // FP64 constants in per-thread registers (gbh_fastmath.cuh)
  __shared__ double red[kThreads / 32];
  const int nb = a.block_list ? a.nlist : L.nblocks;
  for (int s = blockIdx.x; s < nb; s += gridDim.x) {
    const int b = a.block_list ? __ldg(a.block_list + s) : s;
    double smax = 0.0;
    for (int t = threadIdx.x; t < per; t += blockDim.x) {
      const int i = t % L.nx, j = (t / L.nx) % L.ny, k = t / (L.nx * L.ny);
      const long long o =
          (long long)b * L.bstride + ((long long)(k + L.gz) * L.nyp + (j + L.g)) * L.nxp + (i + L.g);
      double U[5], W[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) U[v] = __ldg(a.U + o + v * L.vstride);
      double ir;
      cons_to_prim_ir(U, W, e, ir);
      smax = max_nonneg(smax, signal_speed_ir(W, ir, e, reg_const(__ldg(a.inv_dx + 3 * b), zt),
                                        reg_const(__ldg(a.inv_dx + 3 * b + 1), zt),
                                        reg_const(__ldg(a.inv_dx + 3 * b + 2), zt), d3));
    }
    const double m = block_max<kThreads>(smax, red);
    if (threadIdx.x == 0) atomicMax(a.smax_acc + __ldg(problem + b), (unsigned long long)__double_as_longlong(m));
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) check_kernel(const double* U, const Layout L, const Eos e,
                                                         unsigned long long* count) {
  const long long per = (long long)L.nx * L.ny * L.nz;
  const long long total = per * L.nblocks;
  unsigned long long bad = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / per);
    long long r = t - (long long)b * per;
    const int i = (int)(r % L.nx);
    r /= L.nx;
    const int j = (int)(r % L.ny);
    const int k = (int)(r / L.ny);
    const long long o = GBH_IX((long long)b * L.bstride + ((long long)(k + L.gz) * L.nyp + (j + L.g)) * L.nxp + (i + L.g),
                               (long long)L.nblocks * L.bstride - 4 * L.vstride);
    double u[5];
    bool finite = true;
    for (int v = 0; v < 5; ++v) {
      u[v] = U[o + v * L.vstride];
      finite = finite && isfinite(u[v]);
    }
    const double p = e.gm1 * (u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0]);
    if (!finite || !(u[0] > e.small_rho) || !(p > e.small_p)) ++bad;
  }
  if (bad) atomicAdd(count, bad);
}

// Interior cells between the padded and the interior-only layouts of the nb
// blocks that start at `padded` and `interior`: one thread per cell,
// consecutive threads along x, so both sides read and write whole rows of nx
// doubles (coalesced).  The launcher keeps 5 nx ny nz nb below 2^30, so the
// cell index and its decomposition are 32-bit.
__global__ void __launch_bounds__(kThreads) interior_copy_kernel(double* padded, double* interior, const Layout L,
                                                                 int nb, bool to_padded) {
  const unsigned per = (unsigned)(L.nx * L.ny * L.nz), cells = 5u * per, total = cells * (unsigned)nb;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const unsigned bl = t / cells;
    unsigned r = t - bl * cells;
    const unsigned v = r / per;
    r -= v * per;
    const unsigned i = r % (unsigned)L.nx;
    r /= (unsigned)L.nx;
    const unsigned j = r % (unsigned)L.ny, k = r / (unsigned)L.ny;
    const long long o = (long long)bl * L.bstride + (long long)v * L.vstride +
                        ((long long)(k + L.gz) * L.nyp + (j + L.g)) * L.nxp + (i + L.g);
    if (to_padded)
      padded[GBH_IX(o, (long long)nb * L.bstride)] = interior[GBH_IX(t, total)];
    else
      interior[GBH_IX(t, total)] = padded[GBH_IX(o, (long long)nb * L.bstride)];
  }
}

// 8 independent FMA chains per thread; the multiplier and addend keep the
// values bounded (fixed point 1.0).  Only the first `lanes` lanes of each
// warp run the chains (to measure how the FP64 pipe charges partial warps).
// FP64 pipe probe: 8 independent chains per thread, run by the first `lanes`
// lanes of each warp.  FORM 0: x = fma(x, m, c) with m, c compile-time
// constants (constant-bank operands); 1: the same with m, c in per-thread
// registers (their bit patterns OR-ed with a run-time zero that depends on the
// thread index, so the compiler can neither fold them into constants nor keep
// them in warp-uniform registers); 2: x = x + c (DADD); 3: x = x * m (DMUL),
// c and m in per-thread registers; 4: as 1 with m, c warp-uniform (OR-ed with
// the run-time zero alone).
template <int FORM>
__global__ void fp64_probe_kernel(int iters, int lanes, long long zero, double* out) {
  const long long z = FORM == 4 ? zero : (zero & (long long)threadIdx.x);
  const double m = FORM == 0 ? 0.999999999 : __longlong_as_double(__double_as_longlong(0.999999999) | z);
  const double c = FORM == 0 ? 1e-9 : __longlong_as_double(__double_as_longlong(1e-9) | z);
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * threadIdx.x + 0.1 * k;
  const int n = (int)(threadIdx.x & 31) < lanes ? iters : 0;
  for (int i = 0; i < n; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = FORM == 2 ? x[k] + c : FORM == 3 ? x[k] * m : fma(x[k], m, c);
  }
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) sum += x[k];
  out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = sum;
}

// FP64 instruction count of one call of each arithmetic building block of the
// stage kernel, in the form the kernel uses (register constants, register-FMA
// adds and multiplies).  Each thread makes `iters` dependent calls on the 10
// doubles io[10 t .. 10 t + 9]; the next call's inputs take the low bit of
// the XOR of every output of the last one into their last mantissa bits with
// an integer XOR, so no part of a call can be hoisted or folded and the chain
// adds no FP64 work: ncu's FP64 instruction counters of a launch divided by
// threads x iters are the instructions of one call.
template <int FN>
__global__ void op_count_kernel(int iters, const Eos e0, double* io) {
  const long long zt = thread_zero(e0);
  const Eos e = reg_eos(e0, zt);
  const Rk& rk = e.k;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double x[10];
#pragma unroll
  for (int v = 0; v < 10; ++v) x[v] = io[10 * t + v];
  const double c1 = reg_const(0.3, zt), c2 = reg_const(0.2, zt), c3 = reg_const(0.1, zt);
  long long fb = 0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int v = 0; v < 10; ++v) x[v] = bitsd(dbits(x[v]) ^ (fb & 1));
    fb = 0;
    if constexpr (FN == 0) {          // cons -> prim of one cell
      double W[5];
      fb ^= cons_to_prim(x, W, e);
#pragma unroll
      for (int v = 0; v < 5; ++v) fb ^= dbits(W[v]);
    } else if constexpr (FN == 1) {   // one x/y slope work item (three cells) of one variable
      const double d0 = sub(x[1], x[0], rk), d1 = sub(x[2], x[1], rk), d2 = sub(x[3], x[2], rk);
      const double d3 = sub(x[4], x[3], rk);
      const double t0 = mc_half_slope_d(d0, d1, rk), t1 = mc_half_slope_d(d1, d2, rk);
      const double t2 = mc_half_slope_d(d2, d3, rk);
      const double q[6] = {sub(x[1], t0, rk), add(x[1], t0, rk), sub(x[2], t1, rk), add(x[2], t1, rk),
                           sub(x[3], t2, rk), add(x[3], t2, rk)};
#pragma unroll
      for (int v = 0; v < 6; ++v) fb ^= dbits(q[v]);
    } else if constexpr (FN == 2) {   // one HLLC face
      double F[5];
      hllc_flux(x, x + 5, e, F);
#pragma unroll
      for (int v = 0; v < 5; ++v) fb ^= dbits(F[v]);
    } else if constexpr (FN == 3) {   // the 3-D flux-difference update of one variable
      double r = fma(-c1, sub(x[1], x[2], rk), x[0]);
      r = fma(-c2, sub(x[3], x[4], rk), r);
      r = fma(-c3, sub(x[5], x[6], rk), r);
      fb ^= dbits(r);
    } else if constexpr (FN == 4) {   // the second-stage combine of one variable
      fb ^= dbits(half_any(add(x[1], x[0], rk)));
    } else if constexpr (FN == 5) {   // CFL epilogue of one cell: cons -> prim and 3-D signal speed
      double W[5], ir;
      cons_to_prim_ir(x, W, e, ir);
      fb ^= dbits(signal_speed_ir(W, ir, e, c1, c2, c3, true));
    } else if constexpr (FN == 6) {   // z march: the next z slope and face states of one variable
      const double dn = sub(x[1], x[0], rk);
      const double tz = mc_half_slope_d(x[2], dn, rk);
      fb ^= dbits(sub(x[0], tz, rk)) ^ dbits(add(x[0], tz, rk)) ^ dbits(dn);
    } else {                           // the two face states of a block-boundary face, one variable
      const double d0 = sub(x[1], x[0], rk), d1 = sub(x[2], x[1], rk), d2 = sub(x[3], x[2], rk);
      fb ^= dbits(add(x[1], mc_half_slope_d(d0, d1, rk), rk)) ^ dbits(sub(x[2], mc_half_slope_d(d1, d2, rk), rk));
    }
  }
#pragma unroll
  for (int v = 0; v < 10; ++v) io[10 * t + v] = bitsd(dbits(x[v]) ^ (fb & 1));
}

// Self-test of the refined reciprocal / square roots: out[6][n] =
// rcp_nr, 1.0/x, rsqrt_nr, 1.0/sqrt(x), sqrt_nr, sqrt(x).
__global__ void fastmath_selftest_kernel(const double* x, double* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    out[i] = rcp_nr(v);
    out[n + i] = 1.0 / v;
    out[2 * n + i] = rsqrt_nr(v);
    out[3 * n + i] = 1.0 / sqrt(v);
    out[4 * n + i] = sqrt_nr(v);
    out[5 * n + i] = sqrt(v);
  }
}

// Self-test of the integer-pipe helpers the stage kernel relies on:
// out[6][n] = half_any(x), quarter_any(x), mc_half_slope_d(x, y) with the
// constants in per-thread registers, ge0(x) (1 or 0), min_d(x, y), max_d(x, y).
__global__ void bits_selftest_kernel(const double* x, const double* y, double* out, long long n, long long zero) {
  const long long z = zero & (long long)threadIdx.x;
  const Rk k{reg_const(1.0, z), reg_const(-0.0, z)};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double a = x[i], b = y[i];
    out[i] = half_any(a);
    out[n + i] = quarter_any(a);
    out[2 * n + i] = mc_half_slope_d(a, b, k);
    out[3 * n + i] = ge0(a) ? 1.0 : 0.0;
    out[4 * n + i] = min_d(a, b);
    out[5 * n + i] = max_d(a, b);
  }
}

#ifdef GBH_CHECK
// One index past a 4-element buffer: the check counts it and redirects the
// store to element 0 (the access stays inside the buffer).
__global__ void check_selftest_kernel(double* buf) {
  const long long i = 4;
  buf[GBH_IX(i, 4)] = 1.0;
}
#endif

int grid_for(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  if (g > 152LL * 16) g = 152LL * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

GBH_CHECK_TAKE(check_take_aux)

long long check_selftest() {
#ifdef GBH_CHECK
  double* buf = nullptr;
  if (cudaMalloc(&buf, 4 * sizeof(double)) != cudaSuccess) return -1;
  const long long before = check_take_aux();
  check_selftest_kernel<<<1, 1>>>(buf);
  const cudaError_t e = cudaDeviceSynchronize();
  cudaFree(buf);
  if (e != cudaSuccess || before < 0) return -1;
  return check_take_aux();
#else
  return -1;
#endif
}

cudaError_t launch_fill(const FillArgs& a, cudaStream_t s) {
  const long long items = (long long)a.lay.nblocks * a.lay.nzp;
  fill_kernel<<<(int)(items < 152LL * 16 ? items : 152LL * 16), kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_interior_copy(double* padded, double* interior, const Layout& L, int b0, int nb,
                                 bool to_padded, cudaStream_t s) {
  const long long cells = 5LL * L.nx * L.ny * L.nz;
  const long long per_launch = (1LL << 30) / cells > 0 ? (1LL << 30) / cells : 1;
  for (long long b = b0; b < (long long)b0 + nb; b += per_launch) {
    const int n = (int)((long long)b0 + nb - b < per_launch ? (long long)b0 + nb - b : per_launch);
    interior_copy_kernel<<<grid_for(cells * n, kThreads), kThreads, 0, s>>>(padded + b * L.bstride,
                                                                           interior + b * cells, L, n, to_padded);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_dt_reduce(const DtArgs& a, cudaStream_t s) {
  const long long work = (long long)a.lay.nblocks * a.lay.nx * a.lay.ny * a.lay.nz;
  dt_reduce_kernel<<<grid_for(work, kThreads), kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dt_finalize(unsigned long long* acc, double cfl, double* dt_out, double* hist,
                               cudaStream_t s, int n) {
  dt_finalize_kernel<<<(n + 255) / 256, n < 256 ? n : 256, 0, s>>>(acc, cfl, dt_out, hist, n);
  return cudaGetLastError();
}

cudaError_t launch_dt_reduce_blocks(const DtArgs& a, const int* problem, cudaStream_t s) {
  const int nb = a.block_list ? a.nlist : a.lay.nblocks;
  dt_reduce_blocks_kernel<<<nb < 152 * 8 ? nb : 152 * 8, kThreads, 0, s>>>(a, problem);
  return cudaGetLastError();
}

cudaError_t launch_check(const double* U, Layout lay, Eos eos, unsigned long long* count,
                         cudaStream_t s) {
  const long long work = (long long)lay.nblocks * lay.nx * lay.ny * lay.nz;
  check_kernel<<<grid_for(work, kThreads), kThreads, 0, s>>>(U, lay, eos, count);
  return cudaGetLastError();
}

cudaError_t launch_bits_selftest(const double* x, const double* y, double* out, long long n, cudaStream_t s) {
  bits_selftest_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(x, y, out, n, 0);
  return cudaGetLastError();
}

cudaError_t launch_fastmath_selftest(const double* x, double* out, long long n, cudaStream_t s) {
  fastmath_selftest_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(x, out, n);
  return cudaGetLastError();
}

cudaError_t launch_op_count(int fn, int blocks, int threads, int iters, const Eos& e, double* io, cudaStream_t s) {
  switch (fn) {
    case 0: op_count_kernel<0><<<blocks, threads, 0, s>>>(iters, e, io); break;
    case 1: op_count_kernel<1><<<blocks, threads, 0, s>>>(iters, e, io); break;
    case 2: op_count_kernel<2><<<blocks, threads, 0, s>>>(iters, e, io); break;
    case 3: op_count_kernel<3><<<blocks, threads, 0, s>>>(iters, e, io); break;
    case 4: op_count_kernel<4><<<blocks, threads, 0, s>>>(iters, e, io); break;
    case 5: op_count_kernel<5><<<blocks, threads, 0, s>>>(iters, e, io); break;
    case 6: op_count_kernel<6><<<blocks, threads, 0, s>>>(iters, e, io); break;
    case 7: op_count_kernel<7><<<blocks, threads, 0, s>>>(iters, e, io); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fp64_probe(int blocks, int threads, int iters, int lanes, int form, double* out, cudaStream_t s) {
  switch (form) {
    case 0: fp64_probe_kernel<0><<<blocks, threads, 0, s>>>(iters, lanes, 0, out); break;
    case 1: fp64_probe_kernel<1><<<blocks, threads, 0, s>>>(iters, lanes, 0, out); break;
    case 2: fp64_probe_kernel<2><<<blocks, threads, 0, s>>>(iters, lanes, 0, out); break;
    case 3: fp64_probe_kernel<3><<<blocks, threads, 0, s>>>(iters, lanes, 0, out); break;
    case 4: fp64_probe_kernel<4><<<blocks, threads, 0, s>>>(iters, lanes, 0, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace gbh
