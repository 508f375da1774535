// gbh_adjoint.cu -- hand-written adjoint of the RK stage (vector-Jacobian
// products), for gradients of a final-state loss with respect to the initial
// fields.
//
// The forward stage is Uout = a Un + b (Uin + dt L(Uin)) with L the
// intra-stage calculations (calcEos, calcLims, calcFlux, updSoln; Sec. 4.2,
// Alg. "Intra stage calculations for Spark").  The adjoint needs
// J_L(U)^T mu.  Conventions: dt is held fixed (treated as a constant of the
// step), and every branch of the forward arithmetic keeps the decision it took
// in the forward evaluation (floors, the MC limiter case, the HLLC side and
// whether the wave fan straddles the face, the min / max of the wave-speed
// bounds).
//
// Structure of one VJP (no atomics; results are deterministic):
//  1. face pass, one thread per face of every block and dimension (one
//     launch): recompute the primitives of the face's 4 stencil positions
//     (halo gathered as in the forward kernel), the two MC slopes (with their
//     branch) and the HLLC flux; the flux adjoint of face k is
//     scale (M_k - M_{k-1}) / dx using only this block's own cells (M outside
//     the block is 0), so the two blocks sharing a face each contribute their
//     half of the linear map.  The reverse of HLLC, the face states and the
//     slopes gives the face's contribution to the adjoint of the primitives of
//     its 4 positions, stored in the face's own slots.
//  2. cell pass, one thread per interior cell: sums, in a fixed order, the
//     slots that refer to the cell -- of its own block's faces, of the
//     neighbours' faces whose halo copied it, and of its own halo positions at
//     an outflow edge (the adjoint of the fused guard fill) -- then applies
//     the reverse of the EOS: out = cA A + cB B + J^T(scale M).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbh_check.cuh"
#include "gbh_device.cuh"
#include "gbh_gather.cuh"
#include "gbh_internal.h"

namespace gbh {
namespace {

// ---- reverse of the pointwise pieces ---------------------------------------

// mc_half_slope with the branch it takes: 0 zero, 1 central, 2 |dm|, 3 |dp|.
__device__ __forceinline__ double mc_half_slope_br(double qm, double q0, double qp, int& br) {
  const double dm = q0 - qm;
  const double dp = qp - q0;
  const double s4 = 0.25 * (dm + dp);
  const unsigned long long am = mag_key(dm), ap = mag_key(dp), as = mag_key(s4);
  const unsigned long long m1 = am < ap ? am : ap;
  const bool central = as < m1;
  const unsigned long long m = central ? as : m1;
  const bool same = ((dbits(dm) ^ dbits(dp)) >= 0) && am != 0 && ap != 0;
  br = !same ? 0 : (central ? 1 : (am < ap ? 2 : 3));
  return bitsd(same ? (long long)((m >> 1) | sign_bit(dp)) : 0LL);
}

__device__ __forceinline__ void mc_half_slope_vjp(int br, double bh, double& bqm, double& bq0, double& bqp) {
  const double bdm = br == 1 ? 0.25 * bh : (br == 2 ? bh : 0.0);
  const double bdp = br == 1 ? 0.25 * bh : (br == 3 ? bh : 0.0);
  bqm -= bdm;
  bq0 += bdm - bdp;
  bqp += bdp;
}

// cons_to_prim reporting which floors applied.
__device__ __forceinline__ void cons_to_prim_flags(const double U[5], double W[5], const Eos& e, bool& fr,
                                                   bool& fp) {
  double rho = U[0];
  fr = less_d(rho, e.small_rho);
  if (fr) rho = e.small_rho;
  const double ir = rcp_nr(rho);
  const double u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
  const double m2 = fma(U[3], w, fma(U[2], v, U[1] * u));
  double p = e.gm1 * fma(-0.5, m2, U[4]);
  fp = less_d(p, e.small_p);
  if (fp) p = e.small_p;
  W[0] = rho; W[1] = u; W[2] = v; W[3] = w; W[4] = p;
}

// bU = (dW/dU)^T bW for W = cons_to_prim(U); floored components are constants.
__device__ __forceinline__ void prim_vjp(const double W[5], bool fr, bool fp, const Eos& e, const double bW[5],
                                         double bU[5]) {
  const double ir = rcp_nr(W[0]);
  const double u = W[1], v = W[2], w = W[3];
  const double bp = fp ? 0.0 : bW[4] * e.gm1;
  bU[4] = bp;
  bU[1] = ir * bW[1] - bp * u;
  bU[2] = ir * bW[2] - bp * v;
  bU[3] = ir * bW[3] - bp * w;
  bU[0] = fr ? 0.0 : bW[0] - ir * (u * bW[1] + v * bW[2] + w * bW[3]) + bp * 0.5 * (u * u + v * v + w * w);
}

// Reverse of the HLLC flux of hllc_flux (gbh_device.cuh).  The forward
// intermediates are recomputed in Toro's form (Roe-averaged H~ and transverse
// velocities, both sides' E + p), which equals hllc_flux's arrangement
// algebraically, then (dF/dW)^T bF is accumulated.
__device__ void hllc_flux_vjp(const double WL[5], const double WR[5], const Eos& e, const double bF[5],
                              double bWL[5], double bWR[5]) {
  const double rL = WL[0], uL = WL[1], vL = WL[2], wL = WL[3], pL = WL[4];
  const double rR = WR[0], uR = WR[1], vR = WR[2], wR = WR[3], pR = WR[4];
  // ---- forward (as hllc_flux) ----
  const double aL = rsqrt_nr(rL), aR = rsqrt_nr(rR);
  const double sL = rL * aL, sR = rR * aR;
  const double iL = aL * aL, iR = aR * aR;
  const double kL = fma(wL, wL, fma(vL, vL, uL * uL));
  const double kR = fma(wR, wR, fma(vR, vR, uR * uR));
  const double hL = fma(0.5 * rL, kL, e.g_gm1 * pL);
  const double hR = fma(0.5 * rR, kR, e.g_gm1 * pR);
  const double zL = e.gamma * pL * iL, zR = e.gamma * pR * iR;
  const double qL = rsqrt_nr(zL), qR = rsqrt_nr(zR);   // 1/c (kept for the reverse)
  const double cL = zL * qL, cR = zR * qR;
  const double w = rcp_nr(sL + sR);
  const double wl = sL * w, wr = sR * w;
  const double ut = fma(wl, uL, wr * uR);
  const double vt = fma(wl, vL, wr * vR);
  const double wt = fma(wl, wL, wr * wR);
  const double T = fma(hL, aL, hR * aR);
  const double Ht = T * w;
  const double kt = fma(wt, wt, fma(vt, vt, ut * ut));
  const double zc = e.gm1 * fma(-0.5, kt, Ht);
  const double qc = rsqrt_nr(zc);
  const double ct = zc * qc;
  const double l1 = uL - cL, l2 = ut - ct, r1 = uR + cR, r2 = ut + ct;
  const bool selL1 = !(order_key(l2) < order_key(l1));   // SL = l1
  const bool selR1 = !(order_key(r1) < order_key(r2));   // SR = r1
  const double SL = selL1 ? l1 : l2, SR = selR1 ? r1 : r2;
  const double mL = rL * (SL - uL), mR = rR * (SR - uR);
  const double rd = rcp_nr(mL - mR);
  const double Ss = fma(-mR, uR, fma(mL, uL, pR - pL)) * rd;
  const bool left = ge0(Ss);
  const double rK = sel(left, rL, rR), uK = sel(left, uL, uR), vK = sel(left, vL, vR);
  const double wK = sel(left, wL, wR), pK = sel(left, pL, pR), hK = sel(left, hL, hR);
  const double SK = sel(left, SL, SR), mK = sel(left, mL, mR);
  const bool fan = left ? lt0(SL) : gt0(SR);
  const double rr = rcp_nr(SK - Ss);
  const double delta = (Ss - uK) * rr;
  const double g = sel(fan, SK, 0.0) * delta;
  const double mass = rK * uK;
  const double F0 = fma(g, rK, mass);
  // ---- reverse ----
  const double bF0 = bF[0] + bF[2] * vK + bF[3] * wK;
  const double bvK = bF[2] * F0, bwK = bF[3] * F0;
  double buK = bF[4] * hK;
  double bhK = bF[4] * (uK + g);
  double bg = bF[4] * fma(mK, Ss, hK);
  const double bmK = bF[4] * g * Ss;
  double bSs = bF[4] * g * mK;
  double bmass = bF[1] * uK;
  buK += bF[1] * mass;
  const double bpK = bF[1];
  bg += bF[1] * rK * SK;
  double brK = bF[1] * g * SK;
  double bSK = bF[1] * g * rK;
  bmass += bF0;
  bg += bF0 * rK;
  brK += bF0 * g;
  brK += bmass * uK;
  buK += bmass * rK;
  const double bdelta = fan ? bg * SK : 0.0;
  if (fan) bSK += bg * delta;
  bSs += bdelta * (SK - uK) * rr * rr;
  buK -= bdelta * rr;
  bSK -= bdelta * delta * rr;
  double brL = 0, buL = 0, bvL = 0, bwL = 0, bpL = 0, bhL = 0, bSL = 0, bmL = 0;
  double brR = 0, buR = 0, bvR = 0, bwR = 0, bpR = 0, bhR = 0, bSR = 0, bmR = 0;
  if (left) {
    brL = brK; buL = buK; bvL = bvK; bwL = bwK; bpL = bpK; bhL = bhK; bSL = bSK; bmL = bmK;
  } else {
    brR = brK; buR = buK; bvR = bvK; bwR = bwK; bpR = bpK; bhR = bhK; bSR = bSK; bmR = bmK;
  }
  const double bnum = bSs * rd, bden = -bSs * Ss * rd;
  bpR += bnum;
  bpL -= bnum;
  bmL += bnum * uL + bden;
  buL += bnum * mL;
  bmR -= bnum * uR + bden;
  buR -= bnum * mR;
  brL += bmL * (SL - uL);
  bSL += bmL * rL;
  buL -= bmL * rL;
  brR += bmR * (SR - uR);
  bSR += bmR * rR;
  buR -= bmR * rR;
  double but = 0, bct = 0, bcL = 0, bcR = 0;
  if (selL1) { buL += bSL; bcL -= bSL; } else { but += bSL; bct -= bSL; }
  if (selR1) { buR += bSR; bcR += bSR; } else { but += bSR; bct += bSR; }
  const double bzc = bct * 0.5 * qc;
  const double bHt = bzc * e.gm1, bkt = -0.5 * bzc * e.gm1;
  but += 2.0 * ut * bkt;
  const double bvt = 2.0 * vt * bkt, bwt = 2.0 * wt * bkt;
  const double bT = bHt * w;
  double bw = bHt * T;
  bhL += bT * aL;
  bhR += bT * aR;
  double baL = bT * hL, baR = bT * hR;
  const double bwl = but * uL + bvt * vL + bwt * wL;
  const double bwr = but * uR + bvt * vR + bwt * wR;
  buL += but * wl; bvL += bvt * wl; bwL += bwt * wl;
  buR += but * wr; bvR += bvt * wr; bwR += bwt * wr;
  double bsL = bwl * w, bsR = bwr * w;
  bw += bwl * sL + bwr * sR;
  const double bss = -bw * w * w;
  bsL += bss;
  bsR += bss;
  const double bzL = bcL * 0.5 * qL, bzR = bcR * 0.5 * qR;
  bpL += bzL * e.gamma * iL;
  bpR += bzR * e.gamma * iR;
  const double biL = bzL * e.gamma * pL, biR = bzR * e.gamma * pR;
  brL += bhL * 0.5 * kL;
  brR += bhR * 0.5 * kR;
  const double bkL = bhL * 0.5 * rL, bkR = bhR * 0.5 * rR;
  bpL += bhL * e.g_gm1;
  bpR += bhR * e.g_gm1;
  buL += 2.0 * uL * bkL; bvL += 2.0 * vL * bkL; bwL += 2.0 * wL * bkL;
  buR += 2.0 * uR * bkR; bvR += 2.0 * vR * bkR; bwR += 2.0 * wR * bkR;
  baL += 2.0 * aL * biL + bsL * rL;
  baR += 2.0 * aR * biR + bsR * rR;
  brL += bsL * aL;
  brR += bsR * aR;
  brL += baL * (-0.5 * aL * iL);
  brR += baR * (-0.5 * aR * iR);
  bWL[0] = brL; bWL[1] = buL; bWL[2] = bvL; bWL[3] = bwL; bWL[4] = bpL;
  bWR[0] = brR; bWR[1] = buR; bWR[2] = bvR; bWR[3] = bwR; bWR[4] = bpR;
}

// ---- the face pass: one thread per face -------------------------------------
//
// Face k (k = 0..n_d) of a pencil along dimension d reads the primitives of
// the halo-extended positions k-2..k+1.  Its contribution to the adjoint of
// those four positions is stored in its own slots C[d][b][pencil][k][s][v]
// (s = position - (k-2)); the cell pass sums the slots that refer to a cell.

struct FaceGeom {
  long long total;     // doubles in the slot buffer (checked build)
  long long base[3];   // offset of each dimension's slots in the buffer
  int n[3];            // pencil length per dimension
  int n1[3], n2[3];    // transverse extents per dimension
};

__device__ __forceinline__ long long slot_index(const FaceGeom& G, int d, int b, int pen, int k, int s) {
  const long long npen = (long long)G.n1[d] * G.n2[d];
  return GBH_IX(G.base[d] + ((((long long)b * npen + pen) * (G.n[d] + 1) + k) * 4 + s) * 5, G.total - 4);
}

__device__ __forceinline__ void pencil_to_cell(int d, int pos, int p1, int p2, int& i, int& j, int& k) {
  if (d == 0) { i = pos; j = p1; k = p2; }
  else if (d == 1) { i = p1; j = pos; k = p2; }
  else { i = p1; j = p2; k = pos; }
}

__device__ __forceinline__ long long own_offset(const Layout& L, int b, int i, int j, int k) {
  return GBH_IX((long long)b * L.bstride + ((long long)(k + L.gz) * L.nyp + (j + L.g)) * L.nxp + (i + L.g),
                (long long)L.nblocks * L.bstride - 4 * L.vstride);
}

template <int N, int d>
__device__ __forceinline__ void face_work(const StageArgs& a, const FaceGeom& G, const double* __restrict__ Wp,
                                          const double* __restrict__ M, double scale, double* __restrict__ C,
                                          long long t) {
  const Layout& L = a.lay;
  const int nf = G.n[d] + 1;
  const int k = (int)(t % nf);
  long long r = t / nf;
  const long long npen = (long long)G.n1[d] * G.n2[d];
  const int pen = (int)(r % npen);
  const int b = (int)(r / npen);
  const int p1 = pen % G.n1[d], p2 = pen / G.n1[d];
  const int nd = G.n[d];
  const Eos& e = a.eos;
  const double sc = scale * __ldg(a.inv_dx + 3 * b + d);
  const int rot[5] = {0, 1 + d, d == 0 ? 2 : 1, d == 2 ? 2 : 3, 4};

  double W[4][5];
  int ci, cj, ck;
  for (int s = 0; s < 4; ++s) {
    // primitives of the stencil position (the halo gathered as in the stage kernel)
    pencil_to_cell(d, k - 2 + s, p1, p2, ci, cj, ck);
    const long long o = cell_offset<N>(a, b, ci, cj, ck);
#pragma unroll
    for (int v = 0; v < 5; ++v) W[s][v] = __ldg(Wp + o + v * L.vstride);
  }
  double h0[5], h1[5];
  int b0[5], b1[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    h0[v] = mc_half_slope_br(W[0][v], W[1][v], W[2][v], b0[v]);   // slope of position k-1
    h1[v] = mc_half_slope_br(W[1][v], W[2][v], W[3][v], b1[v]);   // slope of position k
  }
  double bF[5];
  {
    double mk[5] = {0, 0, 0, 0, 0}, mk1[5] = {0, 0, 0, 0, 0};
    if (k < nd) {
      pencil_to_cell(d, k, p1, p2, ci, cj, ck);
      const long long o = own_offset(L, b, ci, cj, ck);
      for (int v = 0; v < 5; ++v) mk[v] = __ldg(M + o + v * L.vstride);
    }
    if (k > 0) {
      pencil_to_cell(d, k - 1, p1, p2, ci, cj, ck);
      const long long o = own_offset(L, b, ci, cj, ck);
      for (int v = 0; v < 5; ++v) mk1[v] = __ldg(M + o + v * L.vstride);
    }
    for (int v = 0; v < 5; ++v) bF[v] = sc * (mk[v] - mk1[v]);
  }
  double wl[5], wr[5], bFr[5], bwl[5], bwr[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    wl[q] = W[1][rot[q]] + h0[rot[q]];
    wr[q] = W[2][rot[q]] - h1[rot[q]];
    bFr[q] = bF[rot[q]];
  }
  hllc_flux_vjp(wl, wr, e, bFr, bwl, bwr);
  double Cs[4][5];
#pragma unroll
  for (int v = 0; v < 5; ++v) Cs[0][v] = Cs[1][v] = Cs[2][v] = Cs[3][v] = 0.0;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int v = rot[q];
    Cs[1][v] += bwl[q];
    Cs[2][v] += bwr[q];
    mc_half_slope_vjp(b0[v], bwl[q], Cs[0][v], Cs[1][v], Cs[2][v]);
    mc_half_slope_vjp(b1[v], -bwr[q], Cs[1][v], Cs[2][v], Cs[3][v]);
  }
  double* out = C + slot_index(G, d, b, pen, k, 0);
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int v = 0; v < 5; ++v) out[s * 5 + v] = Cs[s][v];
}

template <int N>
__global__ void __launch_bounds__(128) vjp_face_kernel(const StageArgs a, const FaceGeom G,
                                                      const double* __restrict__ Wp, const double* __restrict__ M,
                                                      double scale, double* __restrict__ C) {
  const Layout& L = a.lay;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (int d = 0; d < L.ndim; ++d) {
    const long long count = (long long)L.nblocks * G.n1[d] * G.n2[d] * (G.n[d] + 1);
    if (t < count) {
      if (d == 0) face_work<N, 0>(a, G, Wp, M, scale, C, t);
      else if (d == 1) face_work<N, 1>(a, G, Wp, M, scale, C, t);
      else face_work<N, 2>(a, G, Wp, M, scale, C, t);
      return;
    }
    t -= count;
  }
}

// Primitives of every interior cell of Uin (cons_to_prim, floors as in the
// stage kernel) into Wp, state layout; the face pass gathers them.
__global__ void vjp_prim_kernel(const StageArgs a, double* __restrict__ Wp) {
  const Layout& L = a.lay;
  const long long per = (long long)L.nx * L.ny * L.nz;
  const long long total = per * L.nblocks;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / per);
    long long r = t % per;
    const int i = (int)(r % L.nx);
    r /= L.nx;
    const int j = (int)(r % L.ny);
    const int k = (int)(r / L.ny);
    const long long o = own_offset(L, b, i, j, k);
    double U[5], W[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = __ldg(a.Uin + o + v * L.vstride);
    cons_to_prim(U, W, a.eos);
#pragma unroll
    for (int v = 0; v < 5; ++v) Wp[o + v * L.vstride] = W[v];
  }
}

// Sum of the slots of block b, dimension d, pencil pen that refer to the
// halo-extended position q (-2..n_d+1), in increasing face order.
__device__ __forceinline__ void add_position(const FaceGeom& G, const double* __restrict__ C, int d, int b, int pen,
                                             int q, double acc[5]) {
  const int nd = G.n[d];
  for (int k = q - 1; k <= q + 2; ++k) {
    if (k < 0 || k > nd) continue;
    const double* c = C + slot_index(G, d, b, pen, k, q + 2 - k);
    for (int v = 0; v < 5; ++v) acc[v] += c[v];
  }
}

// ---- the cell pass ------------------------------------------------------------

__global__ void vjp_cell_kernel(const StageArgs a, const FaceGeom G, const double* __restrict__ C, const double* A,
                                double cA, const double* B, double cB, double* out) {
  const Layout& L = a.lay;
  const long long per = (long long)L.nx * L.ny * L.nz;
  const long long total = per * L.nblocks;
  const int n[3] = {L.nx, L.ny, L.nz};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / per);
    long long r = t % per;
    const int i = (int)(r % L.nx);
    r /= L.nx;
    const int j = (int)(r % L.ny);
    const int k = (int)(r / L.ny);
    const int c[3] = {i, j, k};
    double bW[5] = {0, 0, 0, 0, 0};
    for (int d = 0; d < L.ndim; ++d) {
      const int pos = c[d];
      const int p1 = d == 0 ? j : i, p2 = d == 2 ? j : k;
      const int pen = p1 + G.n1[d] * p2;
      add_position(G, C, d, b, pen, pos, bW);
      // adjoint of the fused halo gather along d
      for (int side = 0; side < 2; ++side) {
        const bool near = side ? pos >= n[d] - 2 : pos < 2;
        if (!near) continue;
        const int nb = __ldg(a.face_nbr + 6 * b + 2 * d + side);
        if (nb >= 0) {
          add_position(G, C, d, nb, pen, side ? pos - n[d] : pos + n[d], bW);
        } else if (nb == GBH_BC_OUTFLOW && pos == (side ? n[d] - 1 : 0)) {
          add_position(G, C, d, b, pen, side ? n[d] : -1, bW);
          add_position(G, C, d, b, pen, side ? n[d] + 1 : -2, bW);
        }
      }
    }
    const long long o = own_offset(L, b, i, j, k);
    double U[5], W[5], bU[5];
    for (int v = 0; v < 5; ++v) U[v] = __ldg(a.Uin + o + v * L.vstride);
    bool fr, fp;
    cons_to_prim_flags(U, W, a.eos, fr, fp);
    prim_vjp(W, fr, fp, a.eos, bW, bU);
    for (int v = 0; v < 5; ++v) {
      const long long ov = o + v * L.vstride;
      double x = bU[v];
      if (A) x = fma(cA, A[ov], x);
      if (B) x = fma(cB, B[ov], x);
      out[ov] = x;
    }
  }
}

// out = a X + b Y on interior cells (state layout; out may alias X or Y).
__global__ void axpby_kernel(const Layout L, double a, const double* X, double b, const double* Y, double* out) {
  const long long per = (long long)L.nx * L.ny * L.nz;
  const long long total = per * L.nblocks;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int bk = (int)(t / per);
    long long r = t % per;
    const int i = (int)(r % L.nx);
    r /= L.nx;
    const int j = (int)(r % L.ny);
    const int k = (int)(r / L.ny);
    const long long o = own_offset(L, bk, i, j, k);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const long long ov = o + v * L.vstride;
      out[ov] = fma(a, X[ov], b * Y[ov]);
    }
  }
}

// W (primitive, state layout) -> U on interior cells, and its adjoint.
__global__ void prim_to_cons_kernel(const Layout L, const Eos e, const double* W, double* U, const double* lamU,
                                    double* lamW) {
  const long long per = (long long)L.nx * L.ny * L.nz;
  const long long total = per * L.nblocks;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / per);
    long long r = t % per;
    const int i = (int)(r % L.nx);
    r /= L.nx;
    const int j = (int)(r % L.ny);
    const int k = (int)(r / L.ny);
    const long long o = own_offset(L, b, i, j, k);
    const double rho = W[o], u = W[o + L.vstride], v = W[o + 2 * L.vstride], w = W[o + 3 * L.vstride];
    const double p = W[o + 4 * L.vstride];
    const double k2 = u * u + v * v + w * w;
    if (U) {
      U[o] = rho;
      U[o + L.vstride] = rho * u;
      U[o + 2 * L.vstride] = rho * v;
      U[o + 3 * L.vstride] = rho * w;
      U[o + 4 * L.vstride] = fma(0.5 * rho, k2, p * e.inv_gm1);
    }
    if (lamW) {
      const double l0 = lamU[o], l1 = lamU[o + L.vstride], l2 = lamU[o + 2 * L.vstride];
      const double l3 = lamU[o + 3 * L.vstride], l4 = lamU[o + 4 * L.vstride];
      lamW[o] = l0 + u * l1 + v * l2 + w * l3 + 0.5 * k2 * l4;
      lamW[o + L.vstride] = rho * (l1 + u * l4);
      lamW[o + 2 * L.vstride] = rho * (l2 + v * l4);
      lamW[o + 3 * L.vstride] = rho * (l3 + w * l4);
      lamW[o + 4 * L.vstride] = e.inv_gm1 * l4;
    }
  }
}

int grid_for(long long work) {
  long long g = (work + 255) / 256;
  if (g > 152LL * 16) g = 152LL * 16;
  return (int)(g < 1 ? 1 : g);
}

FaceGeom face_geom(const Layout& L) {
  FaceGeom G{};
  const int n[3] = {L.nx, L.ny, L.nz};
  long long off = 0;
  for (int d = 0; d < 3; ++d) {
    G.n[d] = n[d];
    G.n1[d] = d == 0 ? L.ny : L.nx;
    G.n2[d] = d == 2 ? L.ny : L.nz;
    G.base[d] = off;
    if (d < L.ndim) off += (long long)L.nblocks * G.n1[d] * G.n2[d] * (n[d] + 1) * 20;
  }
  G.total = off;
  return G;
}

}  // namespace

GBH_CHECK_TAKE(check_take_adjoint)

size_t stage_vjp_scratch_doubles(const Layout& L) {
  long long total = 0;
  const int n[3] = {L.nx, L.ny, L.nz};
  for (int d = 0; d < L.ndim; ++d) {
    const long long n1 = d == 0 ? L.ny : L.nx, n2 = d == 2 ? L.ny : L.nz;
    total += (long long)L.nblocks * n1 * n2 * (n[d] + 1) * 20;
  }
  return (size_t)total;
}

cudaError_t launch_stage_vjp(const StageArgs& a, const double* M, double scale, const double* A, double cA,
                             const double* B, double cB, double* C, double* Wp, double* out, cudaStream_t s) {
  const Layout& L = a.lay;
  const FaceGeom G = face_geom(L);
  vjp_prim_kernel<<<grid_for((long long)L.nblocks * L.nx * L.ny * L.nz), 256, 0, s>>>(a, Wp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  long long faces = 0;
  for (int d = 0; d < L.ndim; ++d) faces += (long long)L.nblocks * G.n1[d] * G.n2[d] * (G.n[d] + 1);
  const unsigned grid = (unsigned)((faces + 127) / 128);
  switch (L.nx) {
    case 4: vjp_face_kernel<4><<<grid, 128, 0, s>>>(a, G, Wp, M, scale, C); break;
    case 8: vjp_face_kernel<8><<<grid, 128, 0, s>>>(a, G, Wp, M, scale, C); break;
    case 16: vjp_face_kernel<16><<<grid, 128, 0, s>>>(a, G, Wp, M, scale, C); break;
    default: return cudaErrorInvalidValue;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  vjp_cell_kernel<<<grid_for((long long)L.nblocks * L.nx * L.ny * L.nz), 256, 0, s>>>(a, G, C, A, cA, B, cB, out);
  return cudaGetLastError();
}

cudaError_t launch_axpby(const Layout& L, double a, const double* X, double b, const double* Y, double* out,
                         cudaStream_t s) {
  axpby_kernel<<<grid_for((long long)L.nblocks * L.nx * L.ny * L.nz), 256, 0, s>>>(L, a, X, b, Y, out);
  return cudaGetLastError();
}

cudaError_t launch_prim_to_cons(const Layout& L, const Eos& e, const double* W, double* U, const double* lamU,
                                double* lamW, cudaStream_t s) {
  prim_to_cons_kernel<<<grid_for((long long)L.nblocks * L.nx * L.ny * L.nz), 256, 0, s>>>(L, e, W, U, lamU, lamW);
  return cudaGetLastError();
}

}  // namespace gbh
