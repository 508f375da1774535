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

// Every add and multiply below is a register FMA (a + b = fma(a, 1, b),
// a - b = fma(-b, 1, a), a * b = fma(a, b, -0); gbh_fastmath.cuh), with the
// constants of reg_eos in per-thread registers: the same results as the plain
// operations at the FP64 pipe's full issue rate.

// mc_half_slope with the branch it takes: 0 zero, 1 central, 2 |dm|, 3 |dp|.
__device__ __forceinline__ double mc_half_slope_br(double qm, double q0, double qp, int& br, const Rk& k) {
  const double dm = sub(q0, qm, k);
  const double dp = sub(qp, q0, k);
  const double s4 = quarter_any(add(dm, dp, k));
  const unsigned long long am = mag_key(dm), ap = mag_key(dp), as = mag_key(s4);
  const unsigned long long m1 = am < ap ? am : ap;
  const bool central = as < m1;
  const unsigned long long m = central ? as : m1;
  const bool same = ((dbits(dm) ^ dbits(dp)) >= 0) && am != 0 && ap != 0;
  br = !same ? 0 : (central ? 1 : (am < ap ? 2 : 3));
  return bitsd(same ? (long long)((m >> 1) | sign_bit(dp)) : 0LL);
}

// Adjoint of mc_half_slope_br's result scaled by SIGN (+1 or -1): the
// cotangent is SIGN * bh (the sign is applied by the choice of FMA forms, so
// no negated value has to be formed).
template <int SIGN>
__device__ __forceinline__ void mc_half_slope_vjp(int br, double bh, double& bqm, double& bq0, double& bqp,
                                                  const Rk& k) {
  const double bq = quarter_any(bh);
  const double bdm = br == 1 ? bq : (br == 2 ? bh : 0.0);
  const double bdp = br == 1 ? bq : (br == 3 ? bh : 0.0);
  if (SIGN > 0) {
    bqm = sub(bqm, bdm, k);
    bq0 = add(bq0, sub(bdm, bdp, k), k);
    bqp = add(bqp, bdp, k);
  } else {
    bqm = add(bqm, bdm, k);
    bq0 = add(bq0, sub(bdp, bdm, k), k);
    bqp = sub(bqp, bdp, k);
  }
}

// cons_to_prim reporting which floors applied.
__device__ __forceinline__ void cons_to_prim_flags(const double U[5], double W[5], const Eos& e, bool& fr,
                                                   bool& fp) {
  const Rk& k = e.k;
  double rho = U[0];
  fr = less_d(rho, e.small_rho);
  if (fr) rho = e.small_rho;
  const double ir = rcp_nr(rho, k);
  const double u = mul(U[1], ir, k), v = mul(U[2], ir, k), w = mul(U[3], ir, k);
  const double m2 = fma(U[3], w, fma(U[2], v, mul(U[1], u, k)));
  double p = mul(e.gm1, fma(-half_any(m2), k.one, U[4]), k);
  fp = less_d(p, e.small_p);
  if (fp) p = e.small_p;
  W[0] = rho; W[1] = u; W[2] = v; W[3] = w; W[4] = p;
}

// bU = (dW/dU)^T bW for W = cons_to_prim(U); floored components are constants.
__device__ __forceinline__ void prim_vjp(const double W[5], bool fr, bool fp, const Eos& e, const double bW[5],
                                         double bU[5]) {
  const Rk& k = e.k;
  const double ir = rcp_nr(W[0], k);
  const double u = W[1], v = W[2], w = W[3];
  const double bp = fp ? 0.0 : mul(bW[4], e.gm1, k);
  bU[4] = bp;
  bU[1] = fma(ir, bW[1], -mul(bp, u, k));
  bU[2] = fma(ir, bW[2], -mul(bp, v, k));
  bU[3] = fma(ir, bW[3], -mul(bp, w, k));
  const double uw = fma(w, bW[3], fma(v, bW[2], mul(u, bW[1], k)));
  const double k2 = fma(w, w, fma(v, v, mul(u, u, k)));
  bU[0] = fr ? 0.0 : fma(half_any(bp), k2, fma(-ir, uw, bW[0]));
}

// Reverse of hllc_flux (gbh_device.cuh): the forward is recomputed from the
// same formulas, grouped for the reverse sweep (one reciprocal square root of
// rho_L rho_R, the Roe sound speed from w_L c_L^2 + w_R c_R^2 + (gamma-1)/2
// w_L w_R |u_L - u_R|^2, the star state through t = u_K + g), then
// (dF/dW)^T bF is accumulated step by step in reverse.  Branches (the min / max of the wave-speed bounds, the side K,
// the fan) keep the forward's decisions and are taken by selects.
__device__ __forceinline__ void hllc_flux_vjp(const double WL[5], const double WR[5], const Eos& e, const double bF[5],
                              double bWL[5], double bWR[5]) {
  const Rk& k = e.k;
  auto A = [&](double x, double y) { return fma(x, k.one, y); };    // x + y
  auto S = [&](double x, double y) { return fma(-y, k.one, x); };   // x - y
  auto M = [&](double x, double y) { return fma(x, y, k.nz); };     // x * y
  const double rL = WL[0], uL = WL[1], vL = WL[2], wL = WL[3], pL = WL[4];
  const double rR = WR[0], uR = WR[1], vR = WR[2], wR = WR[3], pR = WR[4];
  // ---- forward ----
  const double q = rsqrt_nr(M(rL, rR), k);                 // 1/sqrt(rho_L rho_R)
  const double q2 = M(q, q);
  const double iL = M(rR, q2), iR = M(rL, q2);             // 1/rho
  const double gpL = M(e.gamma, pL), gpR = M(e.gamma, pR);
  const double cL2 = M(gpL, iL), cR2 = M(gpR, iR);         // c^2
  const double qL = rsqrt_nr(cL2, k), qR = rsqrt_nr(cR2, k);   // 1/c
  const double cL = M(cL2, qL), cR = M(cR2, qR);
  const double r = M(rR, q);                               // sqrt(rho_R / rho_L)
  const double wl = rcp_nr(A(r, k.one), k), wr = M(r, wl);
  const double ut = fma(wl, uL, M(wr, uR));
  const double du = S(uL, uR), dv = S(vL, vR), dw = S(wL, wR);
  const double du2 = fma(dw, dw, fma(dv, dv, M(du, du)));
  const double Bw = M(e.hgm1, M(wl, wr));
  const double ct2 = fma(Bw, du2, fma(wl, cL2, M(wr, cR2)));
  const double qc = rsqrt_nr(ct2, k);
  const double ct = M(ct2, qc);
  const double l1 = S(uL, cL), l2 = S(ut, ct), r1 = A(uR, cR), r2 = A(ut, ct);
  const bool selL1 = !(order_key(l2) < order_key(l1));     // S_L = l1
  const bool selR1 = !(order_key(r1) < order_key(r2));     // S_R = r1
  const double SL = selL1 ? l1 : l2, SR = selR1 ? r1 : r2;
  const double dL = S(SL, uL), dR = S(SR, uR);
  const double mL = M(rL, dL), mR = M(rR, dR);
  const double rd = rcp_nr(S(mL, mR), k);
  const double Ss = M(fma(-mR, uR, fma(mL, uL, S(pR, pL))), rd);
  const bool left = ge0(Ss);
  const double rK = sel(left, rL, rR), uK = sel(left, uL, uR), vK = sel(left, vL, vR);
  const double wK = sel(left, wL, wR), pK = sel(left, pL, pR);
  const double SK = sel(left, SL, SR), mK = sel(left, mL, mR), dK = sel(left, dL, dR);
  const bool fan = left ? lt0(SL) : gt0(SR);
  const double R = rcp_nr(S(SK, Ss), k);                   // used inside the fan only
  const double dKR = M(dK, R);
  const double t = sel(fan, M(Ss, dKR), uK);
  const double g = S(t, uK);
  const double kK = fma(wK, wK, fma(vK, vK, M(uK, uK)));
  const double hK = fma(half_pos(rK), kK, M(e.g_gm1, pK));
  const double gm = M(g, mK);
  const double F0 = M(rK, t);
  // ---- reverse ----
  // F2 = vK F0, F3 = wK F0
  const double bF0 = fma(bF[3], wK, fma(bF[2], vK, bF[0]));
  double bvK = M(bF[2], F0), bwK = M(bF[3], F0);
  // F4 = hK t + gm Ss
  const double bhK = M(bF[4], t);
  double bt = M(bF[4], hK);
  double bgm = A(M(bF[4], Ss), bF[1]);                     // with F1's direct term
  double bSs = M(bF[4], gm);
  // F1 = F0 uK + pK + gm
  const double bF0t = fma(bF[1], uK, bF0);
  double buK = M(bF[1], F0);
  double bpK = bF[1];
  // F0 = rK t
  double brK = M(bF0t, t);
  bt = fma(bF0t, rK, bt);
  // gm = g mK
  const double bg = M(bgm, mK);
  const double bmK = M(bgm, g);
  // hK = rK kK / 2 + g_gm1 pK, kK = |u_K|^2
  brK = fma(half_any(kK), bhK, brK);
  const double bkK2 = M(bhK, rK);                          // 2 * (rK / 2) * bhK
  bpK = fma(bhK, e.g_gm1, bpK);
  buK = fma(bkK2, uK, buK);
  bvK = fma(bkK2, vK, bvK);
  bwK = fma(bkK2, wK, bwK);
  // g = t - uK
  bt = A(bt, bg);
  buK = S(buK, bg);
  // t = Ss dK R in the fan, R = 1 / (SK - Ss); t = uK outside it
  const double btS = M(bt, Ss);
  const double nbX = M(M(btS, dK), M(R, R));               // -(adjoint of SK - Ss)
  bSs = sel(fan, A(fma(bt, dKR, bSs), nbX), bSs);
  const double bdK = sel(fan, M(btS, R), 0.0);
  const double nbSK = sel(fan, nbX, 0.0);                  // -(adjoint of SK)
  buK = sel(fan, buK, A(buK, bt));
  // the chosen side
  double brL = sel(left, brK, 0.0), buL = sel(left, buK, 0.0), bvL = sel(left, bvK, 0.0);
  double bwL = sel(left, bwK, 0.0), bpL = sel(left, bpK, 0.0);
  double bmL = sel(left, bmK, 0.0), bdL = sel(left, bdK, 0.0);
  double brR = sel(left, 0.0, brK), buR = sel(left, 0.0, buK), bvR = sel(left, 0.0, bvK);
  double bwR = sel(left, 0.0, bwK), bpR = sel(left, 0.0, bpK);
  double bmR = sel(left, 0.0, bmK), bdR = sel(left, 0.0, bdK);
  const double nbSL = sel(left, nbSK, 0.0), nbSR = sel(left, 0.0, nbSK);
  // Ss = N rd, N = pR - pL + mL uL - mR uR, rd = 1 / (mL - mR)
  const double bN = M(bSs, rd);
  const double nbD = M(bN, Ss);                            // -(adjoint of mL - mR)
  bpR = A(bpR, bN);
  bpL = S(bpL, bN);
  bmL = S(fma(bN, uL, bmL), nbD);
  buL = fma(bN, mL, buL);
  bmR = A(fma(-bN, uR, bmR), nbD);
  buR = fma(-bN, mR, buR);
  // mL = rL dL, mR = rR dR; dL = SL - uL, dR = SR - uR
  brL = fma(bmL, dL, brL);
  bdL = fma(bmL, rL, bdL);
  brR = fma(bmR, dR, brR);
  bdR = fma(bmR, rR, bdR);
  const double bSL = S(bdL, nbSL);
  buL = S(buL, bdL);
  const double bSR = S(bdR, nbSR);
  buR = S(buR, bdR);
  // SL = min(uL - cL, ut - ct), SR = max(uR + cR, ut + ct)
  const double sLl = sel(selL1, bSL, 0.0), sLt = sel(selL1, 0.0, bSL);
  const double sRr = sel(selR1, bSR, 0.0), sRt = sel(selR1, 0.0, bSR);
  buL = A(buL, sLl);
  buR = A(buR, sRr);
  const double but = A(sLt, sRt);
  const double bct = S(sRt, sLt);
  // ct = sqrt(ct2): d ct / d ct2 = qc / 2
  const double bct2 = M(half_any(bct), qc);
  // ct2 = Bw du2 + wl cL2 + wr cR2, Bw = hgm1 wl wr
  const double bBh = M(M(bct2, du2), e.hgm1);
  const double b2 = M(A(bct2, bct2), Bw);                  // 2 * adjoint of du2
  double bwl = fma(bct2, cL2, M(bBh, wr));
  double bwr = fma(bct2, cR2, M(bBh, wl));
  double bcL2 = M(bct2, wl), bcR2 = M(bct2, wr);
  // du2 = du^2 + dv^2 + dw^2
  const double bdu = M(b2, du), bdv = M(b2, dv), bdw = M(b2, dw);
  buL = A(buL, bdu);
  buR = S(buR, bdu);
  bvL = A(bvL, bdv);
  bvR = S(bvR, bdv);
  bwL = A(bwL, bdw);
  bwR = S(bwR, bdw);
  // ut = wl uL + wr uR
  bwl = fma(but, uL, bwl);
  buL = fma(but, wl, buL);
  bwr = fma(but, uR, bwr);
  buR = fma(but, wr, buR);
  // wr = r wl, wl = 1 / (1 + r)
  bwl = fma(bwr, r, bwl);
  const double br = fma(-bwl, M(wl, wl), M(bwr, wl));
  // cL = sqrt(cL2) = cL2 qL, cR likewise; bcL = -sLl, bcR = sRr
  bcL2 = fma(-half_any(sLl), qL, bcL2);
  bcR2 = fma(half_any(sRr), qR, bcR2);
  // cL2 = gamma pL iL, cR2 = gamma pR iR
  bpL = fma(M(bcL2, iL), e.gamma, bpL);
  bpR = fma(M(bcR2, iR), e.gamma, bpR);
  const double biL = M(bcL2, gpL), biR = M(bcR2, gpR);
  // iL = rR q2, iR = rL q2, r = rR q, q2 = q q
  brR = fma(biL, q2, brR);
  brL = fma(biR, q2, brL);
  const double bq2 = fma(biL, rR, M(biR, rL));
  brR = fma(br, q, brR);
  const double bq = fma(br, rR, M(A(bq2, bq2), q));
  // q = (rL rR)^(-1/2): d q / d(rL rR) = -q^3 / 2
  const double nbP = M(M(half_any(bq), q), q2);
  brL = fma(-nbP, rR, brL);
  brR = fma(-nbP, rL, brR);
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
  int n[3];            // pencil length per dimension (the box's: n + 2E)
  int n1[3], n2[3];    // transverse extents per dimension
  int ring[3];         // ring width per dimension (E; 0 in z of a 2-D grid): box position q is cell q - ring
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

template <int N, int d, int E>
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
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  // transverse cells; E = 0: the interior pencils, no offsets (compile time)
  const int p1 = pen % G.n1[d] - (E ? G.ring[t1] : 0), p2 = pen / G.n1[d] - (E ? G.ring[t2] : 0);
  const int nd = G.n[d], Ed = E ? G.ring[d] : 0;
  const long long zt = thread_zero(a.eos);
  const Eos e = reg_eos(a.eos, zt);   // FP64 constants in per-thread registers
  const Rk& kr = e.k;
  const double sc = reg_const(scale * __ldg(a.inv_dx + 3 * b + d), zt);
  const int rot[5] = {0, 1 + d, d == 0 ? 2 : 1, d == 2 ? 2 : 3, 4};

  double W[4][5];
  int ci, cj, ck;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    // primitives of the stencil position (the halo gathered as in the stage
    // kernel; in guard mode the block's own padded cells)
    pencil_to_cell(d, k - 2 + s - Ed, p1, p2, ci, cj, ck);
    const long long o = cell_offset<N>(a, b, ci, cj, ck);
#pragma unroll
    for (int v = 0; v < 5; ++v) W[s][v] = __ldg(Wp + o + v * L.vstride);
  }
  double h0[5], h1[5];
  int b0[5], b1[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    h0[v] = mc_half_slope_br(W[0][v], W[1][v], W[2][v], b0[v], kr);   // slope of position k-1
    h1[v] = mc_half_slope_br(W[1][v], W[2][v], W[3][v], b1[v], kr);   // slope of position k
  }
  double bF[5];
  {
    double mk[5] = {0, 0, 0, 0, 0}, mk1[5] = {0, 0, 0, 0, 0};
    if (k < nd) {
      pencil_to_cell(d, k - Ed, p1, p2, ci, cj, ck);
      const long long o = own_offset(L, b, ci, cj, ck);
      for (int v = 0; v < 5; ++v) mk[v] = __ldg(M + o + v * L.vstride);
    }
    if (k > 0) {
      pencil_to_cell(d, k - 1 - Ed, p1, p2, ci, cj, ck);
      const long long o = own_offset(L, b, ci, cj, ck);
      for (int v = 0; v < 5; ++v) mk1[v] = __ldg(M + o + v * L.vstride);
    }
    for (int v = 0; v < 5; ++v) bF[v] = mul(sc, sub(mk[v], mk1[v], kr), kr);
  }
  double wl[5], wr[5], bFr[5], bwl[5], bwr[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    wl[q] = add(W[1][rot[q]], h0[rot[q]], kr);
    wr[q] = sub(W[2][rot[q]], h1[rot[q]], kr);
    bFr[q] = bF[rot[q]];
  }
  hllc_flux_vjp(wl, wr, e, bFr, bwl, bwr);
  double Cs[4][5];
#pragma unroll
  for (int v = 0; v < 5; ++v) Cs[0][v] = Cs[1][v] = Cs[2][v] = Cs[3][v] = 0.0;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int v = rot[q];
    Cs[1][v] = add(Cs[1][v], bwl[q], kr);
    Cs[2][v] = add(Cs[2][v], bwr[q], kr);
    mc_half_slope_vjp<1>(b0[v], bwl[q], Cs[0][v], Cs[1][v], Cs[2][v], kr);
    mc_half_slope_vjp<-1>(b1[v], bwr[q], Cs[1][v], Cs[2][v], Cs[3][v], kr);   // wr = W2 - h1
  }
  double* out = C + slot_index(G, d, b, pen, k, 0);
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int v = 0; v < 5; ++v) out[s * 5 + v] = Cs[s][v];
}

// E = 0: the interior faces (offsets known to be zero); E = 1: a box whose
// ring widths G.ring are applied at run time.
template <int N, int E>
__global__ void __launch_bounds__(128, 4) vjp_face_kernel(const StageArgs a, const FaceGeom G,
                                                      const double* __restrict__ Wp, const double* __restrict__ M,
                                                      double scale, double* __restrict__ C) {
  const Layout& L = a.lay;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (int d = 0; d < L.ndim; ++d) {
    const long long count = (long long)L.nblocks * G.n1[d] * G.n2[d] * (G.n[d] + 1);
    if (t < count) {
      if (d == 0) face_work<N, 0, E>(a, G, Wp, M, scale, C, t);
      else if (d == 1) face_work<N, 1, E>(a, G, Wp, M, scale, C, t);
      else face_work<N, 2, E>(a, G, Wp, M, scale, C, t);
      return;
    }
    t -= count;
  }
}

// Primitives of every interior cell of Uin (cons_to_prim, floors as in the
// stage kernel) into Wp, state layout; the face pass gathers them.
__global__ void vjp_prim_kernel(const StageArgs a, double* __restrict__ Wp) {
  const Layout& L = a.lay;
  const Eos e = reg_eos(a.eos, thread_zero(a.eos));
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
    cons_to_prim(U, W, e);
#pragma unroll
    for (int v = 0; v < 5; ++v) Wp[o + v * L.vstride] = W[v];
  }
}

// Primitives of every padded cell of Uin into Wp (the box faces of a ring
// stage read the block's own guard cells).
__global__ void vjp_prim_padded_kernel(const StageArgs a, double* __restrict__ Wp) {
  const Layout& L = a.lay;
  const Eos e = reg_eos(a.eos, thread_zero(a.eos));
  const long long total = (long long)L.nblocks * L.bstride / 5;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / L.vstride;
    const long long o = b * L.bstride + (t - b * L.vstride);
    double U[5], W[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = __ldg(a.Uin + o + v * L.vstride);
    cons_to_prim(U, W, e);
#pragma unroll
    for (int v = 0; v < 5; ++v) Wp[o + v * L.vstride] = W[v];
  }
}

// Sum of the slots of block b, dimension d, pencil pen that refer to the
// halo-extended position q (-2..n_d+1), in increasing face order.
__device__ __forceinline__ void add_position(const FaceGeom& G, const double* __restrict__ C, int d, int b, int pen,
                                             int q, double acc[5], const Rk& kr) {
  const int nd = G.n[d];
  for (int k = q - 1; k <= q + 2; ++k) {
    if (k < 0 || k > nd) continue;
    const double* c = C + slot_index(G, d, b, pen, k, q + 2 - k);
    for (int v = 0; v < 5; ++v) acc[v] = add(acc[v], c[v], kr);
  }
}

// ---- the cell pass ------------------------------------------------------------

__global__ void vjp_cell_kernel(const StageArgs a, const FaceGeom G, const double* __restrict__ C, const double* A,
                                double cA, const double* B, double cB, double* out) {
  const Layout& L = a.lay;
  const long long zt = thread_zero(a.eos);
  const Eos e = reg_eos(a.eos, zt);   // FP64 constants in per-thread registers
  const Rk& kr = e.k;
  const double rcA = reg_const(cA, zt), rcB = reg_const(cB, zt);
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
      add_position(G, C, d, b, pen, pos, bW, kr);
      // adjoint of the fused halo gather along d
      for (int side = 0; side < 2; ++side) {
        const bool near = side ? pos >= n[d] - 2 : pos < 2;
        if (!near) continue;
        const int nb = __ldg(a.face_nbr + 6 * b + 2 * d + side);
        if (nb >= 0) {
          add_position(G, C, d, nb, pen, side ? pos - n[d] : pos + n[d], bW, kr);
        } else if (nb == GBH_BC_OUTFLOW && pos == (side ? n[d] - 1 : 0)) {
          add_position(G, C, d, b, pen, side ? n[d] : -1, bW, kr);
          add_position(G, C, d, b, pen, side ? n[d] + 1 : -2, bW, kr);
        }
      }
    }
    const long long o = own_offset(L, b, i, j, k);
    double U[5], W[5], bU[5];
    for (int v = 0; v < 5; ++v) U[v] = __ldg(a.Uin + o + v * L.vstride);
    bool fr, fp;
    cons_to_prim_flags(U, W, e, fr, fp);
    prim_vjp(W, fr, fp, e, bW, bU);
    for (int v = 0; v < 5; ++v) {
      const long long ov = o + v * L.vstride;
      double x = bU[v];
      if (A) x = fma(rcA, A[ov], x);
      if (B) x = fma(rcB, B[ov], x);
      out[ov] = x;
    }
  }
}

// ---- the padded-cell pass of a box VJP (guard mode) ---------------------------
//
// For the stage of ring width G.ring on the block's own padded cells (the
// telescoping mode): every padded cell sums the slots of the box faces whose
// stencils read it, in increasing face order per dimension (positions -2 ..
// n + 2E + 1 of the pencils through it), applies the reverse of the EOS where
// some face read it, and adds up to three linear terms, each on a box of its
// own ring width (the cells where that term's array is defined):
//   out = J^T (scale M) + sum_t [cell in box E_t] c_t X_t.
// Every padded cell of out is written (0 where nothing reaches it).
struct LinTerms {
  const double* X[3];
  double c[3];
  int ring[3];
  int n;
};

__device__ __forceinline__ bool in_box(const Layout& L, int E, int i, int j, int k) {
  return i >= -E && i < L.nx + E && j >= -E && j < L.ny + E && (L.ndim == 2 || (k >= -E && k < L.nz + E));
}

__global__ void vjp_padded_cell_kernel(const StageArgs a, const FaceGeom G, const double* __restrict__ C,
                                       const LinTerms T, double* out) {
  const Layout& L = a.lay;
  const long long zt = thread_zero(a.eos);
  const Eos e = reg_eos(a.eos, zt);   // FP64 constants in per-thread registers
  const Rk& kr = e.k;
  const long long per = (long long)L.nxp * L.nyp * L.nzp;
  const long long total = per * L.nblocks;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / per);
    long long r = t % per;
    const int i = (int)(r % L.nxp) - L.g;
    r /= L.nxp;
    const int j = (int)(r % L.nyp) - L.g;
    const int k = (int)(r / L.nyp) - L.gz;
    const int c[3] = {i, j, k};
    double bW[5] = {0, 0, 0, 0, 0};
    bool read = false;
    for (int d = 0; d < L.ndim; ++d) {
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      const int q1 = c[t1] + G.ring[t1], q2 = c[t2] + G.ring[t2];   // box pencil through the cell
      if (q1 < 0 || q1 >= G.n[t1] || q2 < 0 || q2 >= G.n[t2]) continue;
      const int q = c[d] + G.ring[d];                                 // box position along d
      if (q < -2 || q > G.n[d] + 1) continue;
      add_position(G, C, d, b, q1 + G.n1[d] * q2, q, bW, kr);
      read = true;
    }
    const long long o = own_offset(L, b, i, j, k);
    double bU[5] = {0, 0, 0, 0, 0};
    if (read) {
      double U[5], W[5];
      for (int v = 0; v < 5; ++v) U[v] = __ldg(a.Uin + o + v * L.vstride);
      bool fr, fp;
      cons_to_prim_flags(U, W, e, fr, fp);
      prim_vjp(W, fr, fp, e, bW, bU);
    }
    for (int q = 0; q < T.n; ++q)
      if (in_box(L, T.ring[q], i, j, k)) {
        const double cq = reg_const(T.c[q], zt);
        for (int v = 0; v < 5; ++v) bU[v] = fma(cq, T.X[q][o + v * L.vstride], bU[v]);
      }
    for (int v = 0; v < 5; ++v) out[o + v * L.vstride] = bU[v];
  }
}

// ---- the reverse of the full guard fill (fill_kernel) -----------------------
//
// The fill copies interior cells into guard cells; its adjoint adds every
// guard cell's adjoint to the interior cell it was copied from.  As a gather,
// with one thread per interior cell s of block b and no atomics: per
// dimension the guard cell's coordinate either equals s's (no offset), lies
// across the face of the guard cell's block whose neighbour is b (s within
// g of b's opposite face: a copy from the neighbour), or lies outside an
// outflow face (s on that face: a clamped copy, any of the g guard
// positions).  The guard cell's block is b's neighbour against the
// neighbour offsets; each combination is checked against the tables the fill
// used.  out = lam + the sum over the guard cells, on interior cells.
__global__ void fill_vjp_kernel(const Layout L, const int* nbr, const int* face_nbr, const double* lam, double* out) {
  const int nn = L.ndim == 3 ? 27 : 9;
  const int n[3] = {L.nx, L.ny, L.nz};
  const int g[3] = {L.g, L.g, L.gz};
  const long long per = (long long)L.nx * L.ny * L.nz;
  const long long total = per * L.nblocks;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / per);
    long long r = t % per;
    const int c[3] = {(int)(r % L.nx), (int)((r / L.nx) % L.ny), (int)(r / ((long long)L.nx * L.ny))};
    double acc[5];
    const long long os = own_offset(L, b, c[0], c[1], c[2]);
    for (int v = 0; v < 5; ++v) acc[v] = lam[os + v * L.vstride];
    // options per dimension: 0 the same coordinate, 1 / 2 a copy across the
    // guard block's low / high face, 3 / 4 a clamp at its low / high outflow face
    const int nopt[3] = {5, 5, L.ndim == 3 ? 5 : 1};
    for (int oz = 0; oz < nopt[2]; ++oz)
      for (int oy = 0; oy < nopt[1]; ++oy)
        for (int ox = 0; ox < nopt[0]; ++ox) {
          const int opt[3] = {ox, oy, oz};
          if (ox == 0 && oy == 0 && oz == 0) continue;
          int off[3] = {0, 0, 0};   // offset of b seen from the guard cell's block
          int lo[3], hi[3];         // guard-cell coordinates in the guard block
          bool ok = true;
          for (int d = 0; d < 3 && ok; ++d) {
            switch (opt[d]) {
              case 0: lo[d] = hi[d] = c[d]; break;
              case 1: ok = c[d] >= n[d] - g[d]; off[d] = -1; lo[d] = hi[d] = c[d] - n[d]; break;
              case 2: ok = c[d] < g[d]; off[d] = 1; lo[d] = hi[d] = c[d] + n[d]; break;
              case 3: ok = c[d] == 0; lo[d] = -g[d]; hi[d] = -1; break;
              default: ok = c[d] == n[d] - 1; lo[d] = n[d]; hi[d] = n[d] + g[d] - 1; break;
            }
          }
          if (!ok) continue;
          // the guard cell's block: b's neighbour at -off
          int gb = b;
          if (off[0] || off[1] || off[2]) {
            const int e = L.ndim == 3 ? (1 - off[2]) * 9 + (1 - off[1]) * 3 + (1 - off[0])
                                      : (1 - off[1]) * 3 + (1 - off[0]);
            gb = __ldg(nbr + (long long)nn * b + e);
            if (gb < 0) continue;
            const int eb = L.ndim == 3 ? (off[2] + 1) * 9 + (off[1] + 1) * 3 + (off[0] + 1)
                                       : (off[1] + 1) * 3 + (off[0] + 1);
            if (__ldg(nbr + (long long)nn * gb + eb) != b) continue;   // the fill would read another block
          }
          // the fill clamps exactly at gb's outflow faces
          for (int d = 0; d < L.ndim && ok; ++d) {
            if (opt[d] == 0) continue;
            const int f = 2 * d + ((opt[d] == 2 || opt[d] == 4) ? 1 : 0);
            const bool outflow = __ldg(face_nbr + 6 * gb + f) == GBH_BC_OUTFLOW;
            ok = (opt[d] >= 3) == outflow;
          }
          if (!ok) continue;
          for (int z = lo[2]; z <= hi[2]; ++z)
            for (int y = lo[1]; y <= hi[1]; ++y)
              for (int x = lo[0]; x <= hi[0]; ++x) {
                const long long og = own_offset(L, gb, x, y, z);
                for (int v = 0; v < 5; ++v) acc[v] += lam[og + v * L.vstride];
              }
        }
    for (int v = 0; v < 5; ++v) out[os + v * L.vstride] = acc[v];
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

// Faces of the box of ring width E around every block's interior (E = 0: the
// interior itself), per dimension: pencils over the box's transverse extent,
// n + 2E + 1 faces each.
FaceGeom face_geom(const Layout& L, int E = 0) {
  FaceGeom G{};
  int n[3] = {L.nx, L.ny, L.nz};
  for (int d = 0; d < 3; ++d) {
    G.ring[d] = d < L.ndim ? E : 0;
    n[d] += 2 * G.ring[d];
  }
  long long off = 0;
  for (int d = 0; d < 3; ++d) {
    G.n[d] = n[d];
    G.n1[d] = d == 0 ? n[1] : n[0];
    G.n2[d] = d == 2 ? n[1] : n[2];
    G.base[d] = off;
    if (d < L.ndim) off += (long long)L.nblocks * G.n1[d] * G.n2[d] * (n[d] + 1) * 20;
  }
  G.total = off;
  return G;
}

}  // namespace

GBH_CHECK_TAKE(check_take_adjoint)

size_t stage_vjp_scratch_doubles(const Layout& L, int ring) { return (size_t)face_geom(L, ring).total; }

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
    case 4: vjp_face_kernel<4, 0><<<grid, 128, 0, s>>>(a, G, Wp, M, scale, C); break;
    case 8: vjp_face_kernel<8, 0><<<grid, 128, 0, s>>>(a, G, Wp, M, scale, C); break;
    case 16: vjp_face_kernel<16, 0><<<grid, 128, 0, s>>>(a, G, Wp, M, scale, C); break;
    default: return cudaErrorInvalidValue;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  vjp_cell_kernel<<<grid_for((long long)L.nblocks * L.nx * L.ny * L.nz), 256, 0, s>>>(a, G, C, A, cA, B, cB, out);
  return cudaGetLastError();
}

cudaError_t launch_stage_vjp_box(const StageArgs& a, int ring, const double* M, double scale, const double* const X[3],
                                 const double c[3], const int rings[3], int nterms, double* C, double* Wp, double* out,
                                 cudaStream_t s) {
  const Layout& L = a.lay;
  if (a.gather || ring < 0 || L.g < ring + 2 || nterms < 0 || nterms > 3) return cudaErrorInvalidValue;
  const FaceGeom G = face_geom(L, ring);
  // primitives of every padded cell the box faces read: all of them
  vjp_prim_padded_kernel<<<grid_for((long long)L.nblocks * L.nxp * L.nyp * L.nzp), 256, 0, s>>>(a, Wp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  long long faces = 0;
  for (int d = 0; d < L.ndim; ++d) faces += (long long)L.nblocks * G.n1[d] * G.n2[d] * (G.n[d] + 1);
  const unsigned grid = (unsigned)((faces + 127) / 128);
  // the ring is a run-time offset here (E = 1 selects it); the interior
  // instantiation above keeps its compile-time zero offsets
  switch (L.nx) {
    case 4: vjp_face_kernel<4, 1><<<grid, 128, 0, s>>>(a, G, Wp, M, scale, C); break;
    case 8: vjp_face_kernel<8, 1><<<grid, 128, 0, s>>>(a, G, Wp, M, scale, C); break;
    case 16: vjp_face_kernel<16, 1><<<grid, 128, 0, s>>>(a, G, Wp, M, scale, C); break;
    default: return cudaErrorInvalidValue;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  LinTerms T{};
  T.n = nterms;
  for (int q = 0; q < nterms; ++q) {
    T.X[q] = X[q];
    T.c[q] = c[q];
    T.ring[q] = rings[q];
  }
  vjp_padded_cell_kernel<<<grid_for((long long)L.nblocks * L.nxp * L.nyp * L.nzp), 256, 0, s>>>(a, G, C, T, out);
  return cudaGetLastError();
}

cudaError_t launch_fill_vjp(const Layout& L, const int* nbr, const int* face_nbr, const double* lam, double* out,
                            cudaStream_t s) {
  fill_vjp_kernel<<<grid_for((long long)L.nblocks * L.nx * L.ny * L.nz), 256, 0, s>>>(L, nbr, face_nbr, lam, out);
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
