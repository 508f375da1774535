// gbh_device.cuh -- per-cell and per-face FP64 arithmetic of the stage kernel.
//
// The intra-stage calculations of the paper's hydrodynamics variants
// (Sec. 4.2, Alg. "Intra stage calculations for Spark") are calcLims
// (reconstruction), calcFlux (face fluxes), updSoln (flux-difference update)
// and calcEos (equation of state).  The numerics they leave open are read as:
// ideal-gas EOS with floors, MC-limited piecewise-linear reconstruction of
// primitive variables, and the HLLC flux (Toro's star state, Einfeldt /
// Roe-average wave-speed bounds).
//
// The formulas are arranged to minimise FP64 instructions (the kernel is
// bound by the FP64 pipe): one reciprocal per primitive conversion, one
// reciprocal square root per face side giving both sqrt(rho) and 1/rho, the
// HLLC star state reduced to a single reciprocal, and every comparison done
// on bit patterns (gbh_fastmath.cuh).  Results agree with the plain
// formulas to rounding.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbh_fastmath.cuh"
#include "gbh_internal.h"

namespace gbh {

// calcEos role: conserved (rho, mx, my, mz, E) -> primitive (rho, u, v, w, p),
// p = (gamma-1) (E - (mx u + my v + mz w)/2).  Floors rho at small_rho and p
// at small_p; returns 1 when a floor applied.
__device__ __forceinline__ int cons_to_prim_ir(const double U[5], double W[5], const Eos& e, double& ir) {
  const Rk& k = e.k;
  int hit = 0;
  double rho = U[0];
  if (less_d(rho, e.small_rho)) { rho = e.small_rho; hit = 1; }
  ir = rcp_nr(rho, k);
  const double u = mul(U[1], ir, k), v = mul(U[2], ir, k), w = mul(U[3], ir, k);
  const double m2 = fma(U[3], w, fma(U[2], v, mul(U[1], u, k)));   // >= 0
  double p = mul(e.gm1, fma(-half_any(m2), k.one, U[4]), k);       // (gamma-1) (E - m2/2)
  if (less_d(p, e.small_p)) { p = e.small_p; hit = 1; }
  W[0] = rho; W[1] = u; W[2] = v; W[3] = w; W[4] = p;
  return hit;
}

__device__ __forceinline__ int cons_to_prim(const double U[5], double W[5], const Eos& e) {
  double ir;
  return cons_to_prim_ir(U, W, e, ir);
}

// calcLims role: half of the MC-limited slope at q0,
//   sigma/2 = sign(dp) * min(|dm+dp|/4, |dm|, |dp|) if dm, dp have the same strict sign, else 0,
// so that the face values are q0 -/+ sigma/2.  Sign test and minimum on bit
// patterns.
__device__ __forceinline__ double mc_half_slope(double qm, double q0, double qp) {
  const double dm = q0 - qm;
  const double dp = qp - q0;
  const double s4 = 0.25 * (dm + dp);
  const unsigned long long am = mag_key(dm), ap = mag_key(dp), as = mag_key(s4);
  unsigned long long m = am < ap ? am : ap;
  m = as < m ? as : m;
  const bool same = ((dbits(dm) ^ dbits(dp)) >= 0) && am != 0 && ap != 0;
  return bitsd(same ? (long long)((m >> 1) | sign_bit(dp)) : 0LL);
}

// Half the MC-limited slope from the differences dm = q0 - qm, dp = qp - q0:
//   sigma/2 = sign(dp) * min(|dm+dp|, 4|dm|, 4|dp|) / 4
// if dm, dp have the same strict sign, else 0, so the face values are
// q0 -/+ sigma/2 (register FMAs).  The factors 4 are added to the exponent
// fields of |dm|, |dp| and the division by 4 taken off the exponent of the
// minimum, on the integer pipe: exact for normal numbers (a subnormal |dm| or
// |dp|, or a minimum below 2^-1020, is scaled by shifting the bit pattern,
// which moves the result by less than 2^-1020).  One FP64 operation (the sum).
__device__ __forceinline__ double mc_half_slope_d(double dm, double dp, const Rk& k) {
  const double sum = add(dm, dp, k);
  const unsigned long long am = mag_key(dm), ap = mag_key(dp), as = mag_key(sum);
  unsigned long long m = (am < ap ? am : ap) + (4ULL << 52);   // min(4|dm|, 4|dp|): exponent + 2 in key form
  m = as < m ? as : m;
  m >>= 1;                                                       // magnitude bits of 2 sigma
  m = m >= (3ULL << 52) ? m - (2ULL << 52) : m >> 2;            // / 4
  const bool same = ((dbits(dm) ^ dbits(dp)) >= 0) && am != 0 && ap != 0;
  return bitsd(same ? (long long)(m | sign_bit(dp)) : 0LL);
}

// x / 2 for a positive normal x >= 2^-1021 (one off the exponent field)
__device__ __forceinline__ double half_pos(double x) { return bitsd(dbits(x) - (1LL << 52)); }

// max(a, b) of non-negative doubles on the integer pipe (their bit patterns
// order like their values; fmax is an FP64-pipe instruction).  A NaN operand
// is passed over, as fmax passes it over.
__device__ __forceinline__ double max_nonneg(double a, double b) {
  constexpr unsigned long long kInf = 0x7ff0000000000000ULL;
  unsigned long long x = (unsigned long long)dbits(a), y = (unsigned long long)dbits(b);
  x = x > kInf ? 0ULL : x;
  y = y > kInf ? 0ULL : y;
  return bitsd((long long)(x > y ? x : y));
}

// Maximum over the NT threads of a CTA (NT a power of two) of non-negative
// values: xor shuffles within each warp (over the lanes the CTA has), then
// the warps' maxima through s_warp[NT/32] and one more warp of shuffles.  The
// result is valid in thread 0; every thread of the CTA must call it.
template <int NT>
__device__ __forceinline__ double block_max(double v, double* s_warp) {
  constexpr int WL = NT < 32 ? NT : 32;
  constexpr unsigned mask = WL == 32 ? 0xffffffffu : ((1u << WL) - 1u);
#pragma unroll
  for (int o = WL / 2; o > 0; o >>= 1) v = max_nonneg(v, __shfl_xor_sync(mask, v, o));
  if constexpr (NT > 32) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
      v = lane < NW ? s_warp[lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = max_nonneg(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
  }
  return v;
}

// Signal-speed sum of one cell for the CFL rule; W from cons_to_prim and
// ir = 1 / W[0] (cons_to_prim_ir returns it).
__device__ __forceinline__ double signal_speed_ir(const double W[5], double ir, const Eos& e, double idx,
                                                  double idy, double idz, bool dim3) {
  const Rk& k = e.k;
  const double c = sqrt_nr(mul(mul(e.gamma, W[4], k), ir, k), k);
  // sum_d (|u_d| + c) / dx_d = c (1/dx + 1/dy [+ 1/dz]) + |u| / dx + |v| / dy [+ |w| / dz]
  const double isum = dim3 ? add(add(idx, idy, k), idz, k) : add(idx, idy, k);
  double s = fma(fabs(W[1]), idx, mul(c, isum, k));
  s = fma(fabs(W[2]), idy, s);
  if (dim3) s = fma(fabs(W[3]), idz, s);
  return s;
}

// calcFlux role: HLLC flux through a face whose normal is the first velocity
// component of the rotated states WL (low side) and WR (high side):
// W = (rho, u_n, u_t1, u_t2, p).  F is returned in the same rotated order.
//
// Wave speeds: S_L = min(u_L - c_L, u~ - c~), S_R = max(u_R + c_R, u~ + c~)
// with Roe averages (sqrt(rho) weights); contact speed
// S* = (p_R - p_L + m_L u_L - m_R u_R) / (m_L - m_R), m_K = rho_K (S_K - u_K).
// Side K = L when S* >= 0, else R.  With delta = (S* - u_K) / (S_K - S*),
// Toro's star state satisfies
//   U*_K - U_K = delta [rho_K, rho_K S_K, rho_K v_K, rho_K w_K, h_K + m_K S*]
// (h = E + p), so F = F_K + S_K (U*_K - U_K) becomes, with g = S_K delta and
// t = u_K + g,
//   F0 = rho_K t,  F1 = F0 u_K + p_K + g m_K,  F2 = v_K F0,  F3 = w_K F0,
//   F4 = h_K t + g m_K S*.
// When the whole fan lies on one side (S_L >= 0, or S_R <= 0) g = 0 and
// F = F_K; otherwise t = u_K + g = S* (S_K - u_K) / (S_K - S*).
//
// The Roe averages are evaluated in an algebraically equal form with fewer
// FP64 operations.  One reciprocal square root q = 1/sqrt(rho_L rho_R) gives
// c_L^2 = gamma p_L / rho_L = p_L rho_R (gamma q^2), c_R^2 = p_R rho_L (gamma q^2)
// and r = sqrt(rho_R / rho_L) = rho_R q; the weights are w_L = 1 / (1 + r),
// w_R = r w_L; and, because H_K = c_K^2 / (gamma-1) + |u_K|^2 / 2 and
// w_L + w_R = 1,
//   c~^2 = (gamma-1) (H~ - |u~|^2 / 2) = w_L c_L^2 + w_R c_R^2
//          + (gamma-1)/2 w_L w_R |u_L - u_R|^2
//        = w_L c_L^2 + w_R (c_R^2 + (gamma-1)/2 w_L |u_L - u_R|^2),
// a sum of non-negative terms (no cancellation at high Mach number), so the
// transverse Roe velocities and H~ are not formed.  h_K is formed for the
// chosen side only, and u~ = u_L - w_R (u_L - u_R).  80 FP64 operations per face.
__device__ __forceinline__ void hllc_flux(const double WL[5], const double WR[5], const Eos& e,
                                          double F[5]) {
  const Rk& k = e.k;
  const double rL = WL[0], uL = WL[1], vL = WL[2], wL = WL[3], pL = WL[4];
  const double rR = WR[0], uR = WR[1], vR = WR[2], wR = WR[3], pR = WR[4];

  const double q = rsqrt_nr(mul(rL, rR, k), k);          // 1/sqrt(rho_L rho_R)
  const double gq2 = mul(mul(e.gamma, q, k), q, k);        // gamma / (rho_L rho_R)
  const double cL2 = mul(mul(pL, rR, k), gq2, k), cR2 = mul(mul(pR, rL, k), gq2, k);   // c^2
  const double cL = sqrt_nr(cL2, k), cR = sqrt_nr(cR2, k);

  const double r = mul(rR, q, k);                          // sqrt(rho_R / rho_L)
  const double wl = rcp_nr(add(r, k.one, k), k), wr = mul(r, wl, k);   // Roe weights
  const double du = sub(uL, uR, k), dv = sub(vL, vR, k), dw = sub(wL, wR, k);
  const double ut = fma(-wr, du, uL);                      // w_L u_L + w_R u_R
  const double du2 = fma(dw, dw, fma(dv, dv, mul(du, du, k)));
  const double ct = sqrt_nr(fma(wl, cL2, mul(wr, fma(mul(e.hgm1, wl, k), du2, cR2), k)), k);

  const double SL = min_d(sub(uL, cL, k), sub(ut, ct, k));
  const double SR = max_d(add(uR, cR, k), add(ut, ct, k));
  const double dL = sub(SL, uL, k), dR = sub(SR, uR, k);
  const double mL = mul(rL, dL, k), mR = mul(rR, dR, k);
  const double Ss = mul(fma(-mR, uR, fma(mL, uL, sub(pR, pL, k))), rcp_nr(sub(mL, mR, k), k), k);

  const bool left = ge0(Ss);
  const double rK = sel(left, rL, rR), uK = sel(left, uL, uR), vK = sel(left, vL, vR);
  const double wK = sel(left, wL, wR), pK = sel(left, pL, pR);
  const double SK = sel(left, SL, SR), mK = sel(left, mL, mR), dK = sel(left, dL, dR);
  const bool fan = left ? lt0(SL) : gt0(SR);

  // t = u_K + g; S_K - S* != 0 inside the fan, and t = u_K (g = 0) outside it
  const double t = sel(fan, mul(Ss, mul(dK, rcp_nr(sub(SK, Ss, k), k), k), k), uK);
  const double g = sub(t, uK, k);
  // E + p of the chosen side (rho >= small_rho, a normal number)
  const double hK = fma(half_pos(rK), fma(wK, wK, fma(vK, vK, mul(uK, uK, k))), mul(e.g_gm1, pK, k));
  const double gm = mul(g, mK, k);
  F[0] = mul(rK, t, k);
  F[1] = add(fma(F[0], uK, pK), gm, k);
  F[2] = mul(vK, F[0], k);
  F[3] = mul(wK, F[0], k);
  F[4] = fma(hK, t, mul(gm, Ss, k));
}

}  // namespace gbh
