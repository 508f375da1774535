// gbh_device.cuh -- per-cell and per-face FP64 arithmetic of the stage kernel.
//
// The intra-stage calculations of the paper's hydrodynamics variants
// (Sec. 4.2, Alg. "Intra stage calculations for Spark") are calcLims
// (reconstruction), calcFlux (face fluxes), updSoln (flux-difference update)
// and calcEos (equation of state).  The numerics they leave open are read as:
// ideal-gas EOS with floors, MC-limited piecewise-linear reconstruction of
// primitive variables, and the HLLC flux (Toro's star state, Einfeldt /
// Roe-average wave-speed bounds).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbh_internal.h"

namespace gbh {

// calcEos role: conserved (rho, mx, my, mz, E) -> primitive (rho, u, v, w, p).
// Floors rho at small_rho and p at small_p; returns 1 when a floor applied.
__device__ __forceinline__ int cons_to_prim(const double U[5], double W[5], const Eos& e) {
  int hit = 0;
  double rho = U[0];
  if (rho < e.small_rho) { rho = e.small_rho; hit = 1; }
  const double ir = 1.0 / rho;
  const double u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
  const double ek = 0.5 * (U[1] * u + U[2] * v + U[3] * w);
  double p = e.gm1 * (U[4] - ek);
  if (p < e.small_p) { p = e.small_p; hit = 1; }
  W[0] = rho; W[1] = u; W[2] = v; W[3] = w; W[4] = p;
  return hit;
}

// calcLims role: half of the MC-limited slope at q0,
//   sigma/2 = sign(dp) * min(|dm+dp|/4, |dm|, |dp|) if dm, dp have the same strict sign, else 0,
// so that the face values are q0 -/+ sigma/2.
__device__ __forceinline__ double mc_half_slope(double qm, double q0, double qp) {
  const double dm = q0 - qm;
  const double dp = qp - q0;
  const double h = fmin(0.25 * fabs(dm + dp), fmin(fabs(dm), fabs(dp)));
  return (dm * dp > 0.0) ? copysign(h, dp) : 0.0;
}

// Signal-speed sum of one cell for the CFL rule.
__device__ __forceinline__ double signal_speed(const double W[5], const Eos& e, double idx,
                                               double idy, double idz, bool dim3) {
  const double c = sqrt(e.gamma * W[4] / W[0]);
  double s = (fabs(W[1]) + c) * idx + (fabs(W[2]) + c) * idy;
  if (dim3) s += (fabs(W[3]) + c) * idz;
  return s;
}

// calcFlux role: HLLC flux through a face whose normal is the first velocity
// component of the rotated states WL (low side) and WR (high side):
// W = (rho, u_n, u_t1, u_t2, p).  F is returned in the same rotated order.
//
// Region choice follows the sign of the contact speed S*: side K = L when
// S* >= 0, else R.  The flux is F_K + S_K (U*_K - U_K), with the correction
// switched off (coefficient exactly 0) when the whole fan lies on one side
// (S_L >= 0 or S_R <= 0), which then returns F_K exactly.
__device__ __forceinline__ void hllc_flux(const double WL[5], const double WR[5], const Eos& e,
                                          double F[5]) {
  const double rL = WL[0], uL = WL[1], vL = WL[2], wL = WL[3], pL = WL[4];
  const double rR = WR[0], uR = WR[1], vR = WR[2], wR = WR[3], pR = WR[4];

  const double EL = pL * e.inv_gm1 + 0.5 * rL * (uL * uL + vL * vL + wL * wL);
  const double ER = pR * e.inv_gm1 + 0.5 * rR * (uR * uR + vR * vR + wR * wR);
  const double cL = sqrt(e.gamma * pL / rL);
  const double cR = sqrt(e.gamma * pR / rR);

  // Roe averages (sqrt(rho) weights)
  const double sL = sqrt(rL), sR = sqrt(rR);
  const double inv = 1.0 / (sL + sR);
  const double HL = (EL + pL) / rL, HR = (ER + pR) / rR;
  const double ut = (sL * uL + sR * uR) * inv;
  const double vt = (sL * vL + sR * vR) * inv;
  const double wt = (sL * wL + sR * wR) * inv;
  const double Ht = (sL * HL + sR * HR) * inv;
  const double ct = sqrt(e.gm1 * (Ht - 0.5 * (ut * ut + vt * vt + wt * wt)));

  const double SL = fmin(uL - cL, ut - ct);
  const double SR = fmax(uR + cR, ut + ct);
  const double mL = rL * (SL - uL);
  const double mR = rR * (SR - uR);
  const double Ss = (pR - pL + mL * uL - mR * uR) / (mL - mR);

  const bool left = Ss >= 0.0;
  const double rK = left ? rL : rR, uK = left ? uL : uR, vK = left ? vL : vR, wK = left ? wL : wR;
  const double pK = left ? pL : pR, EK = left ? EL : ER, SK = left ? SL : SR, mK = left ? mL : mR;
  const bool fan = left ? (SL < 0.0) : (SR > 0.0);

  const double mass = rK * uK;
  const double FK0 = mass, FK1 = mass * uK + pK, FK2 = mass * vK, FK3 = mass * wK;
  const double FK4 = uK * (EK + pK);

  const double fac = mK / (SK - Ss);
  const double es = EK / rK + (Ss - uK) * (Ss + pK / mK);
  const double coef = fan ? SK : 0.0;
  F[0] = FK0 + coef * (fac - rK);
  F[1] = FK1 + coef * (fac * Ss - mass);
  F[2] = FK2 + coef * (fac * vK - rK * vK);
  F[3] = FK3 + coef * (fac * wK - rK * wK);
  F[4] = FK4 + coef * (fac * es - EK);
}

}  // namespace gbh
