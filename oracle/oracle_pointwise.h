/*
 * oracle_pointwise.h -- pointwise arithmetic of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE.  The oracle is a plain, slow, obviously-correct CPU
 * statement of the per-block Euler update whose variants the paper generates
 * (Sec. 4.2, Alg. "Intra stage calculations for Spark": calcLims -> calcFlux
 * -> updSoln -> calcEos).  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference legs may use it.  It shares no code with the CUDA
 * library in paper_2401_03378_gb300/ and neither side includes the other.
 *
 * Every function is a template on the scalar type T so that the same source
 * can be instantiated with `double` (the oracle) and with an op-counting type
 * (opcount.cpp) that measures the algorithmic flop count.  Arithmetic is
 * written in the order stated below; the oracle library is compiled with
 * -ffp-contract=off so that no fused multiply-add changes it.
 *
 * The paper names the stages (calcLims, calcFlux, updSoln, calcEos) but not
 * the numerics.  The readings used here:
 *   - reconstruction: piecewise-linear in primitive variables with the
 *     monotonized-central (MC) limiter;
 *   - Riemann solver: HLLC (Toro, Riemann Solvers and Numerical Methods for
 *     Fluid Dynamics, 3rd ed., Sec. 10.4) with Einfeldt / Roe-average wave
 *     speeds (Batten et al. 1997) and the star state of Toro eq. (10.39);
 *   - EOS: ideal gas, p = (gamma-1)(E - rho|u|^2/2), with floors small_rho,
 *     small_p applied only when converting conserved -> primitive.
 */
#pragma once

#include <cmath>

namespace orc {

template <class T> inline T tmin(T a, T b) { return b < a ? b : a; }
template <class T> inline T tmax(T a, T b) { return a < b ? b : a; }
template <class T> inline T tabs(T a) { return a < T(0) ? -a : a; }

/* Conserved (rho, m_x, m_y, m_z, E) -> primitive (rho, u, v, w, p); the
 * calcEos role of Alg. "Intra stage calculations".  Returns 1 when a floor
 * was applied. */
template <class T>
inline int prim_from_cons(const T U[5], T gamma, T small_rho, T small_p, T W[5]) {
  using std::sqrt;
  int hit = 0;
  T rho = U[0];
  if (rho < small_rho) { rho = small_rho; hit = 1; }
  T u = U[1] / rho;
  T v = U[2] / rho;
  T w = U[3] / rho;
  T ekin = T(0.5) * rho * (u * u + v * v + w * w);
  T p = (gamma - T(1)) * (U[4] - ekin);
  if (p < small_p) { p = small_p; hit = 1; }
  W[0] = rho; W[1] = u; W[2] = v; W[3] = w; W[4] = p;
  return hit;
}

/* Monotonized-central limited slope of q at the middle of three cells
 * (calcLims role).  sigma = 0 when the one-sided differences do not have the
 * same strict sign; otherwise sign * min(|dm+dp|/2, 2|dm|, 2|dp|). */
template <class T>
inline T mc_slope(T qm, T q0, T qp) {
  T dm = q0 - qm;
  T dp = qp - q0;
  if (dm * dp <= T(0)) return T(0);
  T a = T(0.5) * tabs(dm + dp);
  T b = T(2) * tabs(dm);
  T c = T(2) * tabs(dp);
  T s = tmin(a, tmin(b, c));
  return dp > T(0) ? s : -s;
}

/* Physical Euler flux along the normal of a face, in the rotated frame
 * W = (rho, u_n, u_t1, u_t2, p) with total energy E. */
template <class T>
inline void euler_flux(const T W[5], T E, T F[5]) {
  T mass = W[0] * W[1];
  F[0] = mass;
  F[1] = mass * W[1] + W[4];
  F[2] = mass * W[2];
  F[3] = mass * W[3];
  F[4] = W[1] * (E + W[4]);
}

template <class T>
inline T total_energy(const T W[5], T gamma) {
  return W[4] / (gamma - T(1)) + T(0.5) * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
}

/* Everything HLLC computes for one face, for the tests that check the star
 * states against the Rankine-Hugoniot / consistency relations. */
template <class T>
struct HllcDetail {
  T SL, SR, Ss;
  T UL[5], UR[5], FL[5], FR[5];
  T UsL[5], UsR[5], FsL[5], FsR[5];
  T F[5];
  int region;  /* 0: F_L, 1: F*_L, 2: F*_R, 3: F_R */
};

/* Star state of side K (Toro eq. 10.39): rho_K (S_K - u_K)/(S_K - S*) times
 * [1, S*, v_K, w_K, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))]. */
template <class T>
inline void hllc_star(const T W[5], T E, T S, T Ss, T Us[5]) {
  T m = W[0] * (S - W[1]);
  T fac = m / (S - Ss);
  Us[0] = fac;
  Us[1] = fac * Ss;
  Us[2] = fac * W[2];
  Us[3] = fac * W[3];
  Us[4] = fac * (E / W[0] + (Ss - W[1]) * (Ss + W[4] / m));
}

/* HLLC flux across a face whose normal is the first velocity component
 * (calcFlux role).  W_L is the state on the low side, W_R on the high side. */
template <class T>
inline void hllc(const T WL[5], const T WR[5], T gamma, T F[5], HllcDetail<T>* d = nullptr) {
  using std::sqrt;
  const T rL = WL[0], uL = WL[1], vL = WL[2], wL = WL[3], pL = WL[4];
  const T rR = WR[0], uR = WR[1], vR = WR[2], wR = WR[3], pR = WR[4];
  const T gm1 = gamma - T(1);

  const T EL = total_energy(WL, gamma);
  const T ER = total_energy(WR, gamma);
  const T cL = sqrt(gamma * pL / rL);
  const T cR = sqrt(gamma * pR / rR);
  const T HL = (EL + pL) / rL;
  const T HR = (ER + pR) / rR;

  /* Roe averages with weights sqrt(rho) */
  const T sL = sqrt(rL);
  const T sR = sqrt(rR);
  const T inv = T(1) / (sL + sR);
  const T ut = (sL * uL + sR * uR) * inv;
  const T vt = (sL * vL + sR * vR) * inv;
  const T wt = (sL * wL + sR * wR) * inv;
  const T Ht = (sL * HL + sR * HR) * inv;
  const T ct = sqrt(gm1 * (Ht - T(0.5) * (ut * ut + vt * vt + wt * wt)));

  /* Einfeldt wave-speed bounds */
  const T SL = tmin(uL - cL, ut - ct);
  const T SR = tmax(uR + cR, ut + ct);

  /* contact speed (Toro eq. 10.37) */
  const T mL = rL * (SL - uL);
  const T mR = rR * (SR - uR);
  const T Ss = (pR - pL + mL * uL - mR * uR) / (mL - mR);

  T FL[5], FR[5];
  if (d) {
    euler_flux(WL, EL, d->FL);
    euler_flux(WR, ER, d->FR);
    const T UL[5] = {rL, rL * uL, rL * vL, rL * wL, EL};
    const T UR[5] = {rR, rR * uR, rR * vR, rR * wR, ER};
    hllc_star(WL, EL, SL, Ss, d->UsL);
    hllc_star(WR, ER, SR, Ss, d->UsR);
    for (int q = 0; q < 5; ++q) {
      d->UL[q] = UL[q];
      d->UR[q] = UR[q];
      d->FsL[q] = d->FL[q] + SL * (d->UsL[q] - UL[q]);
      d->FsR[q] = d->FR[q] + SR * (d->UsR[q] - UR[q]);
    }
    d->SL = SL; d->SR = SR; d->Ss = Ss;
  }

  int region;
  if (T(0) <= SL) {
    region = 0;
    euler_flux(WL, EL, F);
  } else if (T(0) <= Ss) {
    region = 1;
    euler_flux(WL, EL, FL);
    const T UL[5] = {rL, rL * uL, rL * vL, rL * wL, EL};
    T Us[5];
    hllc_star(WL, EL, SL, Ss, Us);
    for (int q = 0; q < 5; ++q) F[q] = FL[q] + SL * (Us[q] - UL[q]);
  } else if (T(0) < SR) {
    region = 2;
    euler_flux(WR, ER, FR);
    const T UR[5] = {rR, rR * uR, rR * vR, rR * wR, ER};
    T Us[5];
    hllc_star(WR, ER, SR, Ss, Us);
    for (int q = 0; q < 5; ++q) F[q] = FR[q] + SR * (Us[q] - UR[q]);
  } else {
    region = 3;
    euler_flux(WR, ER, F);
  }
  if (d) {
    d->region = region;
    for (int q = 0; q < 5; ++q) d->F[q] = F[q];
  }
}

/* Flux-difference operator L(U) of one conserved variable at one cell
 * (updSoln role), summed in the fixed order x, y, z:
 *   L = -(Fx+ - Fx-) idx;  L = L - (Fy+ - Fy-) idy;  L = L - (Fz+ - Fz-) idz. */
template <class T>
inline T flux_divergence(int ndim, T fxm, T fxp, T fym, T fyp, T fzm, T fzp, T idx, T idy, T idz) {
  T L = -(fxp - fxm) * idx;
  L = L - (fyp - fym) * idy;
  if (ndim == 3) L = L - (fzp - fzm) * idz;
  return L;
}

/* One SSP-RK stage in Shu-Osher form: out = a U^n + b (U_in + dt L).  The
 * first stage of SSP-RK2 (a = 0, b = 1) is written as U_in + dt L. */
template <class T>
inline T rk_combine(T uin, T un, T L, T dt, T a, T b) {
  if (a == T(0) && b == T(1)) return uin + dt * L;
  return a * un + b * (uin + dt * L);
}

/* Signal-speed sum of one cell for the CFL rule:
 * s = (|u|+c) idx + (|v|+c) idy [+ (|w|+c) idz]; dt = cfl / max s. */
template <class T>
inline T signal_speed(int ndim, const T W[5], T gamma, T idx, T idy, T idz) {
  using std::sqrt;
  T c = sqrt(gamma * W[4] / W[0]);
  T s = (tabs(W[1]) + c) * idx + (tabs(W[2]) + c) * idy;
  if (ndim == 3) s = s + (tabs(W[3]) + c) * idz;
  return s;
}

}  // namespace orc
