/*
 * opcount.cpp -- algorithmic FP64 operation count of the oracle's arithmetic.
 *
 * TEST INFRASTRUCTURE.  Instantiates the oracle's pointwise templates
 * (oracle_pointwise.h) with a scalar that counts +, -, *, /, sqrt as one
 * operation each (comparisons, min/max, |x| and negation are not counted) and
 * prints the count of every building block as JSON.  The per-zone total is
 * assembled from these counts with the multiplicities of an unblocked grid
 * (one primitive conversion per cell, one limited slope per cell, variable
 * and dimension, one HLLC flux per face, one update per cell and variable).
 */
#include <cmath>
#include <cstdio>

#include "oracle_pointwise.h"

struct Cnt {
  double v;
  static long long n;
  Cnt(double x = 0.0) : v(x) {}
};
long long Cnt::n = 0;

inline Cnt operator+(Cnt a, Cnt b) { ++Cnt::n; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++Cnt::n; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++Cnt::n; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++Cnt::n; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
inline bool operator<=(Cnt a, Cnt b) { return a.v <= b.v; }
inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
inline bool operator==(Cnt a, Cnt b) { return a.v == b.v; }
inline Cnt sqrt(Cnt a) { ++Cnt::n; return Cnt(std::sqrt(a.v)); }

static long long count_prim() {
  Cnt U[5] = {1.2, 0.3, -0.2, 0.1, 2.5}, W[5];
  Cnt::n = 0;
  orc::prim_from_cons<Cnt>(U, 1.4, 1e-12, 1e-14, W);
  return Cnt::n;
}

/* one limited slope plus the two face values q -/+ sigma/2 */
static long long count_slope() {
  Cnt::n = 0;
  Cnt s = orc::mc_slope<Cnt>(1.0, 1.5, 1.8);
  Cnt q = 1.5;
  Cnt qm = q - Cnt(0.5) * s;
  Cnt qp = q + Cnt(0.5) * s;
  (void)qm; (void)qp;
  return Cnt::n;
}

static long long count_hllc(double uL, double uR) {
  Cnt WL[5] = {1.0, uL, 0.1, -0.2, 1.0}, WR[5] = {0.8, uR, 0.05, 0.1, 0.7}, F[5];
  Cnt::n = 0;
  orc::hllc<Cnt>(WL, WR, 1.4, F);
  return Cnt::n;
}

static long long count_update(int ndim, bool combine) {
  Cnt::n = 0;
  Cnt L = orc::flux_divergence<Cnt>(ndim, 1.0, 1.1, 0.9, 1.2, 1.3, 1.0, 128.0, 128.0, 128.0);
  Cnt out = orc::rk_combine<Cnt>(1.0, 0.9, L, 1e-3, combine ? 0.5 : 0.0, combine ? 0.5 : 1.0);
  (void)out;
  return Cnt::n;
}

static long long count_dt(int ndim) {
  Cnt W[5] = {1.0, 0.3, -0.2, 0.1, 1.0};
  Cnt::n = 0;
  Cnt s = orc::signal_speed<Cnt>(ndim, W, 1.4, 128.0, 128.0, 128.0);
  (void)s;
  return Cnt::n;
}

int main() {
  const long long prim = count_prim();
  const long long slope = count_slope();
  const long long hllc_star = count_hllc(0.1, -0.1);   /* subsonic: star region */
  const long long hllc_super = count_hllc(5.0, 5.0);   /* supersonic: F_L */
  const long long upd3_s1 = count_update(3, false), upd3_s2 = count_update(3, true);
  const long long upd2_s1 = count_update(2, false), upd2_s2 = count_update(2, true);
  const long long dt3 = count_dt(3), dt2 = count_dt(2);
  /* per zone and stage on an unblocked 3-D grid, subsonic faces */
  const long long stage1_3d = prim + 15 * slope + 3 * hllc_star + 5 * upd3_s1;
  const long long stage2_3d = prim + 15 * slope + 3 * hllc_star + 5 * upd3_s2;
  const long long stage1_2d = prim + 10 * slope + 2 * hllc_star + 5 * upd2_s1;
  const long long stage2_2d = prim + 10 * slope + 2 * hllc_star + 5 * upd2_s2;
  std::printf(
      "{\"prim\": %lld, \"slope_and_faces\": %lld, \"hllc_star\": %lld, \"hllc_supersonic\": %lld,"
      " \"update3d_stage1\": %lld, \"update3d_stage2\": %lld, \"update2d_stage1\": %lld,"
      " \"update2d_stage2\": %lld, \"dt3d\": %lld, \"dt2d\": %lld,"
      " \"zone_stage1_3d\": %lld, \"zone_stage2_3d\": %lld, \"zone_update_3d\": %lld,"
      " \"zone_stage1_2d\": %lld, \"zone_stage2_2d\": %lld, \"zone_update_2d\": %lld}\n",
      prim, slope, hllc_star, hllc_super, upd3_s1, upd3_s2, upd2_s1, upd2_s2, dt3, dt2, stage1_3d,
      stage2_3d, stage1_3d + stage2_3d + prim + dt3, stage1_2d, stage2_2d,
      stage1_2d + stage2_2d + prim + dt2);
  return 0;
}
