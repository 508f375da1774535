/*
 * hydro_oracle.cpp -- plain FP64 CPU oracle of the block-structured Euler
 * update (guard-cell fill, MC-limited PLM, HLLC, SSP-RK2, CFL time step).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference legs load this library.  It shares no code with the
 * CUDA library (paper_2401_03378_gb300/) and neither side includes the other.
 *
 * What it follows (paper sections; the numerics the paper leaves open are
 * read as stated in oracle_pointwise.h):
 *   - Sec. 2.2: the domain is split into equal blocks, each surrounded by a
 *     halo of guard cells.
 *   - Sec. 4.2, non-telescoping SSP-RK listing: before every RK stage the
 *     guard cells are filled, then every block runs the intra-stage subgraph.
 *   - Alg. "Block initializations" / "Intra stage calculations":
 *     initSoln (keep U^n for the RK combine), calcLims (reconstruction),
 *     calcFlux (face fluxes), updSoln (flux-difference update), calcEos.
 *   - SSP-RK2 (Shu-Osher): U1 = U^n + dt L(U^n);
 *     U^{n+1} = 1/2 U^n + 1/2 (U1 + dt L(U1)); dt is computed from U^n.
 *
 * Layout: U[b][v][k][j][i] (x fastest), padded with ng guard cells per side in
 * x and y (and z in 3-D).  Blocks are numbered lexicographically, x fastest.
 * Neighbours are derived here from the lattice description (the CUDA side
 * receives an explicit neighbour table instead).
 *
 * Build: g++ -O2 -ffp-contract=off -fopenmp -shared -fPIC (see build_oracle.py).
 * The only parallelism is one OpenMP loop over blocks per pass; results do not
 * depend on the thread count.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle_pointwise.h"

extern "C" {
struct OrcGrid {
  int ndim;          /* 2 or 3 */
  int nb[3];         /* blocks per dimension (nb[2] = 1 in 2-D) */
  int n[3];          /* interior cells per block per dimension (n[2] = 1 in 2-D) */
  int ng;            /* guard cells per side: x, y, and z in 3-D */
  int periodic[3];   /* 1 periodic, 0 outflow (zero-gradient) per dimension */
  double dx[3];      /* cell widths */
  double gamma, cfl, small_rho, small_p;
};
}

namespace {

using ll = long long;

struct Geo {
  int ndim;
  int nb[3], n[3], g[3], p[3];
  int periodic[3];
  ll cells;  /* padded cells per block */
  explicit Geo(const OrcGrid& G) {
    ndim = G.ndim;
    for (int d = 0; d < 3; ++d) {
      nb[d] = G.nb[d];
      n[d] = G.n[d];
      g[d] = (d < ndim) ? G.ng : 0;
      p[d] = n[d] + 2 * g[d];
      periodic[d] = G.periodic[d];
    }
    cells = (ll)p[0] * p[1] * p[2];
  }
  ll nblocks() const { return (ll)nb[0] * nb[1] * nb[2]; }
  ll at(ll b, int v, int k, int j, int i) const {
    return (((b * 5 + v) * p[2] + k) * p[1] + j) * (ll)p[0] + i;
  }
  ll cell(int k, int j, int i) const { return ((ll)k * p[1] + j) * p[0] + i; }
  void coords(ll b, int c[3]) const {
    c[0] = (int)(b % nb[0]);
    c[1] = (int)((b / nb[0]) % nb[1]);
    c[2] = (int)(b / ((ll)nb[0] * nb[1]));
  }
  /* Block at lattice offset o from b, or -1 outside a non-periodic edge. */
  ll neighbour(ll b, const int o[3]) const {
    int c[3];
    coords(b, c);
    for (int d = 0; d < 3; ++d) {
      c[d] += o[d];
      if (c[d] < 0 || c[d] >= nb[d]) {
        if (!periodic[d]) return -1;
        c[d] = (c[d] + nb[d]) % nb[d];
      }
    }
    return c[0] + (ll)nb[0] * (c[1] + (ll)nb[1] * c[2]);
  }
  /* Index range of region o (-1 low guards, 0 interior, +1 high guards). */
  void range(int d, int o, int& lo, int& hi) const {
    if (o < 0) { lo = 0; hi = g[d]; }
    else if (o == 0) { lo = g[d]; hi = g[d] + n[d]; }
    else { lo = g[d] + n[d]; hi = p[d]; }
  }
};

/* fill_guardcells (Sec. 4.2): guard regions from neighbour interiors, then
 * zero-gradient (outflow) edges dimension by dimension, x then y then z, so
 * that edge and corner guards at the domain boundary are also defined. */
void fill_guardcells(const OrcGrid& G, double* U) {
  const Geo geo(G);
  const ll nbk = geo.nblocks();
  const int oz_lo = geo.ndim == 3 ? -1 : 0, oz_hi = geo.ndim == 3 ? 1 : 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (ll b = 0; b < nbk; ++b) {
    for (int oz = oz_lo; oz <= oz_hi; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (ox == 0 && oy == 0 && oz == 0) continue;
          const int o[3] = {ox, oy, oz};
          const ll nbr = geo.neighbour(b, o);
          if (nbr < 0) continue;
          int lo[3], hi[3];
          for (int d = 0; d < 3; ++d) geo.range(d, o[d], lo[d], hi[d]);
          for (int v = 0; v < 5; ++v)
            for (int k = lo[2]; k < hi[2]; ++k)
              for (int j = lo[1]; j < hi[1]; ++j)
                for (int i = lo[0]; i < hi[0]; ++i)
                  U[geo.at(b, v, k, j, i)] =
                      U[geo.at(nbr, v, k - oz * geo.n[2], j - oy * geo.n[1], i - ox * geo.n[0])];
        }
  }
  for (int d = 0; d < geo.ndim; ++d) {
    if (geo.periodic[d]) continue;
#pragma omp parallel for schedule(dynamic, 1)
    for (ll b = 0; b < nbk; ++b) {
      int c[3];
      geo.coords(b, c);
      for (int side = 0; side < 2; ++side) {
        const bool edge = side == 0 ? c[d] == 0 : c[d] == geo.nb[d] - 1;
        if (!edge) continue;
        const int src = side == 0 ? geo.g[d] : geo.g[d] + geo.n[d] - 1;
        const int glo = side == 0 ? 0 : geo.g[d] + geo.n[d];
        const int ghi = side == 0 ? geo.g[d] : geo.p[d];
        for (int v = 0; v < 5; ++v)
          for (int k = 0; k < geo.p[2]; ++k)
            for (int j = 0; j < geo.p[1]; ++j)
              for (int i = 0; i < geo.p[0]; ++i) {
                int idx[3] = {i, j, k};
                if (idx[d] < glo || idx[d] >= ghi) continue;
                int s[3] = {i, j, k};
                s[d] = src;
                U[geo.at(b, v, k, j, i)] = U[geo.at(b, v, s[2], s[1], s[0])];
              }
      }
    }
  }
}

void load_cons(const Geo& geo, const double* U, ll b, int k, int j, int i, double u5[5]) {
  for (int v = 0; v < 5; ++v) u5[v] = U[geo.at(b, v, k, j, i)];
}

/* CFL time step: dt = cfl / max over interior cells of all blocks of the
 * signal-speed sum (|u|+c)/dx + (|v|+c)/dy [+ (|w|+c)/dz]. */
double compute_dt(const OrcGrid& G, const double* U) {
  const Geo geo(G);
  const double idx = 1.0 / G.dx[0], idy = 1.0 / G.dx[1], idz = 1.0 / G.dx[2];
  double smax = 0.0;
  const ll nbk = geo.nblocks();
#pragma omp parallel for schedule(dynamic, 1) reduction(max : smax)
  for (ll b = 0; b < nbk; ++b)
    for (int k = geo.g[2]; k < geo.g[2] + geo.n[2]; ++k)
      for (int j = geo.g[1]; j < geo.g[1] + geo.n[1]; ++j)
        for (int i = geo.g[0]; i < geo.g[0] + geo.n[0]; ++i) {
          double u5[5], W[5];
          load_cons(geo, U, b, k, j, i, u5);
          orc::prim_from_cons(u5, G.gamma, G.small_rho, G.small_p, W);
          const double s = orc::signal_speed(geo.ndim, W, G.gamma, idx, idy, idz);
          smax = std::max(smax, s);
        }
  return G.cfl / smax;
}

struct Work {
  std::vector<double> W, Qm[3], Qp[3], F[3];
  std::vector<unsigned char> need;
  void resize(ll cells) {
    W.assign(5 * cells, 0.0);
    need.assign(cells, 0);
    for (int d = 0; d < 3; ++d) {
      Qm[d].assign(5 * cells, 0.0);
      Qp[d].assign(5 * cells, 0.0);
      F[d].assign(5 * cells, 0.0);
    }
  }
};

bool inside(const Geo& geo, int d, int x) { return x >= geo.g[d] && x < geo.g[d] + geo.n[d]; }

/* One block's intra-stage calculation (Alg. "Intra stage calculations"):
 * calcEos on the cells the stencil reads, calcLims, calcFlux, updSoln.
 * Uin must have its guard cells filled.  Returns floor hits on interior cells. */
ll stage_block(const OrcGrid& G, const Geo& geo, ll b, const double* Uin, const double* Un,
               double* Uout, double dt, double a, double bc, Work& w) {
  const ll cells = geo.cells;
  const int nd = geo.ndim;
  ll hits = 0;
  /* cells read by the face stencil: the interior plus a 2-deep slab across
   * each face (edges and corners are never read) */
  for (int k = 0; k < geo.p[2]; ++k)
    for (int j = 0; j < geo.p[1]; ++j)
      for (int i = 0; i < geo.p[0]; ++i) {
        const int x[3] = {i, j, k};
        int out = 0, far = 0;
        for (int d = 0; d < 3; ++d) {
          if (!inside(geo, d, x[d])) {
            ++out;
            const int dist = x[d] < geo.g[d] ? geo.g[d] - x[d] : x[d] - (geo.g[d] + geo.n[d]) + 1;
            if (dist > 2) far = 1;
          }
        }
        const ll c = geo.cell(k, j, i);
        w.need[c] = (out == 0 || (out == 1 && !far)) ? 1 : 0;
        if (!w.need[c]) continue;
        double u5[5], W5[5];
        load_cons(geo, Uin, b, k, j, i, u5);
        const int hit = orc::prim_from_cons(u5, G.gamma, G.small_rho, G.small_p, W5);
        if (out == 0) hits += hit;
        for (int v = 0; v < 5; ++v) w.W[v * cells + c] = W5[v];
      }

  const ll stride[3] = {1, geo.p[0], (ll)geo.p[0] * geo.p[1]};
  /* calcLims: MC slopes and face states, per dimension, on the interior and
   * one cell across each face */
  for (int d = 0; d < nd; ++d)
    for (int k = 0; k < geo.p[2]; ++k)
      for (int j = 0; j < geo.p[1]; ++j)
        for (int i = 0; i < geo.p[0]; ++i) {
          const int x[3] = {i, j, k};
          bool ok = x[d] >= geo.g[d] - 1 && x[d] <= geo.g[d] + geo.n[d];
          for (int e = 0; e < 3; ++e)
            if (e != d && !inside(geo, e, x[e])) ok = false;
          if (!ok) continue;
          const ll c = geo.cell(k, j, i);
          for (int v = 0; v < 5; ++v) {
            const double* q = &w.W[v * cells];
            const double s = orc::mc_slope(q[c - stride[d]], q[c], q[c + stride[d]]);
            w.Qm[d][v * cells + c] = q[c] - 0.5 * s;
            w.Qp[d][v * cells + c] = q[c] + 0.5 * s;
          }
        }

  /* calcFlux: HLLC at every face of the interior, F[d][c] is the flux through
   * the face between c - e_d and c */
  for (int d = 0; d < nd; ++d) {
    /* velocity components in the rotated frame: normal, then the other two */
    const int t1 = d == 0 ? 2 : 1, t2 = d == 2 ? 2 : 3;
    const int vmap[5] = {0, 1 + d, t1, t2, 4};
    for (int k = 0; k < geo.p[2]; ++k)
      for (int j = 0; j < geo.p[1]; ++j)
        for (int i = 0; i < geo.p[0]; ++i) {
          const int x[3] = {i, j, k};
          bool ok = x[d] >= geo.g[d] && x[d] <= geo.g[d] + geo.n[d];
          for (int e = 0; e < 3; ++e)
            if (e != d && !inside(geo, e, x[e])) ok = false;
          if (!ok) continue;
          const ll c = geo.cell(k, j, i);
          double WL[5], WR[5], Fr[5];
          for (int q = 0; q < 5; ++q) {
            WL[q] = w.Qp[d][vmap[q] * cells + c - stride[d]];
            WR[q] = w.Qm[d][vmap[q] * cells + c];
          }
          orc::hllc(WL, WR, G.gamma, Fr);
          for (int q = 0; q < 5; ++q) w.F[d][vmap[q] * cells + c] = Fr[q];
        }
  }

  /* updSoln + RK combine on the interior */
  const double idx = 1.0 / G.dx[0], idy = 1.0 / G.dx[1], idz = 1.0 / G.dx[2];
  for (int k = geo.g[2]; k < geo.g[2] + geo.n[2]; ++k)
    for (int j = geo.g[1]; j < geo.g[1] + geo.n[1]; ++j)
      for (int i = geo.g[0]; i < geo.g[0] + geo.n[0]; ++i) {
        const ll c = geo.cell(k, j, i);
        for (int v = 0; v < 5; ++v) {
          const ll o = v * cells + c;
          const double fzm = nd == 3 ? w.F[2][o] : 0.0;
          const double fzp = nd == 3 ? w.F[2][o + stride[2]] : 0.0;
          const double L = orc::flux_divergence(nd, w.F[0][o], w.F[0][o + 1], w.F[1][o],
                                                w.F[1][o + stride[1]], fzm, fzp, idx, idy, idz);
          const ll gi = geo.at(b, v, k, j, i);
          const double un = Un ? Un[gi] : 0.0;
          Uout[gi] = orc::rk_combine(Uin[gi], un, L, dt, a, bc);
        }
      }
  return hits;
}

ll stage(const OrcGrid& G, const double* Uin, const double* Un, double* Uout, double dt, double a,
         double bc, const ll* blocks, ll nlist) {
  const Geo geo(G);
  const ll count = blocks ? nlist : geo.nblocks();
  ll hits = 0;
#pragma omp parallel reduction(+ : hits)
  {
    Work w;
    w.resize(geo.cells);
#pragma omp for schedule(dynamic, 1)
    for (ll t = 0; t < count; ++t) {
      const ll b = blocks ? blocks[t] : t;
      hits += stage_block(G, geo, b, Uin, Un, Uout, dt, a, bc, w);
    }
  }
  return hits;
}

/* One SSP-RK2 step in place (non-telescoping: fill before every stage). */
ll step(const OrcGrid& G, double* U, double dt) {
  const Geo geo(G);
  const ll total = geo.nblocks() * 5 * geo.cells;
  std::vector<double> U1(U, U + total), U2(total);
  ll hits = 0;
  fill_guardcells(G, U);
  hits += stage(G, U, nullptr, U1.data(), dt, 0.0, 1.0, nullptr, 0);
  fill_guardcells(G, U1.data());
  std::memcpy(U2.data(), U1.data(), total * sizeof(double));
  hits += stage(G, U1.data(), U, U2.data(), dt, 0.5, 0.5, nullptr, 0);
  /* copy the new interior back; guard cells keep the values of the first fill */
  for (ll b = 0; b < geo.nblocks(); ++b)
    for (int v = 0; v < 5; ++v)
      for (int k = geo.g[2]; k < geo.g[2] + geo.n[2]; ++k)
        for (int j = geo.g[1]; j < geo.g[1] + geo.n[1]; ++j)
          for (int i = geo.g[0]; i < geo.g[0] + geo.n[0]; ++i) {
            const ll o = geo.at(b, v, k, j, i);
            U[o] = U2[o];
          }
  return hits;
}

}  // namespace

extern "C" {

int orc_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int orc_prim(const double* U5, double gamma, double small_rho, double small_p, double* W5) {
  return orc::prim_from_cons(U5, gamma, small_rho, small_p, W5);
}

double orc_mc_slope(double qm, double q0, double qp) { return orc::mc_slope(qm, q0, qp); }

void orc_euler_flux(const double* W5, double gamma, double* F5) {
  orc::euler_flux(W5, orc::total_energy(W5, gamma), F5);
}

/* detail layout (double[69]): SL, SR, Ss, region, UL[5], UR[5], FL[5], FR[5],
 * UsL[5], UsR[5], FsL[5], FsR[5], F[5] ... (see oracle.py) */
void orc_hllc(const double* WL, const double* WR, double gamma, double* F5, double* detail) {
  if (!detail) {
    orc::hllc(WL, WR, gamma, F5);
    return;
  }
  orc::HllcDetail<double> d;
  orc::hllc(WL, WR, gamma, F5, &d);
  double* o = detail;
  *o++ = d.SL; *o++ = d.SR; *o++ = d.Ss; *o++ = (double)d.region;
  const double* arrs[9] = {d.UL, d.UR, d.FL, d.FR, d.UsL, d.UsR, d.FsL, d.FsR, d.F};
  for (int a = 0; a < 9; ++a)
    for (int q = 0; q < 5; ++q) *o++ = arrs[a][q];
}

void orc_fill_guardcells(const OrcGrid* G, double* U) { fill_guardcells(*G, U); }

double orc_compute_dt(const OrcGrid* G, const double* U) { return compute_dt(*G, U); }

/* Uout = a*Un + b*(Uin + dt*L(Uin)) on the interior of every block (or of the
 * listed blocks).  Uin's guard cells must be filled; Un may be NULL when a = 0.
 * Returns the number of floor hits on interior cells. */
long long orc_stage(const OrcGrid* G, const double* Uin, const double* Un, double* Uout, double dt,
                    double a, double b, const long long* blocks, long long nlist) {
  return stage(*G, Uin, Un, Uout, dt, a, b, blocks, nlist);
}

long long orc_step(const OrcGrid* G, double* U, double dt) { return step(*G, U, dt); }

/* nsteps SSP-RK2 steps, each with dt = compute_dt(U^n); dt_hist[s] receives dt. */
long long orc_run(const OrcGrid* G, double* U, int nsteps, double* dt_hist) {
  long long hits = 0;
  for (int s = 0; s < nsteps; ++s) {
    const double dt = compute_dt(*G, U);
    if (dt_hist) dt_hist[s] = dt;
    hits += step(*G, U, dt);
  }
  return hits;
}

}  // extern "C"
