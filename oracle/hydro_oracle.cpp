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
struct OrcAmr2 {
  int lo[3], hi[3];  /* bounding box of the fine region in coarse-block units, [lo, hi) per dimension */
  const unsigned char* refined;  /* [coarse blocks]: 1 where the block is refined; NULL: the whole box */
};
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

/* The box a stage updates: the interior widened by `ext` cells on each side
 * of every dimension of the problem (ext = 0: the interior). */
struct Box {
  int lo[3], hi[3];
  Box(const Geo& geo, int ext) {
    for (int d = 0; d < 3; ++d) {
      const int e = d < geo.ndim ? ext : 0;
      lo[d] = geo.g[d] - e;
      hi[d] = geo.g[d] + geo.n[d] + e;
    }
  }
  bool in(int d, int x) const { return x >= lo[d] && x < hi[d]; }
};

/* One block's intra-stage calculation (Alg. "Intra stage calculations"):
 * calcEos on the cells the stencil reads, calcLims, calcFlux, updSoln, on
 * the interior widened by `ext` cells (ext = 2: the first stage of the
 * telescoping mode of Sec. 4.2, which also updates part of the halo).
 * Uin's guard cells must hold valid data 2 cells beyond that box.  Returns
 * floor hits on interior cells. */
ll stage_block(const OrcGrid& G, const Geo& geo, ll b, const double* Uin, const double* Un,
               double* Uout, double dt, double a, double bc, Work& w, int ext = 0) {
  const ll cells = geo.cells;
  const int nd = geo.ndim;
  const Box R(geo, ext);
  ll hits = 0;
  /* cells read by the face stencil: the box plus a 2-deep slab across each
   * of its faces (the box's own edges and corners are never read) */
  for (int k = 0; k < geo.p[2]; ++k)
    for (int j = 0; j < geo.p[1]; ++j)
      for (int i = 0; i < geo.p[0]; ++i) {
        const int x[3] = {i, j, k};
        int out = 0, far = 0, interior = 1;
        for (int d = 0; d < 3; ++d) {
          if (!inside(geo, d, x[d])) interior = 0;
          if (!R.in(d, x[d])) {
            ++out;
            const int dist = x[d] < R.lo[d] ? R.lo[d] - x[d] : x[d] - R.hi[d] + 1;
            if (dist > 2) far = 1;
          }
        }
        const ll c = geo.cell(k, j, i);
        w.need[c] = (out == 0 || (out == 1 && !far)) ? 1 : 0;
        if (!w.need[c]) continue;
        double u5[5], W5[5];
        load_cons(geo, Uin, b, k, j, i, u5);
        const int hit = orc::prim_from_cons(u5, G.gamma, G.small_rho, G.small_p, W5);
        if (interior) hits += hit;
        for (int v = 0; v < 5; ++v) w.W[v * cells + c] = W5[v];
      }

  const ll stride[3] = {1, geo.p[0], (ll)geo.p[0] * geo.p[1]};
  /* calcLims: MC slopes and face states, per dimension, on the box and one
   * cell across each face */
  for (int d = 0; d < nd; ++d)
    for (int k = 0; k < geo.p[2]; ++k)
      for (int j = 0; j < geo.p[1]; ++j)
        for (int i = 0; i < geo.p[0]; ++i) {
          const int x[3] = {i, j, k};
          bool ok = x[d] >= R.lo[d] - 1 && x[d] <= R.hi[d];
          for (int e = 0; e < 3; ++e)
            if (e != d && !R.in(e, x[e])) ok = false;
          if (!ok) continue;
          const ll c = geo.cell(k, j, i);
          for (int v = 0; v < 5; ++v) {
            const double* q = &w.W[v * cells];
            const double s = orc::mc_slope(q[c - stride[d]], q[c], q[c + stride[d]]);
            w.Qm[d][v * cells + c] = q[c] - 0.5 * s;
            w.Qp[d][v * cells + c] = q[c] + 0.5 * s;
          }
        }

  /* calcFlux: HLLC at every face of the box, F[d][c] is the flux through the
   * face between c - e_d and c */
  for (int d = 0; d < nd; ++d) {
    /* velocity components in the rotated frame: normal, then the other two */
    const int t1 = d == 0 ? 2 : 1, t2 = d == 2 ? 2 : 3;
    const int vmap[5] = {0, 1 + d, t1, t2, 4};
    for (int k = 0; k < geo.p[2]; ++k)
      for (int j = 0; j < geo.p[1]; ++j)
        for (int i = 0; i < geo.p[0]; ++i) {
          const int x[3] = {i, j, k};
          bool ok = x[d] >= R.lo[d] && x[d] <= R.hi[d];
          for (int e = 0; e < 3; ++e)
            if (e != d && !R.in(e, x[e])) ok = false;
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

  /* updSoln + RK combine on the box */
  const double idx = 1.0 / G.dx[0], idy = 1.0 / G.dx[1], idz = 1.0 / G.dx[2];
  for (int k = R.lo[2]; k < R.hi[2]; ++k)
    for (int j = R.lo[1]; j < R.hi[1]; ++j)
      for (int i = R.lo[0]; i < R.hi[0]; ++i) {
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
         double bc, const ll* blocks, ll nlist, int ext = 0) {
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
      hits += stage_block(G, geo, b, Uin, Un, Uout, dt, a, bc, w, ext);
    }
  }
  return hits;
}

/* SSP-RK stages in Shu-Osher form (Sec. 4.2 names SSP-RK, multistage, no
 * order): stage s forms U(s) = a_s U^n + b_s (U(s-1) + dt L(U(s-1))), U(0) =
 * U^n, and U^{n+1} = U(S).  Two stages: (0, 1), (1/2, 1/2); three stages:
 * (0, 1), (3/4, 1/4), (1/3, 2/3). */
struct Rk {
  int S;
  double a[3], b[3];
};

Rk rk_scheme(int nstages) {
  if (nstages == 3) return Rk{3, {0.0, 0.75, 1.0 / 3.0}, {1.0, 0.25, 2.0 / 3.0}};
  return Rk{2, {0.0, 0.5, 0.0}, {1.0, 0.5, 0.0}};
}

/* the weight of dt L(U(s-1)) of stage s in U^{n+1}: b_s times the b of
 * every later stage (1/2, 1/2 for two stages; 1/6, 1/6, 2/3 for three) */
double rk_weight(const Rk& r, int s) {
  double w = r.b[s];
  for (int t = s + 1; t < r.S; ++t) w = w * r.b[t];
  return w;
}

void copy_interior(const Geo& geo, const double* src, double* dst) {
  for (ll b = 0; b < geo.nblocks(); ++b)
    for (int v = 0; v < 5; ++v)
      for (int k = geo.g[2]; k < geo.g[2] + geo.n[2]; ++k)
        for (int j = geo.g[1]; j < geo.g[1] + geo.n[1]; ++j)
          for (int i = geo.g[0]; i < geo.g[0] + geo.n[0]; ++i) {
            const ll o = geo.at(b, v, k, j, i);
            dst[o] = src[o];
          }
}

/* One SSP-RK step in place, non-telescoping (Sec. 4.2: a guard fill before
 * every stage).  The new interior is copied back; U's guard cells keep the
 * values of the first fill. */
ll step(const OrcGrid& G, double* U, double dt, int nstages = 2) {
  const Rk r = rk_scheme(nstages);
  const Geo geo(G);
  const ll total = geo.nblocks() * 5 * geo.cells;
  std::vector<double> X(U, U + total), Y(total);
  ll hits = 0;
  fill_guardcells(G, U);
  hits += stage(G, U, nullptr, X.data(), dt, r.a[0], r.b[0], nullptr, 0);
  for (int st = 1; st < r.S; ++st) {
    fill_guardcells(G, X.data());
    std::memcpy(Y.data(), X.data(), total * sizeof(double));
    hits += stage(G, X.data(), U, Y.data(), dt, r.a[st], r.b[st], nullptr, 0);
    std::swap(X, Y);
  }
  copy_interior(geo, X.data(), U);
  return hits;
}

/* One SSP-RK step in place in the telescoping mode (Sec. 4.2): one guard
 * fill, then every stage per block with no exchange in between.  Stage s of
 * S updates the interior widened by 2 (S - s) cells (the PLM face stencil
 * reaches 2 cells), so each later stage finds its input in its own guard
 * cells; the fill must supply 2 S guard cells.  Where a neighbour supplies
 * the halo this equals the non-telescoping step; at an outflow edge the
 * first stages evolve the zero-gradient copies instead of copying the
 * updated boundary cell. */
ll step_telescoping(const OrcGrid& G, double* U, double dt, int nstages = 2) {
  const Rk r = rk_scheme(nstages);
  const Geo geo(G);
  const ll total = geo.nblocks() * 5 * geo.cells;
  ll hits = 0;
  fill_guardcells(G, U);
  std::vector<double> X(U, U + total), Y(U, U + total);
  hits += stage(G, U, nullptr, X.data(), dt, r.a[0], r.b[0], nullptr, 0, 2 * (r.S - 1));
  for (int st = 1; st < r.S; ++st) {
    hits += stage(G, X.data(), U, Y.data(), dt, r.a[st], r.b[st], nullptr, 0, 2 * (r.S - 1 - st));
    std::swap(X, Y);
  }
  copy_interior(geo, X.data(), U);
  return hits;
}

// ---------------------------------------------------------------------------
// Two-level composite grid (refinement ratio 2, one dt for both levels).
//
// Sec. 4.2, all-levels listing: every leaf block of every level is advanced
// in one sweep, then the fluxes at coarse-fine boundaries are communicated
// and the coarse side is corrected; Sec. 2.2: blocks of all levels have the
// same cell counts, only the cell width differs.  Readings (the paper gives
// no formulas):
//   - restriction: a covered coarse cell holds the mean of its 2^d children;
//   - prolongation into fine guard cells across the coarse-fine boundary:
//     u_f = u_c + sum_d s_d sigma_d / 4 (s_d = -1 for the lower child, +1 for
//     the upper) with MC slopes sigma_d of the conserved coarse variables --
//     conservative (the children average to the parent);
//   - flux correction: at a coarse face on the boundary of the fine region
//     the coarse flux is replaced by the mean of the 2^(d-1) fine fluxes
//     through it, in every RK stage, weighted like the stage's L term.
// Layout: coarse blocks 0..n0-1 (the complete coarse lattice; covered blocks
// hold restricted data), then fine blocks n0..n0+n1-1 (lattice over the
// bounding box of the fine region, x fastest).  The refined coarse blocks are
// any set of whole blocks (a box, an L, separate boxes) at least one block
// away from the domain boundary; the fine lattice's blocks whose parent is not
// refined do not exist (their slots in the array are skipped).
struct Amr2 {
  OrcGrid C, F;
  int lo[3], hi[3];
  ll n0, n1;
  std::vector<unsigned char> refined;   /* [n0] */
};

Amr2 make_amr2(const OrcGrid& C, const OrcAmr2& R) {
  Amr2 A;
  A.C = C;
  A.F = C;
  for (int d = 0; d < 3; ++d) {
    A.lo[d] = d < C.ndim ? R.lo[d] : 0;
    A.hi[d] = d < C.ndim ? R.hi[d] : 1;
    A.F.nb[d] = d < C.ndim ? 2 * (A.hi[d] - A.lo[d]) : 1;
    A.F.dx[d] = C.dx[d] * 0.5;
    A.F.periodic[d] = 0;
  }
  A.n0 = (ll)C.nb[0] * C.nb[1] * C.nb[2];
  A.n1 = (ll)A.F.nb[0] * A.F.nb[1] * A.F.nb[2];
  A.refined.assign(A.n0, 0);
  const Geo gc(C);
  for (ll b = 0; b < A.n0; ++b) {
    int c[3];
    gc.coords(b, c);
    bool in = true;
    for (int d = 0; d < 3; ++d) in = in && c[d] >= A.lo[d] && c[d] < A.hi[d];
    A.refined[b] = in && (!R.refined || R.refined[b]);
  }
  return A;
}

/* a coarse block covered by the fine level */
bool covered(const Amr2& A, const Geo& gc, ll b) {
  (void)gc;
  return A.refined[b] != 0;
}

/* fine lattice block f exists: its parent coarse block is refined */
bool fine_exists(const Amr2& A, const Geo& gc, const Geo& gf, ll f) {
  int c[3], p[3];
  gf.coords(f, c);
  for (int d = 0; d < 3; ++d) p[d] = d < gc.ndim ? A.lo[d] + c[d] / 2 : 0;
  return A.refined[p[0] + (ll)gc.nb[0] * (p[1] + (ll)gc.nb[1] * p[2])] != 0;
}

/* the fine block at lattice offset o from fine block f, or -1 where there is none */
ll fine_neighbour(const Amr2& A, const Geo& gc, const Geo& gf, ll f, const int o[3]) {
  const ll nb = gf.neighbour(f, o);
  return nb >= 0 && fine_exists(A, gc, gf, nb) ? nb : -1;
}

int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

/* value of coarse interior cell at global coarse cell coordinates X */
double coarse_value(const Geo& gc, const double* U, int v, const int X[3]) {
  int bc[3], loc[3];
  for (int d = 0; d < 3; ++d) {
    bc[d] = X[d] / gc.n[d];
    loc[d] = X[d] - bc[d] * gc.n[d] + gc.g[d];
  }
  const ll b = bc[0] + (ll)gc.nb[0] * (bc[1] + (ll)gc.nb[1] * bc[2]);
  return U[gc.at(b, v, loc[2], loc[1], loc[0])];
}

/* fine block f's global fine-cell coordinates of its padded cell (i, j, k) */
void fine_global(const Geo& gf, ll f, int i, int j, int k, int X[3]) {
  int c[3];
  gf.coords(f, c);
  const int p[3] = {i, j, k};
  for (int d = 0; d < 3; ++d) X[d] = c[d] * gf.n[d] + p[d] - gf.g[d];
}

void amr2_restrict(const Amr2& A, double* U) {
  const Geo gc(A.C), gf(A.F);
  const int nd = A.C.ndim;
  const double w = nd == 3 ? 0.125 : 0.25;
#pragma omp parallel for schedule(dynamic, 1)
  for (ll b = 0; b < A.n0; ++b) {
    if (!covered(A, gc, b)) continue;
    int c[3];
    gc.coords(b, c);
    for (int v = 0; v < 5; ++v)
      for (int k = 0; k < gc.n[2]; ++k)
        for (int j = 0; j < gc.n[1]; ++j)
          for (int i = 0; i < gc.n[0]; ++i) {
            const int X[3] = {c[0] * gc.n[0] + i, c[1] * gc.n[1] + j, c[2] * gc.n[2] + k};
            int fX[3];
            for (int d = 0; d < 3; ++d) fX[d] = d < nd ? 2 * (X[d] - A.lo[d] * gc.n[d]) : 0;
            double s = 0.0;
            for (int dz = 0; dz < (nd == 3 ? 2 : 1); ++dz)
              for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                  const int Y[3] = {fX[0] + dx, fX[1] + dy, fX[2] + dz};
                  int fb[3], loc[3];
                  for (int d = 0; d < 3; ++d) {
                    fb[d] = Y[d] / gf.n[d];
                    loc[d] = Y[d] - fb[d] * gf.n[d] + gf.g[d];
                  }
                  const ll f = fb[0] + (ll)gf.nb[0] * (fb[1] + (ll)gf.nb[1] * fb[2]);
                  s = s + U[gc.at(A.n0 + f, v, loc[2], loc[1], loc[0])];
                }
            U[gc.at(b, v, k + gc.g[2], j + gc.g[1], i + gc.g[0])] = s * w;
          }
  }
}

/* guard cells of every fine block: same-level copies where the fine
 * neighbour exists, conservative linear prolongation from the coarse level
 * elsewhere.  The coarse level's interior must be current (restricted). */
void amr2_fill_fine(const Amr2& A, double* U) {
  const Geo gc(A.C), gf(A.F);
  const int nd = A.C.ndim;
#pragma omp parallel for schedule(dynamic, 1)
  for (ll f = 0; f < A.n1; ++f) {
    if (!fine_exists(A, gc, gf, f)) continue;
    for (int k = 0; k < gf.p[2]; ++k)
      for (int j = 0; j < gf.p[1]; ++j)
        for (int i = 0; i < gf.p[0]; ++i) {
          const int x[3] = {i, j, k};
          int o[3];
          bool interior = true;
          for (int d = 0; d < 3; ++d) {
            o[d] = x[d] < gf.g[d] ? -1 : (x[d] >= gf.g[d] + gf.n[d] ? 1 : 0);
            if (o[d]) interior = false;
          }
          if (interior) continue;
          const ll nb = fine_neighbour(A, gc, gf, f, o);
          if (nb >= 0) {
            for (int v = 0; v < 5; ++v)
              U[gf.at(A.n0 + f, v, k, j, i)] =
                  U[gf.at(A.n0 + nb, v, k - o[2] * gf.n[2], j - o[1] * gf.n[1], i - o[0] * gf.n[0])];
            continue;
          }
          int X[3], P[3], sgn[3];
          fine_global(gf, f, i, j, k, X);
          for (int d = 0; d < 3; ++d) {
            if (d < nd) {
              const int h = fdiv(X[d], 2);
              P[d] = A.lo[d] * gc.n[d] + h;
              sgn[d] = (X[d] - 2 * h) == 0 ? -1 : 1;
            } else {
              P[d] = 0;
              sgn[d] = 0;
            }
          }
          for (int v = 0; v < 5; ++v) {
            double val = coarse_value(gc, U, v, P);
            for (int d = 0; d < nd; ++d) {
              int Pm[3] = {P[0], P[1], P[2]}, Pp[3] = {P[0], P[1], P[2]};
              Pm[d] -= 1;
              Pp[d] += 1;
              const double sig = orc::mc_slope(coarse_value(gc, U, v, Pm), coarse_value(gc, U, v, P),
                                               coarse_value(gc, U, v, Pp));
              val = val + 0.25 * sig * (double)sgn[d];
            }
            U[gf.at(A.n0 + f, v, k, j, i)] = val;
          }
        }
  }
}

/* Flux registers: the fluxes through the boundary faces of the fine region
 * (fine side) and through the coarse faces adjacent to it (coarse side). */
struct FluxReg {
  std::vector<std::vector<double>> face;   /* [(block)*6 + face] -> [5][t2][t1] or empty */
};

void tangential(int d, int& t1, int& t2) {
  t1 = d == 0 ? 1 : 0;
  t2 = d == 2 ? 1 : 2;
}

void record_face(const Geo& g, const Work& w, int d, int side, std::vector<double>& out) {
  int t1, t2;
  tangential(d, t1, t2);
  const int n1 = g.n[t1], n2 = g.n[t2];
  out.assign((size_t)5 * n1 * n2, 0.0);
  const ll cells = g.cells;
  for (int v = 0; v < 5; ++v)
    for (int b2 = 0; b2 < n2; ++b2)
      for (int b1 = 0; b1 < n1; ++b1) {
        int x[3];
        x[d] = side ? g.g[d] + g.n[d] : g.g[d];   /* F[d][c]: face between c - e_d and c */
        x[t1] = g.g[t1] + b1;
        x[t2] = g.g[t2] + b2;
        out[((size_t)v * n2 + b2) * n1 + b1] = w.F[d][v * cells + g.cell(x[2], x[1], x[0])];
      }
}

/* Record the fluxes of block t's faces on a coarse-fine boundary: a coarse
 * leaf block's faces towards a covered block, a fine block's faces with no
 * fine neighbour. */
void record_cf_faces(const Amr2& A, const Geo& gc, const Geo& gf, ll t, const Work& w, FluxReg& R) {
  for (int d = 0; d < A.C.ndim; ++d)
    for (int side = 0; side < 2; ++side) {
      int o[3] = {0, 0, 0};
      o[d] = side ? 1 : -1;
      if (t < A.n0) {
        const ll nb = gc.neighbour(t, o);
        if (nb >= 0 && covered(A, gc, nb)) record_face(gc, w, d, side, R.face[t * 6 + 2 * d + side]);
      } else if (fine_neighbour(A, gc, gf, t - A.n0, o) < 0) {
        record_face(gf, w, d, side, R.face[t * 6 + 2 * d + side]);
      }
    }
}

ll amr2_stage(const Amr2& A, const double* Uin, const double* Un, double* Uout, double dt, double a, double bcoef,
              FluxReg& R) {
  const Geo gc(A.C), gf(A.F);
  const ll total = A.n0 + A.n1;
  R.face.assign(total * 6, std::vector<double>());
  ll hits = 0;
#pragma omp parallel reduction(+ : hits)
  {
    Work w;
    w.resize(gc.cells);
#pragma omp for schedule(dynamic, 1)
    for (ll t = 0; t < total; ++t) {
      if (t < A.n0) {
        if (covered(A, gc, t)) continue;
        hits += stage_block(A.C, gc, t, Uin, Un, Uout, dt, a, bcoef, w);
      } else {
        if (!fine_exists(A, gc, gf, t - A.n0)) continue;
        hits += stage_block(A.F, gf, t, Uin, Un, Uout, dt, a, bcoef, w);
      }
      record_cf_faces(A, gc, gf, t, w, R);
    }
  }
  return hits;
}

/* The leaf blocks of level `lev` (0 coarse, 1 fine) through every stage of
 * a telescoping step (Fig. "Level-by-levels, Telescoping": per block, every
 * stage, no exchange in between): stage s on the interior widened by
 * 2 (S - s) cells, X[s] -> X[s+1], X[0] = U^n.  The fluxes through the
 * block's coarse-fine faces in stage s go to R[s]. */
ll amr2_level_telescoping(const Amr2& A, const Rk& r, int lev, std::vector<double>* X, double dt, FluxReg* R) {
  const Geo gc(A.C), gf(A.F);
  const ll b0 = lev ? A.n0 : 0, b1 = lev ? A.n0 + A.n1 : A.n0;
  const OrcGrid& G = lev ? A.F : A.C;
  const Geo& geo = lev ? gf : gc;
  ll hits = 0;
#pragma omp parallel reduction(+ : hits)
  {
    Work w;
    w.resize(gc.cells);
#pragma omp for schedule(dynamic, 1)
    for (ll t = b0; t < b1; ++t) {
      if (lev ? !fine_exists(A, gc, gf, t - A.n0) : covered(A, gc, t)) continue;
      for (int st = 0; st < r.S; ++st) {
        hits += stage_block(G, geo, t, X[st].data(), st ? X[0].data() : nullptr, X[st + 1].data(), dt, r.a[st],
                            r.b[st], w, 2 * (r.S - 1 - st));
        record_cf_faces(A, gc, gf, t, w, R[st]);
      }
    }
  }
  return hits;
}

/* Replace, on the coarse side, the flux through every coarse face on the
 * boundary of the fine region by the mean of the fine fluxes through it:
 * U += coef * dt * (F_coarse - mean F_fine) / dx on the low side of the
 * face, with the opposite sign on the high side (coef = the stage's b). */
void amr2_reflux(const Amr2& A, double* U, double dt, double coef, const FluxReg& R) {
  const Geo gc(A.C), gf(A.F);
  const int nd = A.C.ndim;
  for (ll b = 0; b < A.n0; ++b) {
    if (covered(A, gc, b)) continue;
    int c[3];
    gc.coords(b, c);
    for (int d = 0; d < nd; ++d)
      for (int side = 0; side < 2; ++side) {
        const std::vector<double>& Fc = R.face[b * 6 + 2 * d + side];
        if (Fc.empty()) continue;
        int t1, t2;
        tangential(d, t1, t2);
        const int n1 = gc.n[t1], n2 = gc.n[t2];
        const double idx = 1.0 / A.C.dx[d];
        /* the fine region lies on the `side` of this face; its boundary
         * faces there are the fine blocks' faces of the opposite side */
        const int fside = 1 - side;
        const int nfine = nd == 3 ? 4 : 2;
        for (int b2 = 0; b2 < n2; ++b2)
          for (int b1 = 0; b1 < n1; ++b1) {
            int T[3];                                 /* global coarse coordinates of the face cell's tangentials */
            T[t1] = c[t1] * gc.n[t1] + b1;
            T[t2] = c[t2] * gc.n[t2] + b2;
            /* fine cell next to the face along d: the face lies at coarse
             * cell coordinate X (between cells X - 1 and X); the fine region
             * begins there (side 1) or ends there (side 0) */
            const int X = (c[d] + side) * gc.n[d];
            const int fd = 2 * (X - A.lo[d] * gc.n[d]) - (side ? 0 : 1);
            double fsum[5] = {0, 0, 0, 0, 0};
            for (int q2 = 0; q2 < (nd == 3 ? 2 : 1); ++q2)
              for (int q1 = 0; q1 < 2; ++q1) {
                int Y[3];
                Y[d] = fd;
                Y[t1] = 2 * (T[t1] - A.lo[t1] * gc.n[t1]) + q1;
                Y[t2] = nd == 3 || t2 < nd ? 2 * (T[t2] - A.lo[t2] * gc.n[t2]) + q2 : 0;
                int fb[3], loc[3];
                for (int e = 0; e < 3; ++e) {
                  fb[e] = Y[e] / gf.n[e];
                  loc[e] = Y[e] - fb[e] * gf.n[e];
                }
                const ll f = fb[0] + (ll)gf.nb[0] * (fb[1] + (ll)gf.nb[1] * fb[2]);
                const std::vector<double>& Ff = R.face[(A.n0 + f) * 6 + 2 * d + fside];
                const int fn1 = gf.n[t1], fn2 = gf.n[t2];
                for (int v = 0; v < 5; ++v) fsum[v] = fsum[v] + Ff[((size_t)v * fn2 + loc[t2]) * fn1 + loc[t1]];
                (void)fn2;
              }
            int x[3];
            x[d] = side ? gc.g[d] + gc.n[d] - 1 : gc.g[d];
            x[t1] = gc.g[t1] + b1;
            x[t2] = gc.g[t2] + b2;
            for (int v = 0; v < 5; ++v) {
              const double fmean = fsum[v] / (double)nfine;
              const double fcv = Fc[((size_t)v * n2 + b2) * n1 + b1];
              const double corr = side ? (fcv - fmean) : (fmean - fcv);
              U[gc.at(b, v, x[2], x[1], x[0])] += coef * dt * corr * idx;
            }
          }
      }
  }
}

double amr2_compute_dt(const Amr2& A, const double* U) {
  const Geo gc(A.C);
  double smax = 0.0;
  for (int lev = 0; lev < 2; ++lev) {
    const OrcGrid& G = lev ? A.F : A.C;
    const double idx = 1.0 / G.dx[0], idy = 1.0 / G.dx[1], idz = 1.0 / G.dx[2];
    const ll b0 = lev ? A.n0 : 0, b1 = lev ? A.n0 + A.n1 : A.n0;
    const Geo gf(A.F);
    for (ll b = b0; b < b1; ++b) {
      if (lev ? !fine_exists(A, gc, gf, b - A.n0) : covered(A, gc, b)) continue;
      for (int k = gc.g[2]; k < gc.g[2] + gc.n[2]; ++k)
        for (int j = gc.g[1]; j < gc.g[1] + gc.n[1]; ++j)
          for (int i = gc.g[0]; i < gc.g[0] + gc.n[0]; ++i) {
            double u5[5], W[5];
            load_cons(gc, U, b, k, j, i, u5);
            orc::prim_from_cons(u5, A.C.gamma, A.C.small_rho, A.C.small_p, W);
            smax = std::max(smax, orc::signal_speed(gc.ndim, W, A.C.gamma, idx, idy, idz));
          }
    }
  }
  return A.C.cfl / smax;
}

void amr2_prepare(const Amr2& A, double* U) {
  amr2_restrict(A, U);
  fill_guardcells(A.C, U);   /* coarse lattice = the first n0 blocks */
  amr2_fill_fine(A, U);
}

/* One SSP-RK step on the two-level grid, all-levels non-telescoping: every
 * stage prepares its input (restriction, coarse fill, fine fill), updates the
 * leaf blocks and corrects the coarse side with weight b_s. */
ll amr2_step(const Amr2& A, double* U, double dt, int nstages = 2) {
  const Rk r = rk_scheme(nstages);
  const Geo gc(A.C);
  const ll total = (A.n0 + A.n1) * 5 * gc.cells;
  std::vector<double> X(U, U + total), Y(total);
  FluxReg R;
  ll hits = 0;
  amr2_prepare(A, U);
  hits += amr2_stage(A, U, nullptr, X.data(), dt, r.a[0], r.b[0], R);
  amr2_reflux(A, X.data(), dt, r.b[0], R);
  for (int st = 1; st < r.S; ++st) {
    amr2_prepare(A, X.data());
    std::memcpy(Y.data(), X.data(), total * sizeof(double));
    hits += amr2_stage(A, X.data(), U, Y.data(), dt, r.a[st], r.b[st], R);
    amr2_reflux(A, Y.data(), dt, r.b[st], R);
    std::swap(X, Y);
  }
  const Geo gf(A.F);
  for (ll b = 0; b < A.n0 + A.n1; ++b) {
    if (b < A.n0 ? covered(A, gc, b) : !fine_exists(A, gc, gf, b - A.n0)) continue;
    for (int v = 0; v < 5; ++v)
      for (int k = gc.g[2]; k < gc.g[2] + gc.n[2]; ++k)
        for (int j = gc.g[1]; j < gc.g[1] + gc.n[1]; ++j)
          for (int i = gc.g[0]; i < gc.g[0] + gc.n[0]; ++i) {
            const ll o = gc.at(b, v, k, j, i);
            U[o] = X[o];
          }
  }
  amr2_restrict(A, U);
  return hits;
}

/* One SSP-RK step on the two-level grid in the level-by-level, telescoping
 * variant (Sec. 4.2 and Fig. "Level-by-levels, Telescoping"): one guard fill
 * for both levels (restriction, coarse fill, fine fill with prolongation of
 * all guard layers), then the levels from the finest down, each block through
 * every stage on its own guard data; the coarse side of the fine region is
 * then corrected with the fine fluxes, stage by stage, each with the weight
 * its L term has in U^{n+1} (rk_weight); the step ends with the restriction.
 * One dt for both levels.  Needs 2 S guard cells. */
ll amr2_step_telescoping(const Amr2& A, double* U, double dt, int nstages = 2) {
  const Rk r = rk_scheme(nstages);
  const Geo gc(A.C);
  const ll nblk = A.n0 + A.n1;
  const ll total = nblk * 5 * gc.cells;
  FluxReg R[3];
  for (int st = 0; st < r.S; ++st) R[st].face.assign(nblk * 6, std::vector<double>());
  ll hits = 0;
  amr2_prepare(A, U);
  std::vector<double> X[4];
  for (int st = 0; st <= r.S; ++st) X[st].assign(U, U + total);
  for (int lev = 1; lev >= 0; --lev) hits += amr2_level_telescoping(A, r, lev, X, dt, R);
  double* out = X[r.S].data();
  for (int st = 0; st < r.S; ++st) amr2_reflux(A, out, dt, rk_weight(r, st), R[st]);
  const Geo gf(A.F);
  for (ll b = 0; b < nblk; ++b) {
    if (b < A.n0 ? covered(A, gc, b) : !fine_exists(A, gc, gf, b - A.n0)) continue;
    for (int v = 0; v < 5; ++v)
      for (int k = gc.g[2]; k < gc.g[2] + gc.n[2]; ++k)
        for (int j = gc.g[1]; j < gc.g[1] + gc.n[1]; ++j)
          for (int i = gc.g[0]; i < gc.g[0] + gc.n[0]; ++i) {
            const ll o = gc.at(b, v, k, j, i);
            U[o] = out[o];
          }
  }
  amr2_restrict(A, U);
  return hits;
}

// ---------------------------------------------------------------------------
// Adjoint of the stage and of the SSP-RK2 step (dt held fixed, branches as in
// the forward evaluation).  Each face's flux is differentiated with respect
// to the conserved values of its 4 stencil cells by forward-mode dual
// numbers over the oracle's own pointwise functions (oracle_pointwise.h):
// comparisons act on the values, so every branch keeps its forward decision.
// The transposed data flow (faces -> stencil cells -> guard fill -> sources)
// is then summed plainly.
template <int K>
struct Dual {
  double v;
  double d[K];
  Dual(double x = 0.0) : v(x) { for (int i = 0; i < K; ++i) d[i] = 0.0; }
};
template <int K> Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) { Dual<K> r(a.v + b.v); for (int i = 0; i < K; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int K> Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) { Dual<K> r(a.v - b.v); for (int i = 0; i < K; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int K> Dual<K> operator-(const Dual<K>& a) { Dual<K> r(-a.v); for (int i = 0; i < K; ++i) r.d[i] = -a.d[i]; return r; }
template <int K> Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) { Dual<K> r(a.v * b.v); for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int K> Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r(a.v / b.v);
  for (int i = 0; i < K; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}
template <int K> Dual<K> sqrt(const Dual<K>& a) { Dual<K> r(std::sqrt(a.v)); for (int i = 0; i < K; ++i) r.d[i] = a.d[i] / (2.0 * r.v); return r; }
template <int K> bool operator<(const Dual<K>& a, const Dual<K>& b) { return a.v < b.v; }
template <int K> bool operator<=(const Dual<K>& a, const Dual<K>& b) { return a.v <= b.v; }
template <int K> bool operator>(const Dual<K>& a, const Dual<K>& b) { return a.v > b.v; }
template <int K> bool operator==(const Dual<K>& a, const Dual<K>& b) { return a.v == b.v; }

using D20 = Dual<20>;

/* The transposed face loop of one stage on the box of width `ring` around
 * the interior (ring = 0: the interior; ring > 0: a stage of the telescoping
 * mode, which reads U's own cells 2 beyond the box): for the cotangent M on
 * the box's cells, J_L(U)^T (scale M) is added into adj at every padded cell
 * the face stencils read. */
void stage_vjp_local(const OrcGrid& G, const double* U, const double* M, double scale, double* adj, int ring) {
  const Geo geo(G);
  const ll nbk = geo.nblocks();
  const ll cells = geo.cells;
  const int nd = geo.ndim;
  const Box R(geo, ring);
  const ll stride[3] = {1, geo.p[0], (ll)geo.p[0] * geo.p[1]};
#pragma omp parallel for schedule(dynamic, 1)
  for (ll b = 0; b < nbk; ++b) {
    for (int d = 0; d < nd; ++d) {
      const double idx = 1.0 / G.dx[d];
      const int t1 = d == 0 ? 2 : 1, t2 = d == 2 ? 2 : 3;
      const int vmap[5] = {0, 1 + d, t1, t2, 4};
      for (int k = 0; k < geo.p[2]; ++k)
        for (int j = 0; j < geo.p[1]; ++j)
          for (int i = 0; i < geo.p[0]; ++i) {
            const int x[3] = {i, j, k};
            bool ok = x[d] >= R.lo[d] && x[d] <= R.hi[d];
            for (int e = 0; e < 3; ++e)
              if (e != d && !R.in(e, x[e])) ok = false;
            if (!ok) continue;
            const ll c = geo.cell(k, j, i);
            /* flux adjoint from this block's own cells c - e_d and c */
            double lamF[5];
            for (int v = 0; v < 5; ++v) {
              const double mc = R.in(d, x[d]) ? M[geo.at(b, v, k, j, i) ] : 0.0;
              const int xm = x[d] - 1;
              const double mm = R.in(d, xm) ? M[geo.at(b, v, k, j, i) - stride[d]] : 0.0;
              lamF[v] = scale * idx * (mc - mm);
            }
            /* the 4 stencil cells c-2e, c-e, c, c+e as dual inputs (20 slots) */
            D20 W[4][5];
            for (int s = 0; s < 4; ++s) {
              D20 u5[5];
              const ll cs = c + (s - 2) * stride[d];
              for (int v = 0; v < 5; ++v) {
                u5[v] = D20(U[b * 5 * cells + v * cells + cs]);
                u5[v].d[5 * s + v] = 1.0;
              }
              orc::prim_from_cons(u5, D20(G.gamma), D20(G.small_rho), D20(G.small_p), W[s]);
            }
            D20 WL[5], WR[5], F[5];
            for (int q = 0; q < 5; ++q) {
              const int v = vmap[q];
              const D20 sL = orc::mc_slope(W[0][v], W[1][v], W[2][v]);
              const D20 sR = orc::mc_slope(W[1][v], W[2][v], W[3][v]);
              WL[q] = W[1][v] + D20(0.5) * sL;
              WR[q] = W[2][v] - D20(0.5) * sR;
            }
            orc::hllc(WL, WR, D20(G.gamma), F);
            for (int s = 0; s < 4; ++s) {
              const ll cs = c + (s - 2) * stride[d];
              for (int v = 0; v < 5; ++v) {
                double acc = 0.0;
                for (int q = 0; q < 5; ++q) acc += lamF[vmap[q]] * F[q].d[5 * s + v];
                adj[b * 5 * cells + v * cells + cs] += acc;
              }
            }
          }
    }
  }
}

/* J_L(U)^T (scale M) on the interior of every block; U must have its guard
 * cells filled.  out is written on interior cells. */
void stage_vjp(const OrcGrid& G, const double* U, const double* M, double scale, double* out) {
  const Geo geo(G);
  const ll nbk = geo.nblocks();
  const ll cells = geo.cells;
  const int nd = geo.ndim;
  std::vector<double> ext(nbk * 5 * cells, 0.0);   /* adjoint of the conserved stencil inputs */
  stage_vjp_local(G, U, M, scale, ext.data(), 0);
  /* adjoint of the guard fill (face slabs only: the stencil reads no
   * corners): a guard position hands its adjoint to the interior cell it was
   * copied from -- the neighbour's, or the block's own boundary cell at an
   * outflow edge */
#pragma omp parallel for schedule(dynamic, 1)
  for (ll b = 0; b < nbk; ++b)
    for (int k = geo.g[2]; k < geo.g[2] + geo.n[2]; ++k)
      for (int j = geo.g[1]; j < geo.g[1] + geo.n[1]; ++j)
        for (int i = geo.g[0]; i < geo.g[0] + geo.n[0]; ++i)
          for (int v = 0; v < 5; ++v) out[geo.at(b, v, k, j, i)] = ext[geo.at(b, v, k, j, i)];
  for (ll b = 0; b < nbk; ++b)
    for (int d = 0; d < nd; ++d)
      for (int side = 0; side < 2; ++side) {
        int o[3] = {0, 0, 0};
        o[d] = side ? 1 : -1;
        const ll nb = geo.neighbour(b, o);
        for (int k = 0; k < geo.p[2]; ++k)
          for (int j = 0; j < geo.p[1]; ++j)
            for (int i = 0; i < geo.p[0]; ++i) {
              const int x[3] = {i, j, k};
              bool slab = side ? (x[d] >= geo.g[d] + geo.n[d] && x[d] < geo.g[d] + geo.n[d] + 2)
                               : (x[d] >= geo.g[d] - 2 && x[d] < geo.g[d]);
              for (int e = 0; e < 3; ++e)
                if (e != d && !inside(geo, e, x[e])) slab = false;
              if (!slab) continue;
              int src[3] = {i, j, k};
              ll sb = b;
              if (nb >= 0) {
                sb = nb;
                src[d] = x[d] - o[d] * geo.n[d];
              } else {
                src[d] = side ? geo.g[d] + geo.n[d] - 1 : geo.g[d];
              }
              for (int v = 0; v < 5; ++v)
                out[geo.at(sb, v, src[2], src[1], src[0])] += ext[geo.at(b, v, k, j, i)];
            }
      }
}

/* dJ/dU^n of one SSP-RK step of S stages (dt held fixed) from dJ/dU^{n+1}:
 * the Shu-Osher recursion U(s) = a_s U^n + b_s (U(s-1) + dt L(U(s-1))) run
 * backwards.  With lam_S = lam the adjoint of U(S) = U^{n+1},
 *   lam_{s-1} = b_s lam_s + J_L(U(s-1))^T (b_s dt lam_s),
 * and U^n collects lam_0 plus a_s lam_s from every stage. */
void step_adjoint(const OrcGrid& G, const double* Un, double dt, const double* lam, double* lam_prev,
                  int nstages = 2) {
  const Rk r = rk_scheme(nstages);
  const Geo geo(G);
  const ll total = geo.nblocks() * 5 * geo.cells;
  /* forward: X[s] = U(s) with filled guard cells, s = 0 .. S-1 */
  std::vector<std::vector<double>> X(r.S);
  X[0].assign(Un, Un + total);
  fill_guardcells(G, X[0].data());
  for (int st = 1; st < r.S; ++st) {
    X[st] = X[st - 1];
    stage(G, X[st - 1].data(), X[0].data(), X[st].data(), dt, r.a[st - 1], r.b[st - 1], nullptr, 0);
    fill_guardcells(G, X[st].data());
  }
  std::vector<double> cur(lam, lam + total), acc(total, 0.0), jt(total, 0.0);
  for (int st = r.S - 1; st >= 0; --st) {
    /* stage st maps U(st) to U(st+1) with (a, b) = (r.a[st], r.b[st]) */
    std::fill(jt.begin(), jt.end(), 0.0);
    stage_vjp(G, X[st].data(), cur.data(), r.b[st] * dt, jt.data());
    for (ll b = 0; b < geo.nblocks(); ++b)
      for (int v = 0; v < 5; ++v)
        for (int k = geo.g[2]; k < geo.g[2] + geo.n[2]; ++k)
          for (int j = geo.g[1]; j < geo.g[1] + geo.n[1]; ++j)
            for (int i = geo.g[0]; i < geo.g[0] + geo.n[0]; ++i) {
              const ll o = geo.at(b, v, k, j, i);
              acc[o] = acc[o] + r.a[st] * cur[o];
              cur[o] = r.b[st] * cur[o] + jt[o];
            }
  }
  for (ll b = 0; b < geo.nblocks(); ++b)
    for (int v = 0; v < 5; ++v)
      for (int k = geo.g[2]; k < geo.g[2] + geo.n[2]; ++k)
        for (int j = geo.g[1]; j < geo.g[1] + geo.n[1]; ++j)
          for (int i = geo.g[0]; i < geo.g[0] + geo.n[0]; ++i) {
            const ll o = geo.at(b, v, k, j, i);
            lam_prev[o] = acc[o] + cur[o];
          }
}

/* dJ/dU^n of one telescoping SSP-RK step (step_telescoping, dt held fixed)
 * from dJ/dU^{n+1} on interior cells.  Forward: Uf = fill(U^n) (all guard
 * layers), X_0 = Uf, stage s writes X_{s+1} = a_s Uf + b_s (X_s + dt L(X_s))
 * on the box of width ring_s = 2 (S-1-s) from X_s's own cells, and keeps Uf's
 * values elsewhere.  Backwards, with lam_S the cotangent of X_S:
 *   on box_s:   Uf gets a_s lam_{s+1};  lam_s = b_s lam_{s+1} + J_L(X_s)^T (b_s dt lam_{s+1}),
 *   elsewhere:  Uf gets lam_{s+1} (X_{s+1} holds Uf's values there),
 * X_0 = Uf gets lam_0, and the fill is reversed: every guard cell's adjoint
 * goes to the interior cell its value was copied from.  That source map is
 * read off by filling an array that holds each interior cell's own index
 * (the fill only copies values). */
void step_adjoint_telescoping(const OrcGrid& G, const double* Un, double dt, const double* lam, double* lam_prev,
                              int nstages = 2) {
  const Rk r = rk_scheme(nstages);
  const Geo geo(G);
  const ll nbk = geo.nblocks();
  const ll total = nbk * 5 * geo.cells;
  std::vector<double> Uf(Un, Un + total);
  fill_guardcells(G, Uf.data());
  std::vector<std::vector<double>> X(r.S);
  X[0] = Uf;
  for (int st = 0; st + 1 < r.S; ++st) {
    X[st + 1] = Uf;
    stage(G, X[st].data(), st ? Uf.data() : nullptr, X[st + 1].data(), dt, r.a[st], r.b[st], nullptr, 0,
          2 * (r.S - 1 - st));
  }
  /* lam_S: the cotangent on interior cells */
  std::vector<double> cur(total, 0.0), accU(total, 0.0), jt(total, 0.0);
  for (ll b = 0; b < nbk; ++b)
    for (int v = 0; v < 5; ++v)
      for (int k = geo.g[2]; k < geo.g[2] + geo.n[2]; ++k)
        for (int j = geo.g[1]; j < geo.g[1] + geo.n[1]; ++j)
          for (int i = geo.g[0]; i < geo.g[0] + geo.n[0]; ++i) cur[geo.at(b, v, k, j, i)] = lam[geo.at(b, v, k, j, i)];
  for (int st = r.S - 1; st >= 0; --st) {
    const int ring = 2 * (r.S - 1 - st);
    const Box R(geo, ring);
    std::fill(jt.begin(), jt.end(), 0.0);
    /* the cotangent of the box cells only: the stage writes nothing else */
    std::vector<double> M(total, 0.0);
    for (ll b = 0; b < nbk; ++b)
      for (int v = 0; v < 5; ++v)
        for (int k = 0; k < geo.p[2]; ++k)
          for (int j = 0; j < geo.p[1]; ++j)
            for (int i = 0; i < geo.p[0]; ++i)
              if (R.in(0, i) && R.in(1, j) && R.in(2, k)) M[geo.at(b, v, k, j, i)] = cur[geo.at(b, v, k, j, i)];
    stage_vjp_local(G, X[st].data(), M.data(), r.b[st] * dt, jt.data(), ring);
    for (ll b = 0; b < nbk; ++b)
      for (int v = 0; v < 5; ++v)
        for (int k = 0; k < geo.p[2]; ++k)
          for (int j = 0; j < geo.p[1]; ++j)
            for (int i = 0; i < geo.p[0]; ++i) {
              const ll o = geo.at(b, v, k, j, i);
              if (R.in(0, i) && R.in(1, j) && R.in(2, k)) {
                accU[o] = accU[o] + r.a[st] * cur[o];
                cur[o] = r.b[st] * cur[o] + jt[o];
              } else {
                accU[o] = accU[o] + cur[o];
                cur[o] = jt[o];
              }
            }
  }
  for (ll o = 0; o < total; ++o) accU[o] = accU[o] + cur[o];
  /* reverse of the fill */
  std::vector<double> src(total, -1.0);
  for (ll b = 0; b < nbk; ++b)
    for (int v = 0; v < 5; ++v)
      for (int k = geo.g[2]; k < geo.g[2] + geo.n[2]; ++k)
        for (int j = geo.g[1]; j < geo.g[1] + geo.n[1]; ++j)
          for (int i = geo.g[0]; i < geo.g[0] + geo.n[0]; ++i) src[geo.at(b, v, k, j, i)] = (double)geo.at(b, v, k, j, i);
  fill_guardcells(G, src.data());
  std::vector<double> out(total, 0.0);
  for (ll o = 0; o < total; ++o) {
    const ll from = (ll)src[o];
    if (from >= 0) out[from] += accU[o];
  }
  for (ll b = 0; b < nbk; ++b)
    for (int v = 0; v < 5; ++v)
      for (int k = geo.g[2]; k < geo.g[2] + geo.n[2]; ++k)
        for (int j = geo.g[1]; j < geo.g[1] + geo.n[1]; ++j)
          for (int i = geo.g[0]; i < geo.g[0] + geo.n[0]; ++i) {
            const ll o = geo.at(b, v, k, j, i);
            lam_prev[o] = out[o];
          }
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

/* The same on the interior widened by ext cells (0 or 2; ext = 2 needs 4
 * guard cells, the first stage of the telescoping mode); -1 if invalid. */
long long orc_stage_ext(const OrcGrid* G, const double* Uin, const double* Un, double* Uout, double dt,
                        double a, double b, int ext) {
  if (ext < 0 || G->ng < ext + 2) return -1;
  return stage(*G, Uin, Un, Uout, dt, a, b, nullptr, 0, ext);
}

long long orc_step(const OrcGrid* G, double* U, double dt) { return step(*G, U, dt); }

/* One telescoping-mode step; -1 if the grid has fewer than 4 guard cells. */
long long orc_step_telescoping(const OrcGrid* G, double* U, double dt) {
  if (G->ng < 4) return -1;
  return step_telescoping(*G, U, dt);
}

/* One step with nstages (2 or 3) stages, telescoping or not; -1 if nstages
 * is invalid or the telescoping mode lacks its 2 nstages guard cells. */
long long orc_step_rk(const OrcGrid* G, double* U, double dt, int nstages, int telescoping) {
  if ((nstages != 2 && nstages != 3) || (telescoping && G->ng < 2 * nstages)) return -1;
  return telescoping ? step_telescoping(*G, U, dt, nstages) : step(*G, U, dt, nstages);
}

/* nsteps steps, each with dt = compute_dt(U^n); dt_hist[s] receives dt.
 * telescoping != 0 selects the telescoping mode; nstages 2 or 3. */
long long orc_run(const OrcGrid* G, double* U, int nsteps, double* dt_hist, int telescoping, int nstages) {
  if ((nstages != 2 && nstages != 3) || (telescoping && G->ng < 2 * nstages)) return -1;
  long long hits = 0;
  for (int s = 0; s < nsteps; ++s) {
    const double dt = compute_dt(*G, U);
    if (dt_hist) dt_hist[s] = dt;
    hits += telescoping ? step_telescoping(*G, U, dt, nstages) : step(*G, U, dt, nstages);
  }
  return hits;
}

/* ---- two-level composite grid (coarse blocks first, then fine blocks) ---- */

void orc2_restrict(const OrcGrid* G, const OrcAmr2* R, double* U) { amr2_restrict(make_amr2(*G, *R), U); }

void orc2_fill(const OrcGrid* G, const OrcAmr2* R, double* U) { amr2_prepare(make_amr2(*G, *R), U); }

double orc2_compute_dt(const OrcGrid* G, const OrcAmr2* R, const double* U) {
  return amr2_compute_dt(make_amr2(*G, *R), U);
}

long long orc2_step(const OrcGrid* G, const OrcAmr2* R, double* U, double dt) {
  return amr2_step(make_amr2(*G, *R), U, dt);
}

/* One stage without flux correction (reflux = 0) or with it (reflux = 1):
 * prepares Uin (restriction + guard fills) and writes the leaf blocks of Uout. */
long long orc2_stage(const OrcGrid* G, const OrcAmr2* R, double* Uin, const double* Un, double* Uout, double dt,
                     double a, double b, int reflux) {
  const Amr2 A = make_amr2(*G, *R);
  FluxReg reg;
  amr2_prepare(A, Uin);
  const ll hits = amr2_stage(A, Uin, Un, Uout, dt, a, b, reg);
  if (reflux) amr2_reflux(A, Uout, dt, b, reg);
  return hits;
}

/* One level-by-level telescoping step; -1 if the grid has fewer than 4 guard cells. */
long long orc2_step_telescoping(const OrcGrid* G, const OrcAmr2* R, double* U, double dt) {
  if (G->ng < 4) return -1;
  return amr2_step_telescoping(make_amr2(*G, *R), U, dt);
}

/* One step with nstages stages: all-levels non-telescoping, or (telescoping
 * != 0) level-by-level telescoping; -1 if invalid. */
long long orc2_step_rk(const OrcGrid* G, const OrcAmr2* R, double* U, double dt, int nstages, int telescoping) {
  if ((nstages != 2 && nstages != 3) || (telescoping && G->ng < 2 * nstages)) return -1;
  const Amr2 A = make_amr2(*G, *R);
  return telescoping ? amr2_step_telescoping(A, U, dt, nstages) : amr2_step(A, U, dt, nstages);
}

/* nsteps steps with the CFL dt of the leaf cells; telescoping != 0 selects
 * the level-by-level telescoping variant, else all-levels non-telescoping. */
long long orc2_run(const OrcGrid* G, const OrcAmr2* R, double* U, int nsteps, double* dt_hist, int telescoping,
                   int nstages) {
  if ((nstages != 2 && nstages != 3) || (telescoping && G->ng < 2 * nstages)) return -1;
  const Amr2 A = make_amr2(*G, *R);
  long long hits = 0;
  amr2_restrict(A, U);
  for (int s = 0; s < nsteps; ++s) {
    const double dt = amr2_compute_dt(A, U);
    if (dt_hist) dt_hist[s] = dt;
    hits += telescoping ? amr2_step_telescoping(A, U, dt, nstages) : amr2_step(A, U, dt, nstages);
  }
  return hits;
}

/* ---- adjoint (dt held fixed) ---- */

/* out = J_L(U)^T (scale M) on interior cells; U's guard cells are filled here
 * on a copy. */
void orc_stage_vjp(const OrcGrid* G, const double* U, const double* M, double scale, double* out) {
  const Geo geo(*G);
  std::vector<double> Uf(U, U + geo.nblocks() * 5 * geo.cells);
  fill_guardcells(*G, Uf.data());
  stage_vjp(*G, Uf.data(), M, scale, out);
}

void orc_step_adjoint(const OrcGrid* G, const double* Un, double dt, const double* lam_next, double* lam_prev) {
  step_adjoint(*G, Un, dt, lam_next, lam_prev);
}

/* The same for nstages (2 or 3) stages; -1 if nstages is invalid. */
int orc_step_adjoint_rk(const OrcGrid* G, const double* Un, double dt, const double* lam_next, double* lam_prev,
                        int nstages) {
  if (nstages != 2 && nstages != 3) return -1;
  step_adjoint(*G, Un, dt, lam_next, lam_prev, nstages);
  return 0;
}

/* Adjoint of the telescoping step of nstages (2 or 3) stages; -1 if nstages is
 * invalid or the guard width is below 2 * nstages. */
int orc_step_adjoint_telescoping(const OrcGrid* G, const double* Un, double dt, const double* lam_next,
                                 double* lam_prev, int nstages) {
  if ((nstages != 2 && nstages != 3) || G->ng < 2 * nstages) return -1;
  step_adjoint_telescoping(*G, Un, dt, lam_next, lam_prev, nstages);
  return 0;
}

}  // extern "C"
