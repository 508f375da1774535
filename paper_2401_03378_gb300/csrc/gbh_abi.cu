// gbh_abi.cu -- the C ABI of libgbhydro.so (declared in include/gbhydro.h).
//
// The context owns: the device copies of the neighbour tables and inverse
// cell widths, one state-sized scratch buffer (the intermediate SSP-RK2 stage
// U1), and a few device words (signal-speed accumulator, floor counter, check
// counter).  Every entry point validates its arguments before enqueuing work
// and reports failures as GBH_ERR_* codes with a message; no host
// synchronisation happens unless the entry point says so.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gbhydro.h"
#include "gbh_internal.h"

using gbh::Eos;
using gbh::Layout;

struct gbh_ctx {
  Layout lay{};
  Eos eos{};
  double cfl = 0.0;
  int device = 0;
  int* d_nbr = nullptr;            // [nblocks][3^ndim]
  int* d_face = nullptr;           // [nblocks][6]
  double* d_inv_dx = nullptr;      // [nblocks][3]
  double* d_scratch = nullptr;     // U(1), one state
  double* d_scratch2 = nullptr;    // U(2) of three-stage SSP-RK (allocated by gbh_set_rk_stages)
  int nstages = 2;                 // SSP-RK stages (2 or 3)
  // primitive variables carried from stage to stage on uniform grids (halo
  // gathered): two arrays of the state's layout (gbh_set_prim_carry)
  double* d_W[2] = {nullptr, nullptr};
  bool prim_carry = false;
  // the face pre-pass of the interior stages (gbh_set_face_prepass): the
  // fluxes through every block face, [nblocks][6][5][nx * nx (3-D) or nx]
  double* d_bflux = nullptr;
  bool face_prepass = false;
  unsigned long long* d_words = nullptr;  // [0] smax accumulator, [1] floor count, [2] check count
  // host-buffer path (allocated on first use)
  double* d_host_state = nullptr;
  double* d_host_dt = nullptr;
  double* d_host_hist = nullptr;
  int host_hist_cap = 0;
  // two-level composite grid (gbh_create_refined)
  bool refined = false;
  int* d_parent = nullptr;
  int* d_children = nullptr;
  int* d_active = nullptr;          // leaf blocks
  int nactive = 0;
  int* d_covered = nullptr;
  int* d_fine = nullptr;
  int* d_flux_slot = nullptr;       // [nblocks][6]
  double* d_flux_reg = nullptr;
  double* d_flux_reg2 = nullptr;    // registers of stages 2 and 3 (telescoping; allocated on first use)
  double* d_flux_reg3 = nullptr;
  size_t flux_reg_doubles = 0;
  gbh::RefluxEntry* d_reflux = nullptr;
  int* d_reflux_of = nullptr;       // [nblocks][6]: flux-correction entry of a coarse leaf face, or -1
  int2* d_cf_faces = nullptr;
  gbh::AmrArgs amr{};
  // batched ensembles (gbh_create_batched): per-block problem id, per-problem CFL accumulators
  int nproblems = 1;
  int* d_problem = nullptr;
  unsigned long long* d_smax = nullptr;  // [nproblems]; points into d_words for a single problem
  unsigned long long* d_smax_own = nullptr;
  // stage-kernel work decomposition (gbh_autotune)
  int kchunk = 0;                   // z planes per work item (3-D); 0 = the whole block
  int items_per_cta = 1;
  int ysplit[3] = {1, 1, 1};        // row bands of the plane tile for ring widths 0, 2, 4
  // CUDA graph of hydro_advance_graph
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  const double* graph_U = nullptr;
  const double* graph_dt = nullptr;
  int graph_steps = 0;
  // telescoping mode (gbh_set_telescoping): one guard fill per step
  bool telescoping = false;
  // adjoint buffers (allocated on first use): per-face adjoint slots, intermediate adjoint
  double* d_adj_lamW = nullptr;
  double* d_adj_tmp = nullptr;
  double* d_adj_prim = nullptr;     // primitives of the state a VJP linearises about
  double* d_adj_tmp2 = nullptr;     // second intermediate adjoint (three stages)
  double* d_adj_fill = nullptr;     // telescoping adjoint: the filled copy of Un
  double* d_adj_tele = nullptr;     // telescoping adjoint: the adjoint of the filled state
  size_t adj_slot_doubles = 0;      // size of d_adj_lamW
  // pipelined host-buffer step (hydro_step_host), set up on first use: chunks
  // of consecutive blocks, the highest chunk any face neighbour of a chunk
  // lives in, streams (copy in, stage 1, stage 2, copy out) and events
  std::vector<int> h_face;          // host copy of the face table
  int pipe_chunks = 0;
  int pipe_chunks_wanted = 0;       // gbh_set_host_pipeline (0: about two CTAs per SM per chunk)
  std::vector<int> pipe_first, pipe_need;
  cudaStream_t pipe_stream[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> pipe_ev;   // [3][chunks]: copied in, stage 1 done, stage 2 done
  cudaEvent_t pipe_mark[3] = {nullptr, nullptr, nullptr};
  int* d_ident = nullptr;           // identity block list
  double* d_pipe_out = nullptr;     // the new state
  double* d_pipe_dt = nullptr;      // its CFL dt
  double* d_pipe_int = nullptr;     // interior-only staging (hydro_step_host_interior)
  // kernel timing
  bool timing = false;
  std::vector<cudaEvent_t> ev;     // pairs (start, stop)
  size_t ev_used = 0;
  char err[512] = {0};
};

namespace {

thread_local char g_create_err[512] = {0};

int set_err(gbh_ctx* c, int code, const char* fmt, ...) {
  char* buf = c ? c->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_err(gbh_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return GBH_OK;
  return set_err(c, GBH_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

long long state_elems(const Layout& L) { return (long long)L.nblocks * L.bstride; }

int check_ctx(gbh_ctx* c) {
  if (!c) return set_err(nullptr, GBH_ERR_INVAL, "null context");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(c, e, "cudaGetDevice");
  if (dev != c->device)
    return set_err(c, GBH_ERR_INVAL, "current device %d differs from the context's device %d", dev, c->device);
  return GBH_OK;
}

bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

int check_dt(gbh_ctx* c, double dt) {
  if (!std::isfinite(dt) || !(dt > 0.0)) return set_err(c, GBH_ERR_INVAL, "dt must be finite and > 0 (got %g)", dt);
  return GBH_OK;
}

int record_start(gbh_ctx* c, cudaStream_t s, cudaEvent_t* stop) {
  *stop = nullptr;
  if (!c->timing) return GBH_OK;
  if (c->ev_used + 2 > c->ev.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return set_err(c, GBH_ERR_CUDA, "cudaEventCreate failed");
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return set_err(c, GBH_ERR_CUDA, "cudaEventCreate failed");
    }
    c->ev.push_back(a);
    c->ev.push_back(b);
  }
  cudaEvent_t a = c->ev[c->ev_used], b = c->ev[c->ev_used + 1];
  c->ev_used += 2;
  *stop = b;
  return cuda_err(c, cudaEventRecord(a, s), "cudaEventRecord");
}

// One stage launch.  ring > 0: the telescoping form that also updates that
// many guard cells around the interior, from Uin's own guard cells.
// range_first >= 0: `list` is the identity list of blocks [range_first,
// range_first + nlist), one of a sequence of consecutive ranges whose stages
// run in block order on one stream (the face pre-pass then serves it too).
int stage_launch(gbh_ctx* c, const double* Uin, const double* Un, double* Uout, const double* dt_dev,
                 double dt, double a, double b, bool gather, bool dt_epilogue, cudaStream_t s, int ring = 0,
                 double* flux_reg = nullptr, const int* list = nullptr, int nlist = 0,
                 const double* Win = nullptr, double* Wout = nullptr, int range_first = -1) {
  gbh::StageArgs A{};
  A.Uin = Uin;
  A.Un = Un;
  A.Uout = Uout;
  A.Win = Win;
  A.Wout = Wout;
  A.face_nbr = c->d_face;
  A.inv_dx = c->d_inv_dx;
  A.dt_dev = dt_dev;
  A.dt = dt;
  A.a = a;
  A.b = b;
  A.combine = (a == 0.0 && b == 1.0) ? 0 : (a == 0.5 && b == 0.5) ? 2 : 1;
  A.gather = gather ? 1 : 0;
  gbh::stage_args_common(&A, c->lay, c->eos);
  A.smax_acc = dt_epilogue ? c->d_smax : nullptr;
  A.floor_count = c->d_words + 1;
  A.problem = c->d_problem;
  if (ring > 0 && c->lay.ndim == 3) {
    // a ring-updating stage spans nz + 2*ring planes
    const int span = c->lay.nz + 2 * ring;
    A.kchunk = c->kchunk > 0 ? c->kchunk : span;
    A.nchunks = (span + A.kchunk - 1) / A.kchunk;
  } else if (c->lay.ndim == 3 && c->kchunk > 0) {
    A.kchunk = c->kchunk;
    A.nchunks = (c->lay.nz + c->kchunk - 1) / c->kchunk;
  }
  A.items_per_cta = c->items_per_cta;
  A.ysplit = (ring == 0 || ring == 2 || ring == 4) ? c->ysplit[ring / 2] : 1;
  const bool prepass = c->face_prepass && c->d_bflux && ring == 0 && gather && (!list || range_first >= 0) &&
                       A.ysplit == 1 && A.nchunks == 1;
  if (c->refined) {
    A.block_list = c->d_active;
    A.nlist = c->nactive;
    A.flux_slot = c->d_flux_slot;
    A.flux_reg = flux_reg ? flux_reg : c->d_flux_reg;
    A.flux_reg_len = (long long)c->flux_reg_doubles;
  }
  if (list) {
    A.block_list = list;
    A.nlist = nlist;
  }
  cudaEvent_t stop;
  int rc = record_start(c, s, &stop);
  if (rc) return rc;
  if (prepass) {
    // each block face solved once, then read by the stage
    const int lo = list ? range_first : 0, hi = list ? range_first + nlist : -1;
    if ((rc = cuda_err(c, gbh::launch_face_fluxes(A, c->d_bflux, s, lo, hi), "face pre-pass launch"))) return rc;
    A.bflux = c->d_bflux;
  }
  rc = cuda_err(c, ring > 0 ? gbh::launch_stage_ring(A, ring, s) : gbh::launch_stage(A, s), "stage kernel launch");
  if (rc) return rc;
  if (stop) rc = cuda_err(c, cudaEventRecord(stop, s), "cudaEventRecord");
  return rc;
}

// One stage on a two-level composite grid (all-levels variant): restrict the
// covered coarse blocks of Uin, prolong into the fine guard slabs that face
// the coarser level, update the leaf blocks (writing the boundary fluxes to
// the flux registers), and correct the coarse side of the fine-region
// boundary.  Uin's covered blocks and fine guard cells are rewritten.  With
// dt_epilogue (the last stage) the stage kernel and the correction also leave
// the CFL signal-speed max of the leaf cells of Uout in the accumulator.
// Win (the primitive carry): the primitives of Uin's leaf cells, to which the
// restriction and the prolongation add those of the cells they write, so the
// stage reads no conserved cell it would have to convert; Wout: where the
// stage and the correction leave the primitives of Uout.
int refined_stage(gbh_ctx* c, double* Uin, const double* Un, double* Uout, const double* dt_dev, double dt,
                  double a, double b, bool dt_epilogue, cudaStream_t s, double* Win = nullptr,
                  double* Wout = nullptr) {
  int rc = cuda_err(c, gbh::launch_restrict(Uin, c->amr, s, Win), "restrict launch");
  if (rc) return rc;
  rc = cuda_err(c, gbh::launch_prolong(Uin, c->amr, 2, true, s, Win), "prolong launch");
  if (rc) return rc;
  rc = stage_launch(c, Uin, Un, Uout, dt_dev, dt, a, b, true, dt_epilogue, s, 0, nullptr, nullptr, 0, Win, Wout);
  if (rc) return rc;
  return cuda_err(c, gbh::launch_reflux(Uout, c->amr, dt_dev, dt, b, dt_epilogue ? c->d_smax : nullptr, s, Wout),
                  "reflux launch");
}

// Shu-Osher coefficients of the SSP-RK stages: U(s) = a_s U^n + b_s (U(s-1) +
// dt L(U(s-1))); two stages (0, 1), (1/2, 1/2); three stages (0, 1),
// (3/4, 1/4), (1/3, 2/3).
struct RkCoef {
  int S;
  double a[3], b[3];
};

RkCoef rk_coef(int nstages) {
  if (nstages == 3) return RkCoef{3, {0.0, 0.75, 1.0 / 3.0}, {1.0, 0.25, 2.0 / 3.0}};
  return RkCoef{2, {0.0, 0.5, 0.0}, {1.0, 0.5, 0.0}};
}

// weight of stage s's dt L term in U^{n+1}: b_s times the b of every later stage
double rk_weight(const RkCoef& r, int s) {
  double w = r.b[s];
  for (int t = s + 1; t < r.S; ++t) w = w * r.b[t];
  return w;
}

// output buffer of stage s: the scratch states, the last stage writes U
double* stage_out(gbh_ctx* c, int s, double* U) {
  if (s == c->nstages - 1) return U;
  return s == 0 ? c->d_scratch : c->d_scratch2;
}

double* flux_regs(gbh_ctx* c, int s) { return s == 0 ? c->d_flux_reg : s == 1 ? c->d_flux_reg2 : c->d_flux_reg3; }

// Primitive variables carried through the stages of one entry-point call
// (non-telescoping steps): `in` is the array holding the primitives of the
// current state (-1: none, so the next stage converts on load); each stage's
// epilogue writes those of its output into the other array, except the
// call's last stage unless last_out.  A state handed in by the caller is
// always converted on load.
struct PrimChain {
  int in = -1;
  bool last_out = false;
};

// The primitive arrays stage st of r reads and writes under the chain pc (null
// when the carry is off), and the chain advanced past the stage.
void chain_stage(gbh_ctx* c, PrimChain* pc, bool last, double** Win, double** Wout) {
  *Win = *Wout = nullptr;
  if (!pc || c->telescoping || !c->prim_carry || !c->d_W[0]) return;
  const int wo = (!last || pc->last_out) ? (pc->in == 0 ? 1 : 0) : -1;
  if (pc->in >= 0) *Win = c->d_W[pc->in];
  if (wo >= 0) *Wout = c->d_W[wo];
  pc->in = wo;
}

// One SSP-RK step on a two-level grid, all-levels non-telescoping; ends with
// the restriction of the new state so that covered coarse cells hold the
// mean of their children.  dt_epilogue: the CFL max of the new leaf cells goes
// into the accumulator (the restriction changes covered blocks only).
int refined_step(gbh_ctx* c, double* U, const double* dt_dev, double dt, bool dt_epilogue, cudaStream_t s,
                 PrimChain* pc = nullptr) {
  const RkCoef r = rk_coef(c->nstages);
  double* in = U;
  for (int st = 0; st < r.S; ++st) {
    double* out = stage_out(c, st, U);
    double *Win, *Wout;
    chain_stage(c, pc, st == r.S - 1, &Win, &Wout);
    int rc = refined_stage(c, in, st ? U : nullptr, out, dt_dev, dt, r.a[st], r.b[st],
                           dt_epilogue && st == r.S - 1, s, Win, Wout);
    if (rc) return rc;
    in = out;
  }
  return cuda_err(c, gbh::launch_restrict(U, c->amr, s), "restrict launch");
}

// One SSP-RK step on a uniform (or batched) grid.  Non-telescoping: every
// stage gathers its halo from the neighbours.  Telescoping (Sec. 4.2): one
// guard fill of U (all layers), then stage s of S updates the interior
// widened by 2 (S - s) cells from its input's own guard cells; no exchange
// between the stages.  The last stage may carry the dt epilogue.  pc: the
// call's primitive chain (non-telescoping; null or no arrays: every stage
// converts on load).
int uniform_step(gbh_ctx* c, double* U, const double* dt_dev, double dt, bool dt_epilogue, cudaStream_t s,
                 PrimChain* pc = nullptr) {
  const RkCoef r = rk_coef(c->nstages);
  int rc = GBH_OK;
  if (c->telescoping) {
    gbh::FillArgs F{U, c->d_nbr, c->d_face, c->lay};
    if ((rc = cuda_err(c, gbh::launch_fill(F, s), "fill kernel launch"))) return rc;
  }
  const double* in = U;
  for (int st = 0; st < r.S; ++st) {
    double* out = stage_out(c, st, U);
    const bool last = st == r.S - 1;
    const int ring = c->telescoping ? 2 * (r.S - 1 - st) : 0;
    double *Win, *Wout;
    chain_stage(c, pc, last, &Win, &Wout);
    rc = stage_launch(c, in, st ? U : nullptr, out, dt_dev, dt, r.a[st], r.b[st], !c->telescoping,
                      last && dt_epilogue, s, ring, nullptr, nullptr, 0, Win, Wout);
    if (rc) return rc;
    in = out;
  }
  return GBH_OK;
}

// One SSP-RK step on a two-level grid in the level-by-level telescoping
// variant (Sec. 4.2, Fig. "Level-by-levels, Telescoping"): one guard fill for
// both levels (restriction, same-level copies, prolongation of all guard
// layers), every stage of every leaf block from its own guard data with the
// coarse-fine face fluxes of stage s in register set s, the coarse-side
// correction with each stage's weight in U^{n+1}, restriction.  The two
// levels need no data from each other inside the step, so both go through
// the same launches; the paper's finest-first level loop orders nothing here.
// dt_epilogue: the CFL max of the new leaf cells goes into the accumulator
// (the last stage's epilogue, and the last correction for the cells it changes).
int refined_telescoping_step(gbh_ctx* c, double* U, const double* dt_dev, double dt, bool dt_epilogue,
                             cudaStream_t s) {
  const RkCoef r = rk_coef(c->nstages);
  int rc = cuda_err(c, gbh::launch_restrict(U, c->amr, s), "restrict launch");
  if (rc) return rc;
  gbh::FillArgs F{U, c->d_nbr, c->d_face, c->lay};
  if ((rc = cuda_err(c, gbh::launch_fill(F, s), "fill kernel launch"))) return rc;
  if ((rc = cuda_err(c, gbh::launch_prolong(U, c->amr, c->lay.g, false, s), "prolong launch"))) return rc;
  const double* in = U;
  for (int st = 0; st < r.S; ++st) {
    double* out = stage_out(c, st, U);
    rc = stage_launch(c, in, st ? U : nullptr, out, dt_dev, dt, r.a[st], r.b[st], false,
                      dt_epilogue && st == r.S - 1, s, 2 * (r.S - 1 - st), flux_regs(c, st));
    if (rc) return rc;
    in = out;
  }
  for (int st = 0; st < r.S; ++st) {
    gbh::AmrArgs A = c->amr;
    A.flux_reg = flux_regs(c, st);
    unsigned long long* acc = dt_epilogue && st == r.S - 1 ? c->d_smax : nullptr;
    if ((rc = cuda_err(c, gbh::launch_reflux(U, A, dt_dev, dt, rk_weight(r, st), acc, s), "reflux launch")))
      return rc;
  }
  return cuda_err(c, gbh::launch_restrict(U, c->amr, s), "restrict launch");
}

gbh::DtArgs dt_args(gbh_ctx* c, const double* U) {
  gbh::DtArgs A{U, c->d_inv_dx, c->lay, c->eos, c->d_smax, nullptr, 0};
  if (c->refined) {
    A.block_list = c->d_active;
    A.nlist = c->nactive;
  }
  return A;
}

// CFL time step(s) of U into dt_dev (one per problem) and, if given, hist.
int reduce_dt(gbh_ctx* c, const double* U, double* dt_dev, double* hist, cudaStream_t s) {
  cudaError_t e = c->d_problem ? gbh::launch_dt_reduce_blocks(dt_args(c, U), c->d_problem, s)
                               : gbh::launch_dt_reduce(dt_args(c, U), s);
  int rc = cuda_err(c, e, "dt reduce launch");
  if (rc) return rc;
  return cuda_err(c, gbh::launch_dt_finalize(c->d_smax, c->cfl, dt_dev, hist, s, c->nproblems),
                  "dt finalize launch");
}

int ensure_adjoint_buffers(gbh_ctx* c) {
  const size_t bytes = sizeof(double) * (size_t)state_elems(c->lay);
  cudaError_t e = cudaSuccess;
  // face slots: the interior faces, or in the telescoping mode the faces of
  // the widest ring stage's box
  const size_t slots = gbh::stage_vjp_scratch_doubles(c->lay, c->telescoping ? 2 * (c->nstages - 1) : 0);
  if (c->d_adj_lamW && c->adj_slot_doubles < slots) {
    cudaFree(c->d_adj_lamW);
    c->d_adj_lamW = nullptr;
  }
  if (!c->d_adj_lamW) {
    e = cudaMalloc(&c->d_adj_lamW, sizeof(double) * slots);
    c->adj_slot_doubles = e == cudaSuccess ? slots : 0;
  }
  if (e == cudaSuccess && !c->d_adj_tmp) e = cudaMalloc(&c->d_adj_tmp, bytes);
  if (e == cudaSuccess && !c->d_adj_prim) e = cudaMalloc(&c->d_adj_prim, bytes);
  if (e == cudaSuccess && c->nstages == 3 && !c->d_adj_tmp2) e = cudaMalloc(&c->d_adj_tmp2, bytes);
  if (e == cudaSuccess && c->telescoping && !c->d_adj_fill) e = cudaMalloc(&c->d_adj_fill, bytes);
  if (e == cudaSuccess && c->telescoping && !c->d_adj_tele) e = cudaMalloc(&c->d_adj_tele, bytes);
  if (e != cudaSuccess) return set_err(c, GBH_ERR_NOMEM, "adjoint buffers: %s", cudaGetErrorString(e));
  return GBH_OK;
}

gbh::StageArgs vjp_args(gbh_ctx* c, const double* U) {
  gbh::StageArgs A{};
  gbh::stage_args_common(&A, c->lay, c->eos);
  A.Uin = U;
  A.face_nbr = c->d_face;
  A.inv_dx = c->d_inv_dx;
  A.gather = 1;
  return A;
}

int adjoint_supported(gbh_ctx* c) {
  if (c->refined) return set_err(c, GBH_ERR_UNSUPPORTED, "the adjoint is not implemented on two-level contexts");
  if (c->nproblems > 1) return set_err(c, GBH_ERR_UNSUPPORTED, "the adjoint takes one dt: not on batched contexts");
  return GBH_OK;
}

void drop_graph(gbh_ctx* c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  c->graph_U = nullptr;
  c->graph_dt = nullptr;
  c->graph_steps = 0;
}

}  // namespace

namespace gbh {

int validate_params(const gbh_params* p, bool allow_coarser) {
  if (!p) return set_err(nullptr, GBH_ERR_INVAL, "params is NULL");
  if (p->ndim != 2 && p->ndim != 3) return set_err(nullptr, GBH_ERR_INVAL, "ndim must be 2 or 3 (got %d)", p->ndim);
  if (p->nblocks < 1) return set_err(nullptr, GBH_ERR_INVAL, "nblocks must be >= 1");
  if (p->nxb < 1 || p->nyb < 1 || p->nzb < 1) return set_err(nullptr, GBH_ERR_INVAL, "block sizes must be >= 1");
  if (p->ndim == 2 && p->nzb != 1) return set_err(nullptr, GBH_ERR_INVAL, "2-D requires nzb == 1");
  if (p->ndim == 3 && p->nzb < 2) return set_err(nullptr, GBH_ERR_INVAL, "3-D requires nzb >= 2");
  if (p->nguard < 2) return set_err(nullptr, GBH_ERR_INVAL, "nguard must be >= 2 (the stencil reads 2 cells)");
  int nmin = p->nxb < p->nyb ? p->nxb : p->nyb;
  if (p->ndim == 3 && p->nzb < nmin) nmin = p->nzb;
  if (p->nguard > nmin) return set_err(nullptr, GBH_ERR_INVAL, "nguard (%d) must not exceed the block size (%d)", p->nguard, nmin);
  if (!(p->gamma > 1.0) || !std::isfinite(p->gamma)) return set_err(nullptr, GBH_ERR_INVAL, "gamma must be > 1");
  if (!(p->cfl > 0.0 && p->cfl <= 1.0)) return set_err(nullptr, GBH_ERR_INVAL, "cfl must be in (0, 1]");
  if (!(p->small_rho > 0.0) || !(p->small_p > 0.0)) return set_err(nullptr, GBH_ERR_INVAL, "floors must be > 0");
  if (!(p->small_rho >= 1e-150))
    return set_err(nullptr, GBH_ERR_INVAL,
                   "small_rho must be >= 1e-150 (the HLLC flux takes 1/sqrt(rho_L rho_R), which must stay a normal number)");
  if (!p->nbr || !p->dx) return set_err(nullptr, GBH_ERR_INVAL, "nbr and dx tables are required");
  const int nn = p->ndim == 3 ? 27 : 9;
  const int centre = p->ndim == 3 ? 13 : 4;
  for (long long b = 0; b < p->nblocks; ++b) {
    for (int e = 0; e < nn; ++e) {
      const int v = p->nbr[b * nn + e];
      if (v >= p->nblocks || (v < 0 && v != GBH_BC_OUTFLOW && !(allow_coarser && v == GBH_NBR_COARSER)))
        return set_err(nullptr, GBH_ERR_INVAL, "nbr[%lld][%d] = %d is out of range", b, e, v);
    }
    if (p->nbr[b * nn + centre] != (int)b)
      return set_err(nullptr, GBH_ERR_INVAL, "nbr[%lld] centre entry must be the block itself", b);
    for (int d = 0; d < 3; ++d) {
      const double h = p->dx[b * 3 + d];
      if (d < p->ndim && !(h > 0.0 && std::isfinite(h)))
        return set_err(nullptr, GBH_ERR_INVAL, "dx[%lld][%d] must be finite and > 0", b, d);
    }
  }
  if (p->nxb != p->nyb || (p->nxb != 4 && p->nxb != 8 && p->nxb != 16))
    return set_err(nullptr, GBH_ERR_UNSUPPORTED, "this build supports nxb == nyb in {4, 8, 16} (got %d x %d)", p->nxb, p->nyb);
  return GBH_OK;
}

void layout_from_params(const gbh_params* p, Layout* L, Eos* e) {
  L->ndim = p->ndim;
  L->nx = p->nxb;
  L->ny = p->nyb;
  L->nz = p->nzb;
  L->g = p->nguard;
  L->gz = p->ndim == 3 ? p->nguard : 0;
  L->nxp = L->nx + 2 * L->g;
  L->nyp = L->ny + 2 * L->g;
  L->nzp = L->nz + 2 * L->gz;
  L->nblocks = p->nblocks;
  L->vstride = (long long)L->nxp * L->nyp * L->nzp;
  L->bstride = 5 * L->vstride;
  e->gamma = p->gamma;
  e->gm1 = p->gamma - 1.0;
  e->inv_gm1 = 1.0 / (p->gamma - 1.0);
  e->g_gm1 = p->gamma / (p->gamma - 1.0);
  e->small_rho = p->small_rho;
  e->small_p = p->small_p;
  e->hgm1 = 0.5 * (p->gamma - 1.0);
  e->k.one = 1.0;
  e->k.nz = -0.0;
  e->opaque = 0;
}

void face_table_from_params(const gbh_params* p, long long b, int face[6], double inv_dx[3]) {
  const int nn = p->ndim == 3 ? 27 : 9;
  const int32_t* row = p->nbr + b * nn;
  auto at = [&](int ox, int oy, int oz) {
    return p->ndim == 3 ? row[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)] : row[(oy + 1) * 3 + (ox + 1)];
  };
  face[0] = at(-1, 0, 0);
  face[1] = at(1, 0, 0);
  face[2] = at(0, -1, 0);
  face[3] = at(0, 1, 0);
  face[4] = p->ndim == 3 ? at(0, 0, -1) : GBH_BC_OUTFLOW;
  face[5] = p->ndim == 3 ? at(0, 0, 1) : GBH_BC_OUTFLOW;
  for (int d = 0; d < 3; ++d) inv_dx[d] = (d < p->ndim) ? 1.0 / p->dx[3 * b + d] : 0.0;
}

void stage_args_common(StageArgs* A, const Layout& L, const Eos& e) {
  A->lay = L;
  A->eos = e;
  A->kchunk = L.ndim == 3 ? L.nz : 1;   // one work item per block
  A->nchunks = 1;
  A->items_per_cta = 1;
  A->ysplit = 1;
}

int set_create_error(int code, const char* msg) { return set_err(nullptr, code, "%s", msg); }

}  // namespace gbh

using gbh::validate_params;

static int create_common(const gbh_params* p, gbh_ctx** out);
extern "C" int gbh_destroy(gbh_ctx* c);

static int step_cfl(gbh_ctx* c, double* U, double* dt_dev, cudaStream_t s, PrimChain* pc) {
  int rc = c->refined ? (c->telescoping ? refined_telescoping_step(c, U, dt_dev, 0.0, true, s)
                                        : refined_step(c, U, dt_dev, 0.0, true, s, pc))
                      : uniform_step(c, U, dt_dev, 0.0, true, s, pc);
  if (rc) return rc;
  return cuda_err(c, gbh::launch_dt_finalize(c->d_smax, c->cfl, dt_dev, nullptr, s, c->nproblems),
                  "dt finalize launch");
}



// The two arrays of the primitive carry.  If they cannot
// be allocated the carry stays off and every stage converts on load (the
// results are the same bit for bit); returns whether it is on.
// The face pre-pass buffer (uniform contexts); off if it cannot be allocated.
// Switched on at creation for 3-D contexts only: in 2-D a block plane has few
// boundary faces for what the extra launch costs (the 96-problem 2-D ensemble
// measured 1.2% slower with it, the 256^3 3-D step 3.3% faster).
static bool alloc_face_buffer(gbh_ctx* c, bool at_create = false) {
  if (at_create && c->lay.ndim != 3) return false;
  if (!c->d_bflux) {
    const size_t nf = (size_t)c->lay.nx * (c->lay.ndim == 3 ? (c->lay.nz > c->lay.nx ? c->lay.nz : c->lay.nx) : 1);
    if (cudaMalloc(&c->d_bflux, sizeof(double) * 6 * 5 * nf * (size_t)c->lay.nblocks) != cudaSuccess) {
      c->d_bflux = nullptr;
      cudaGetLastError();
      c->face_prepass = false;
      return false;
    }
  }
  c->face_prepass = true;
  return true;
}

static bool alloc_prim_buffers(gbh_ctx* c) {
  if (!c->d_W[0]) {
    const size_t bytes = sizeof(double) * state_elems(c->lay);
    double *w0 = nullptr, *w1 = nullptr;
    if (cudaMalloc(&w0, bytes) != cudaSuccess || cudaMalloc(&w1, bytes) != cudaSuccess) {
      cudaFree(w0);
      cudaFree(w1);
      cudaGetLastError();      // the failed allocation is not an error of the context
      c->prim_carry = false;
      return false;
    }
    c->d_W[0] = w0;
    c->d_W[1] = w1;
  }
  c->prim_carry = true;
  return true;
}

static int create_common(const gbh_params* p, gbh_ctx** out) {
  gbh_ctx* c = new (std::nothrow) gbh_ctx();
  if (!c) return set_err(nullptr, GBH_ERR_NOMEM, "host allocation failed");
  gbh::layout_from_params(p, &c->lay, &c->eos);
  const Layout& L = c->lay;
  c->cfl = p->cfl;

  const int nn = p->ndim == 3 ? 27 : 9;
  std::vector<int> face(6 * (size_t)p->nblocks, GBH_BC_OUTFLOW);
  std::vector<double> inv(3 * (size_t)p->nblocks, 0.0);
  for (long long b = 0; b < p->nblocks; ++b) gbh::face_table_from_params(p, b, &face[6 * b], &inv[3 * b]);

  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_nbr, sizeof(int) * nn * (size_t)p->nblocks);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_face, sizeof(int) * face.size());
  if (e == cudaSuccess) e = cudaMalloc(&c->d_inv_dx, sizeof(double) * inv.size());
  if (e == cudaSuccess) e = cudaMalloc(&c->d_words, sizeof(unsigned long long) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_scratch, sizeof(double) * state_elems(L));
  if (e == cudaSuccess) e = cudaMemcpy(c->d_nbr, p->nbr, sizeof(int) * nn * (size_t)p->nblocks, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_face, face.data(), sizeof(int) * face.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_inv_dx, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->d_words, 0, sizeof(unsigned long long) * 4);
  if (e == cudaSuccess) e = gbh::stage_prepare(L.nx, L.ndim);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? GBH_ERR_NOMEM : GBH_ERR_CUDA;
    set_err(nullptr, code, "gbh_create: %s", cudaGetErrorString(e));
    gbh_destroy(c);
    return code;
  }
  c->d_smax = c->d_words;
  c->h_face = std::move(face);
  *out = c;
  return GBH_OK;
}


extern "C" {

int gbh_create(const gbh_params* p, gbh_ctx** out) {
  if (!out) return set_err(nullptr, GBH_ERR_INVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_params(p, false);
  if (rc) return rc;
  if ((rc = create_common(p, out))) return rc;
  alloc_prim_buffers(*out);
  alloc_face_buffer(*out, true);
  return GBH_OK;
}

// Problem ids of a batched context: in range, and no neighbour (or, on two
// levels, parent or child) in another problem.
static int check_problems(const gbh_params* p, const int32_t* problem, int nproblems, const gbh_refinement* r) {
  if (!problem || nproblems < 1) return set_err(nullptr, GBH_ERR_INVAL, "problem table and nproblems >= 1 are required");
  const int nn = p->ndim == 3 ? 27 : 9;
  for (long long b = 0; b < p->nblocks; ++b) {
    const int pb = problem[b];
    if (pb < 0 || pb >= nproblems) return set_err(nullptr, GBH_ERR_INVAL, "problem[%lld] = %d out of range", b, pb);
  }
  for (long long b = 0; b < p->nblocks; ++b) {
    const int pb = problem[b];
    for (int e = 0; e < nn; ++e) {
      const int v = p->nbr[b * nn + e];
      if (v >= 0 && problem[v] != pb)
        return set_err(nullptr, GBH_ERR_INVAL, "block %lld and its neighbour %d belong to different problems", b, v);
    }
    if (r) {
      const int P = r->parent[4 * b];
      if (P >= 0 && P < p->nblocks && problem[P] != pb)
        return set_err(nullptr, GBH_ERR_INVAL, "block %lld and its parent %d belong to different problems", b, P);
    }
  }
  return GBH_OK;
}

// Per-block problem ids and per-problem CFL accumulators on a new context.
static int attach_problems(gbh_ctx* c, const gbh_params* p, const int32_t* problem, int nproblems) {
  cudaError_t e = cudaMalloc(&c->d_problem, sizeof(int) * (size_t)p->nblocks);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_problem, problem, sizeof(int) * (size_t)p->nblocks, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_smax_own, sizeof(unsigned long long) * nproblems);
  if (e == cudaSuccess) e = cudaMemset(c->d_smax_own, 0, sizeof(unsigned long long) * nproblems);
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? GBH_ERR_NOMEM : GBH_ERR_CUDA;
    return set_err(nullptr, code, "problem tables: %s", cudaGetErrorString(e));
  }
  c->d_smax = c->d_smax_own;
  c->nproblems = nproblems;
  c->amr.problem = c->d_problem;
  return GBH_OK;
}

int gbh_create_refined_batched(const gbh_params* p, const gbh_refinement* r, const int32_t* problem, int nproblems,
                               gbh_ctx** out) {
  if (!out) return set_err(nullptr, GBH_ERR_INVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_params(p, true);
  if (rc) return rc;
  if (!r || !r->parent || !r->children) return set_err(nullptr, GBH_ERR_INVAL, "refinement tables are required");
  for (long long b = 0; b < p->nblocks; ++b)
    if (r->parent[4 * b] >= p->nblocks) return set_err(nullptr, GBH_ERR_INVAL, "parent[%lld] out of range", b);
  if ((rc = check_problems(p, problem, nproblems, r))) return rc;
  gbh_ctx* c = nullptr;
  if ((rc = gbh_create_refined(p, r, &c))) return rc;
  if ((rc = attach_problems(c, p, problem, nproblems))) {
    gbh_destroy(c);
    return rc;
  }
  *out = c;
  return GBH_OK;
}

int gbh_create_refined(const gbh_params* p, const gbh_refinement* r, gbh_ctx** out) {
  if (!out) return set_err(nullptr, GBH_ERR_INVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_params(p, true);
  if (rc) return rc;
  if (!r || !r->parent || !r->children) return set_err(nullptr, GBH_ERR_INVAL, "refinement tables are required");
  const int nd = p->ndim, nn = nd == 3 ? 27 : 9, nch = nd == 3 ? 8 : 4;
  const int n[3] = {p->nxb, p->nyb, p->nzb};
  if (p->nxb % 2 || (nd == 3 && p->nzb != p->nxb))
    return set_err(nullptr, GBH_ERR_UNSUPPORTED, "two-level grids need even, cubic (3-D) or square (2-D) blocks");
  const long long NB = p->nblocks;
  const int32_t* par = r->parent;
  const int32_t* chl = r->children;
  for (long long b = 0; b < NB; ++b) {
    const int P = par[4 * b];
    if (P < 0) {
      if (P != -1 || par[4 * b + 1] || par[4 * b + 2] || par[4 * b + 3])
        return set_err(nullptr, GBH_ERR_INVAL, "parent[%lld] of a level-0 block must be (-1, 0, 0, 0)", b);
      for (int e = 0; e < nn; ++e)
        if (p->nbr[b * nn + e] == GBH_NBR_COARSER)
          return set_err(nullptr, GBH_ERR_INVAL, "level-0 block %lld has a GBH_NBR_COARSER entry", b);
      continue;
    }
    if (P >= NB || par[4 * P] != -1)
      return set_err(nullptr, GBH_ERR_UNSUPPORTED, "block %lld: only two levels are supported", b);
    int oct = 0;
    for (int d = 0; d < 3; ++d) {
      const int o = par[4 * b + 1 + d];
      if (d >= nd ? o != 0 : (o != 0 && o != n[d] / 2))
        return set_err(nullptr, GBH_ERR_INVAL, "parent offset of block %lld is not 0 or n/2", b);
      if (o) oct |= 1 << d;
      if (d < nd && std::fabs(p->dx[3 * b + d] * 2.0 - p->dx[3 * P + d]) > 1e-14 * p->dx[3 * P + d])
        return set_err(nullptr, GBH_ERR_INVAL, "block %lld: cell width must be half its parent's", b);
    }
    if (chl[8 * P + oct] != (int)b)
      return set_err(nullptr, GBH_ERR_INVAL, "children of %d do not list block %lld", P, b);
  }
  for (long long b = 0; b < NB; ++b) {
    const bool has = chl[8 * b] >= 0;
    for (int o = 0; o < 8; ++o) {
      const int ch = chl[8 * b + o];
      if (!has || o >= nch) {
        if (ch != -1) return set_err(nullptr, GBH_ERR_INVAL, "children[%lld][%d] must be -1", b, o);
      } else if (ch < 0 || ch >= NB || par[4 * ch] != (int)b) {
        return set_err(nullptr, GBH_ERR_INVAL, "children[%lld][%d] = %d is not a child of it", b, o, ch);
      }
    }
  }
  // lists, flux-register slots and the flux-correction entries
  std::vector<int> active, covered, fine, slot(6 * (size_t)NB, -1);
  std::vector<gbh::RefluxEntry> refl;
  std::vector<int2> cf_faces;
  std::vector<int> face(6 * (size_t)NB);
  std::vector<double> inv(3);
  for (long long b = 0; b < NB; ++b) gbh::face_table_from_params(p, b, &face[6 * b], inv.data());
  int nslots = 0;
  for (long long b = 0; b < NB; ++b) {
    (chl[8 * b] >= 0 ? covered : active).push_back((int)b);
    if (par[4 * b] < 0) continue;
    bool any = false;
    for (int e = 0; e < nn; ++e) any = any || p->nbr[b * nn + e] == GBH_NBR_COARSER;
    if (any) fine.push_back((int)b);
    for (int f = 0; f < 2 * nd; ++f)
      if (face[6 * b + f] == GBH_NBR_COARSER) {
        slot[6 * b + f] = nslots++;
        cf_faces.push_back(make_int2((int)b, f));
      }
  }
  // one entry per coarse leaf face with refined blocks beyond it; a block can
  // border the refined region through several faces (an L, a notch), and
  // reflux_of names each face's entry so that a cell next to several of them
  // takes all their corrections from one thread
  std::vector<int> reflux_of(6 * (size_t)NB, -1);
  for (long long b = 0; b < NB; ++b) {
    if (par[4 * b] >= 0 || chl[8 * b] >= 0) continue;
    for (int f = 0; f < 2 * nd; ++f) {
      const int nb = face[6 * b + f];
      if (nb < 0 || chl[8 * nb] < 0) continue;
      gbh::RefluxEntry en{};
      en.block = (int)b;
      en.face = f;
      en.coarse_slot = slot[6 * b + f] = nslots++;
      const int d = f >> 1, side = f & 1;
      const int t1d = d == 0 ? 1 : 0, t2d = d == 2 ? 1 : 2;
      for (int q = 0; q < 4; ++q) en.fine_slot[q] = -1;
      for (int q2 = 0; q2 < (nd == 3 ? 2 : 1); ++q2)
        for (int q1 = 0; q1 < 2; ++q1) {
          const int oct = ((side ? 0 : 1) << d) | (q1 << t1d) | (nd == 3 ? (q2 << t2d) : 0);
          const int ch = chl[8 * nb + oct];
          const int fs = slot[6 * (size_t)ch + 2 * d + (1 - side)];
          if (fs < 0)
            return set_err(nullptr, GBH_ERR_INVAL, "fine block %d facing coarse block %lld is not marked GBH_NBR_COARSER", ch, b);
          en.fine_slot[q1 + 2 * q2] = fs;
        }
      reflux_of[6 * b + f] = (int)refl.size();
      refl.push_back(en);
    }
  }
  gbh_ctx* c = nullptr;
  if ((rc = create_common(p, &c))) return rc;
  c->refined = true;
  c->nactive = (int)active.size();
  const size_t fstride = 5 * (size_t)p->nxb * (nd == 3 ? p->nxb : 1);
  cudaError_t e = cudaMalloc(&c->d_parent, sizeof(int) * 4 * NB);
  auto up = [&](void** dst, const void* src, size_t bytes) {
    if (e != cudaSuccess) return;
    if (bytes == 0) bytes = 8;
    e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess && src) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  if (e == cudaSuccess) e = cudaMemcpy(c->d_parent, par, sizeof(int) * 4 * NB, cudaMemcpyHostToDevice);
  up((void**)&c->d_children, chl, sizeof(int) * 8 * NB);
  up((void**)&c->d_active, active.data(), sizeof(int) * active.size());
  up((void**)&c->d_covered, covered.empty() ? nullptr : covered.data(), sizeof(int) * covered.size());
  up((void**)&c->d_fine, fine.empty() ? nullptr : fine.data(), sizeof(int) * fine.size());
  up((void**)&c->d_flux_slot, slot.data(), sizeof(int) * slot.size());
  c->flux_reg_doubles = fstride * (size_t)(nslots ? nslots : 1);
  up((void**)&c->d_flux_reg, nullptr, sizeof(double) * c->flux_reg_doubles);
  up((void**)&c->d_reflux, refl.empty() ? nullptr : refl.data(), sizeof(gbh::RefluxEntry) * refl.size());
  up((void**)&c->d_reflux_of, reflux_of.data(), sizeof(int) * reflux_of.size());
  up((void**)&c->d_cf_faces, cf_faces.empty() ? nullptr : cf_faces.data(), sizeof(int2) * cf_faces.size());
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? GBH_ERR_NOMEM : GBH_ERR_CUDA;
    set_err(nullptr, code, "gbh_create_refined: %s", cudaGetErrorString(e));
    gbh_destroy(c);
    return code;
  }
  gbh::AmrArgs& A = c->amr;
  A.lay = c->lay;
  A.nbr = c->d_nbr;
  A.parent = c->d_parent;
  A.children = c->d_children;
  A.covered = c->d_covered;
  A.ncovered = (int)covered.size();
  A.fine = c->d_fine;
  A.nfine = (int)fine.size();
  A.reflux = c->d_reflux;
  A.reflux_of = c->d_reflux_of;
  A.nreflux = (int)refl.size();
  A.cf_faces = c->d_cf_faces;
  A.ncf_faces = (int)cf_faces.size();
  A.flux_reg = c->d_flux_reg;
  A.flux_reg_len = (long long)c->flux_reg_doubles;
  A.inv_dx = c->d_inv_dx;
  A.eos = c->eos;
  A.floor_count = c->d_words + 1;
  alloc_prim_buffers(c);
  alloc_face_buffer(c, true);
  *out = c;
  return GBH_OK;
}

int gbh_create_batched(const gbh_params* p, const int32_t* problem, int nproblems, gbh_ctx** out) {
  if (!out) return set_err(nullptr, GBH_ERR_INVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_params(p, false);
  if (rc) return rc;
  if ((rc = check_problems(p, problem, nproblems, nullptr))) return rc;
  gbh_ctx* c = nullptr;
  if ((rc = create_common(p, &c))) return rc;
  if ((rc = attach_problems(c, p, problem, nproblems))) {
    gbh_destroy(c);
    return rc;
  }
  alloc_prim_buffers(c);
  alloc_face_buffer(c, true);
  *out = c;
  return GBH_OK;
}

// Mean time of `reps` stage launches (after one untimed launch) into the
// context's scratch state, with the decomposition the context holds.
static int time_stage(gbh_ctx* c, const double* U, int ring, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t s,
                      float* ms) {
  int rc = GBH_OK;
  for (int rep = 0; rep < 3 && rc == GBH_OK; ++rep) {
    if (rep == 1) rc = cuda_err(c, cudaEventRecord(e0, s), "cudaEventRecord");
    if (!rc) rc = stage_launch(c, U, nullptr, c->d_scratch, nullptr, 1e-300, 0.0, 1.0, ring == 0, false, s, ring);
  }
  if (!rc) rc = cuda_err(c, cudaEventRecord(e1, s), "cudaEventRecord");
  if (!rc) rc = cuda_err(c, cudaEventSynchronize(e1), "cudaEventSynchronize");
  if (!rc) rc = cuda_err(c, cudaEventElapsedTime(ms, e0, e1), "cudaEventElapsedTime");
  return rc;
}

int gbh_autotune(gbh_ctx* c, const double* U, int* kchunk_out, int* items_out, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U || !aligned8(U)) return set_err(c, GBH_ERR_INVAL, "null or misaligned state pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const bool timing = c->timing;
  c->timing = false;
  drop_graph(c);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  std::vector<int> kcs = {0};
  if (c->lay.ndim == 3 && c->lay.nz >= 8 && c->lay.nz % 2 == 0) kcs.push_back(c->lay.nz / 2);
  std::vector<int> splits = {1};
  if (c->lay.nx >= 8) splits.push_back(2);
  const long long nlist = c->refined ? c->nactive : c->lay.nblocks;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_err(c, GBH_ERR_CUDA, "cudaEventCreate failed");
  // the interior stage: z-chunk x CTAs' items x row bands (an unsplit tile
  // keeps two CTAs per SM resident, a band four)
  float best = 1e30f;
  int best_kc = 0, best_ipc = 1, best_split = 1;
  for (int split : splits) {
    for (int kc : kcs) {
      const long long nitems = nlist * (kc > 0 ? (c->lay.nz + kc - 1) / kc : 1) * split;
      const long long resident = 2LL * split * sms;
      const long long persistent = (nitems + resident - 1) / resident;
      std::vector<int> ipcs = {1, 2, 4};
      if (persistent > 4) ipcs.push_back((int)persistent);
      for (int ipc : ipcs) {
        c->kchunk = kc;
        c->items_per_cta = ipc;
        c->ysplit[0] = split;
        float ms = 0.f;
        if ((rc = time_stage(c, U, 0, e0, e1, s, &ms))) break;
        if (ms < best) {
          best = ms;
          best_kc = kc;
          best_ipc = ipc;
          best_split = split;
        }
      }
      if (rc) break;
    }
    if (rc) break;
  }
  c->kchunk = best_kc;
  c->items_per_cta = best_ipc;
  c->ysplit[0] = best_split;
  // the ring stages of the telescoping mode (ring 2; and 4 with three
  // stages): row bands with the decomposition chosen above, on U's own guard
  // cells as they are (the time does not depend on their values)
  if (!rc && c->telescoping) {
    for (int ring = 2; ring <= 2 * (c->nstages - 1) && !rc; ring += 2) {
      if (c->lay.g < ring + 2) continue;
      float best_r = 1e30f;
      int pick = 1;
      for (int split : splits) {
        c->ysplit[ring / 2] = split;
        float ms = 0.f;
        if ((rc = time_stage(c, U, ring, e0, e1, s, &ms))) break;
        if (ms < best_r) {
          best_r = ms;
          pick = split;
        }
      }
      c->ysplit[ring / 2] = pick;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timing = timing;
  cudaMemsetAsync(c->d_words + 1, 0, sizeof(unsigned long long), s);   // trial launches may count floors
  if (rc) return rc;
  if (kchunk_out) *kchunk_out = best_kc > 0 ? best_kc : c->lay.nz;
  if (items_out) *items_out = best_ipc;
  return GBH_OK;
}

int gbh_set_tile_split(gbh_ctx* c, int ring, int ysplit) {
  if (!c) return set_err(nullptr, GBH_ERR_INVAL, "null context");
  if (ring != 0 && ring != 2 && ring != 4) return set_err(c, GBH_ERR_INVAL, "ring must be 0, 2 or 4 (got %d)", ring);
  if (ysplit != 1 && !(ysplit == 2 && c->lay.nx >= 8))
    return set_err(c, GBH_ERR_INVAL, "ysplit must be 1, or 2 for blocks of at least 8 cells per side (got %d)",
                   ysplit);
  drop_graph(c);
  c->ysplit[ring / 2] = ysplit;
  return GBH_OK;
}

int gbh_get_tile_split(gbh_ctx* c, int ring, int* ysplit) {
  if (!c) return set_err(nullptr, GBH_ERR_INVAL, "null context");
  if (ring != 0 && ring != 2 && ring != 4) return set_err(c, GBH_ERR_INVAL, "ring must be 0, 2 or 4 (got %d)", ring);
  if (!ysplit) return set_err(c, GBH_ERR_INVAL, "null output pointer");
  *ysplit = c->ysplit[ring / 2];
  return GBH_OK;
}

// Buffers a (telescoping, nstages) combination needs: a second scratch state
// for three stages, one flux-register set per stage on two-level contexts
// in the telescoping mode.
static int ensure_step_buffers(gbh_ctx* c, bool telescoping, int nstages) {
  cudaError_t e = cudaSuccess;
  if (nstages == 3 && !c->d_scratch2) e = cudaMalloc(&c->d_scratch2, sizeof(double) * state_elems(c->lay));
  if (e == cudaSuccess && c->refined && telescoping) {
    if (!c->d_flux_reg2) e = cudaMalloc(&c->d_flux_reg2, sizeof(double) * c->flux_reg_doubles);
    if (e == cudaSuccess && nstages == 3 && !c->d_flux_reg3)
      e = cudaMalloc(&c->d_flux_reg3, sizeof(double) * c->flux_reg_doubles);
  }
  if (e != cudaSuccess) return set_err(c, GBH_ERR_NOMEM, "step buffers: %s", cudaGetErrorString(e));
  return GBH_OK;
}

int gbh_set_host_pipeline(gbh_ctx* c, int chunks) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (chunks < 0 || chunks > 64) return set_err(c, GBH_ERR_INVAL, "chunks must be in [0, 64] (got %d)", chunks);
  for (cudaEvent_t ev : c->pipe_ev) cudaEventDestroy(ev);
  c->pipe_ev.clear();
  c->pipe_chunks = 0;          // chunks and events are set up again on the next hydro_step_host
  c->pipe_chunks_wanted = chunks;
  return GBH_OK;
}

int gbh_set_telescoping(gbh_ctx* c, int enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (enable && c->lay.g < 2 * c->nstages)
    return set_err(c, GBH_ERR_INVAL, "the telescoping mode with %d stages needs nguard >= %d (got %d)", c->nstages,
                   2 * c->nstages, c->lay.g);
  if ((rc = ensure_step_buffers(c, enable != 0, c->nstages))) return rc;
  drop_graph(c);
  c->telescoping = enable != 0;
  return GBH_OK;
}

int gbh_set_rk_stages(gbh_ctx* c, int nstages) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (nstages != 2 && nstages != 3) return set_err(c, GBH_ERR_INVAL, "nstages must be 2 or 3 (got %d)", nstages);
  if (c->telescoping && c->lay.g < 2 * nstages)
    return set_err(c, GBH_ERR_INVAL, "the telescoping mode with %d stages needs nguard >= %d (got %d)", nstages,
                   2 * nstages, c->lay.g);
  if ((rc = ensure_step_buffers(c, c->telescoping, nstages))) return rc;
  drop_graph(c);
  c->nstages = nstages;
  return GBH_OK;
}

int gbh_set_prim_carry(gbh_ctx* c, int enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  drop_graph(c);
  if (!enable) {
    cudaError_t e = cudaDeviceSynchronize();   // no stage in flight may still use the arrays
    cudaFree(c->d_W[0]);
    cudaFree(c->d_W[1]);
    c->d_W[0] = c->d_W[1] = nullptr;
    c->prim_carry = false;
    return cuda_err(c, e, "cudaDeviceSynchronize");
  }
  if (!alloc_prim_buffers(c)) return set_err(c, GBH_ERR_NOMEM, "primitive arrays: device allocation failed");
  return GBH_OK;
}

int gbh_set_face_prepass(gbh_ctx* c, int enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  drop_graph(c);
  if (!enable) {
    c->face_prepass = false;
    return GBH_OK;
  }
  if (!alloc_face_buffer(c)) return set_err(c, GBH_ERR_NOMEM, "face pre-pass buffer: device allocation failed");
  return GBH_OK;
}

int gbh_get_face_prepass(gbh_ctx* c, int* enabled) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!enabled) return set_err(c, GBH_ERR_INVAL, "enabled is NULL");
  *enabled = c->face_prepass && c->d_bflux ? 1 : 0;
  return GBH_OK;
}

int gbh_get_prim_carry(gbh_ctx* c, int* enabled) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!enabled) return set_err(c, GBH_ERR_INVAL, "enabled is NULL");
  *enabled = c->prim_carry && c->d_W[0] ? 1 : 0;
  return GBH_OK;
}

int gbh_set_decomposition(gbh_ctx* c, int kchunk, int items_per_cta) {
  if (!c) return set_err(nullptr, GBH_ERR_INVAL, "null context");
  if (items_per_cta < 1 || kchunk < 0 || (kchunk > 0 && (c->lay.ndim != 3 || kchunk < 2 || kchunk > c->lay.nz)))
    return set_err(c, GBH_ERR_INVAL, "invalid decomposition (kchunk %d, items per CTA %d)", kchunk, items_per_cta);
  drop_graph(c);
  c->kchunk = (kchunk == c->lay.nz) ? 0 : kchunk;
  c->items_per_cta = items_per_cta;
  return GBH_OK;
}

int hydro_advance_graph(gbh_ctx* c, double* U, int nsteps, double* dt_dev, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (nsteps < 1) return set_err(c, GBH_ERR_INVAL, "nsteps must be >= 1");
  if (!U || !dt_dev || !aligned8(U) || !aligned8(dt_dev)) return set_err(c, GBH_ERR_INVAL, "null or misaligned pointer");
  if (c->timing) return set_err(c, GBH_ERR_INVAL, "disable kernel timing before capturing a graph");
  if (!(c->graph_exec && c->graph_U == U && c->graph_dt == dt_dev && c->graph_steps == nsteps)) {
    drop_graph(c);
    cudaError_t e = cudaSuccess;
    if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_err(c, e, "begin capture");
    PrimChain pc;
    for (int n = 0; n < nsteps && rc == GBH_OK; ++n) {
      pc.last_out = n < nsteps - 1;
      rc = step_cfl(c, U, dt_dev, c->cap_stream, &pc);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_err(c, e, "end capture");
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->graph_exec = nullptr;
      return cuda_err(c, e, "graph instantiate");
    }
    c->graph_U = U;
    c->graph_dt = dt_dev;
    c->graph_steps = nsteps;
  }
  return cuda_err(c, cudaGraphLaunch(c->graph_exec, (cudaStream_t)stream), "graph launch");
}

int hydro_stage_vjp(gbh_ctx* c, const double* U, const double* M, double scale, const double* A, double cA,
                    const double* B, double cB, double* out, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = adjoint_supported(c))) return rc;
  if (!U || !M || !out || !aligned8(U) || !aligned8(M) || !aligned8(out) || (A && !aligned8(A)) || (B && !aligned8(B)))
    return set_err(c, GBH_ERR_INVAL, "null or misaligned pointer");
  if (!std::isfinite(scale) || !std::isfinite(cA) || !std::isfinite(cB)) return set_err(c, GBH_ERR_INVAL, "non-finite coefficient");
  const long long n = state_elems(c->lay);
  if ((out < U + n && U < out + n) || (out < M + n && M < out + n))
    return set_err(c, GBH_ERR_INVAL, "out must not overlap U or M");
  if ((rc = ensure_adjoint_buffers(c))) return rc;
  return cuda_err(c, gbh::launch_stage_vjp(vjp_args(c, U), M, scale, A, cA, B, cB, c->d_adj_lamW, c->d_adj_prim, out,
                                           (cudaStream_t)stream), "stage VJP launch");
}

// Adjoint of one telescoping step (Sec. 4.2, telescoping mode; readings C17,
// C18).  Forward, recomputed: Uf = fill(Un) with all guard layers, then the
// ring stages X_1 .. X_{S-1} (stage s updates the box of ring width
// 2 (S - 1 - s) from its input's own cells), then U^{n+1} = a Uf + b (X_{S-1}
// + dt L(X_{S-1})) on the interior.  Backward: with M the cotangent of
// stage s's output on its box, the cotangent of its input is
// b_s M + J_L(X_s)^T (b_s dt M), and a_s M goes to Uf directly; the last VJP
// (stage 0, on Uf) adds the direct terms, and the reverse of the fill gives
// dJ/dUn.  Every VJP reads the blocks' own padded cells (no halo gather).
static int step_adjoint_telescoping(gbh_ctx* c, const double* Un, double dt, const double* lam, double* lam_prev,
                                    cudaStream_t s) {
  const RkCoef r = rk_coef(c->nstages);
  const long long n = state_elems(c->lay);
  int rc = cuda_err(c, cudaMemcpyAsync(c->d_adj_fill, Un, sizeof(double) * n, cudaMemcpyDeviceToDevice, s),
                    "cudaMemcpyAsync");
  if (rc) return rc;
  gbh::FillArgs F{c->d_adj_fill, c->d_nbr, c->d_face, c->lay};
  if ((rc = cuda_err(c, gbh::launch_fill(F, s), "fill kernel launch"))) return rc;
  double* X[3] = {c->d_adj_fill, c->d_scratch, c->d_scratch2};
  for (int st = 0; st + 1 < r.S; ++st) {
    rc = stage_launch(c, X[st], st ? X[0] : nullptr, X[st + 1], nullptr, dt, r.a[st], r.b[st], false, false, s,
                      2 * (r.S - 1 - st));
    if (rc) return rc;
  }
  // cotangents of the stages' outputs: M[S] = lam (interior); M[s] = that of X_s
  const double* M[4] = {nullptr, nullptr, nullptr, nullptr};
  double* cur[3] = {c->d_adj_tele, c->d_adj_tmp, c->d_adj_tmp2};
  M[r.S] = lam;
  for (int st = r.S - 1; st >= 0; --st) {
    const int ring = 2 * (r.S - 1 - st);
    const double* Xt[3];
    double ct[3];
    int rt[3];
    int nt = 0;
    Xt[nt] = M[st + 1]; ct[nt] = r.b[st]; rt[nt] = ring; ++nt;
    if (st == 0)   // the direct terms a_s M_{s+1} of the later stages
      for (int q = 1; q < r.S; ++q) {
        Xt[nt] = M[q + 1]; ct[nt] = r.a[q]; rt[nt] = 2 * (r.S - 1 - q); ++nt;
      }
    gbh::StageArgs A = vjp_args(c, X[st]);
    A.gather = 0;
    rc = cuda_err(c, gbh::launch_stage_vjp_box(A, ring, M[st + 1], r.b[st] * dt, Xt, ct, rt, nt, c->d_adj_lamW,
                                                c->d_adj_prim, cur[st], s), "box VJP launch");
    if (rc) return rc;
    M[st] = cur[st];
  }
  return cuda_err(c, gbh::launch_fill_vjp(c->lay, c->d_nbr, c->d_face, c->d_adj_tele, lam_prev, s),
                  "fill VJP launch");
}

static int step_adjoint_common(gbh_ctx* c, const double* Un, const double* U1, double dt, const double* lam_next,
                               double* lam_prev, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = adjoint_supported(c))) return rc;
  if ((rc = check_dt(c, dt))) return rc;
  if (!Un || !lam_next || !lam_prev || !aligned8(Un) || !aligned8(lam_next) || !aligned8(lam_prev) ||
      (U1 && !aligned8(U1)))
    return set_err(c, GBH_ERR_INVAL, "null or misaligned pointer");
  const long long n = state_elems(c->lay);
  if (lam_prev < Un + n && Un < lam_prev + n) return set_err(c, GBH_ERR_INVAL, "lam_prev must not overlap Un");
  if (U1 && lam_prev < U1 + n && U1 < lam_prev + n) return set_err(c, GBH_ERR_INVAL, "lam_prev must not overlap U1");
  if ((rc = ensure_adjoint_buffers(c))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (c->telescoping) {
    if (U1) return set_err(c, GBH_ERR_UNSUPPORTED, "the stored-state adjoint is of the non-telescoping step");
    return step_adjoint_telescoping(c, Un, dt, lam_next, lam_prev, s);
  }
  if (c->nstages == 3) {
    if (U1) return set_err(c, GBH_ERR_UNSUPPORTED, "the stored-state adjoint is of the two-stage step");
    // forward: U1 = Un + dt L(Un); U2 = 3/4 Un + 1/4 (U1 + dt L(U1))
    rc = stage_launch(c, Un, nullptr, c->d_scratch, nullptr, dt, 0.0, 1.0, true, false, s);
    if (!rc) rc = stage_launch(c, c->d_scratch, Un, c->d_scratch2, nullptr, dt, 0.75, 0.25, true, false, s);
    if (rc) return rc;
    // U^{n+1} = 1/3 Un + 2/3 (U2 + dt L(U2)):  lam_U2 = 2/3 lam + J_L(U2)^T (2/3 dt lam)
    rc = cuda_err(c, gbh::launch_stage_vjp(vjp_args(c, c->d_scratch2), lam_next, 2.0 / 3.0 * dt, lam_next, 2.0 / 3.0,
                                           nullptr, 0.0, c->d_adj_lamW, c->d_adj_prim, c->d_adj_tmp2, s),
                  "stage VJP launch");
    if (rc) return rc;
    // lam_U1 = 1/4 lam_U2 + J_L(U1)^T (1/4 dt lam_U2)
    rc = cuda_err(c, gbh::launch_stage_vjp(vjp_args(c, c->d_scratch), c->d_adj_tmp2, 0.25 * dt, c->d_adj_tmp2, 0.25,
                                           nullptr, 0.0, c->d_adj_lamW, c->d_adj_prim, c->d_adj_tmp, s),
                  "stage VJP launch");
    if (rc) return rc;
    // Un's direct terms 1/3 lam + 3/4 lam_U2, then lam_n = those + lam_U1 + J_L(Un)^T (dt lam_U1)
    rc = cuda_err(c, gbh::launch_axpby(c->lay, 0.75, c->d_adj_tmp2, 1.0 / 3.0, lam_next, c->d_adj_tmp2, s),
                  "axpby launch");
    if (rc) return rc;
    return cuda_err(c, gbh::launch_stage_vjp(vjp_args(c, Un), c->d_adj_tmp, dt, c->d_adj_tmp, 1.0, c->d_adj_tmp2, 1.0,
                                             c->d_adj_lamW, c->d_adj_prim, lam_prev, s),
                    "stage VJP launch");
  }
  if (!U1) {
    // U1 = Un + dt L(Un) (recomputed forward stage)
    rc = stage_launch(c, Un, nullptr, c->d_scratch, nullptr, dt, 0.0, 1.0, true, false, s);
    if (rc) return rc;
    U1 = c->d_scratch;
  }
  // U^{n+1} = 1/2 Un + 1/2 (U1 + dt L(U1)):  lam_U1 = 1/2 lam + J_L(U1)^T (dt/2 lam)
  rc = cuda_err(c, gbh::launch_stage_vjp(vjp_args(c, U1), lam_next, 0.5 * dt, lam_next, 0.5, nullptr, 0.0,
                                         c->d_adj_lamW, c->d_adj_prim, c->d_adj_tmp, s), "stage VJP launch");
  if (rc) return rc;
  // lam_n = 1/2 lam + lam_U1 + J_L(Un)^T (dt lam_U1)
  return cuda_err(c, gbh::launch_stage_vjp(vjp_args(c, Un), c->d_adj_tmp, dt, lam_next, 0.5, c->d_adj_tmp, 1.0,
                                           c->d_adj_lamW, c->d_adj_prim, lam_prev, s), "stage VJP launch");
}

int hydro_step_adjoint(gbh_ctx* c, const double* Un, double dt, const double* lam_next, double* lam_prev,
                       void* stream) {
  return step_adjoint_common(c, Un, nullptr, dt, lam_next, lam_prev, stream);
}

int hydro_step_adjoint_stored(gbh_ctx* c, const double* Un, const double* U1, double dt, const double* lam_next,
                              double* lam_prev, void* stream) {
  if (!U1) return set_err(c, GBH_ERR_INVAL, "U1 is NULL");
  return step_adjoint_common(c, Un, U1, dt, lam_next, lam_prev, stream);
}

int hydro_prim_to_cons(gbh_ctx* c, const double* W, double* U, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!W || !U || !aligned8(W) || !aligned8(U)) return set_err(c, GBH_ERR_INVAL, "null or misaligned pointer");
  return cuda_err(c, gbh::launch_prim_to_cons(c->lay, c->eos, W, U, nullptr, nullptr, (cudaStream_t)stream),
                  "prim_to_cons launch");
}

int hydro_prim_to_cons_vjp(gbh_ctx* c, const double* W, const double* lamU, double* lamW, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!W || !lamU || !lamW || !aligned8(W) || !aligned8(lamU) || !aligned8(lamW))
    return set_err(c, GBH_ERR_INVAL, "null or misaligned pointer");
  return cuda_err(c, gbh::launch_prim_to_cons(c->lay, c->eos, W, nullptr, lamU, lamW, (cudaStream_t)stream),
                  "prim_to_cons VJP launch");
}

int gbh_destroy(gbh_ctx* c) {
  if (!c) return GBH_OK;
  cudaDeviceSynchronize();
  cudaFree(c->d_nbr);
  cudaFree(c->d_face);
  cudaFree(c->d_inv_dx);
  cudaFree(c->d_words);
  cudaFree(c->d_scratch);
  cudaFree(c->d_W[0]);
  cudaFree(c->d_W[1]);
  cudaFree(c->d_bflux);
  cudaFree(c->d_host_state);
  cudaFree(c->d_host_dt);
  cudaFree(c->d_host_hist);
  cudaFree(c->d_parent);
  cudaFree(c->d_children);
  cudaFree(c->d_active);
  cudaFree(c->d_covered);
  cudaFree(c->d_fine);
  cudaFree(c->d_flux_slot);
  cudaFree(c->d_flux_reg);
  cudaFree(c->d_flux_reg2);
  cudaFree(c->d_flux_reg3);
  cudaFree(c->d_scratch2);
  cudaFree(c->d_reflux);
  cudaFree(c->d_reflux_of);
  cudaFree(c->d_cf_faces);
  cudaFree(c->d_problem);
  cudaFree(c->d_adj_lamW);
  cudaFree(c->d_adj_tmp);
  cudaFree(c->d_adj_prim);
  cudaFree(c->d_adj_fill);
  cudaFree(c->d_adj_tele);
  cudaFree(c->d_adj_tmp2);
  cudaFree(c->d_smax_own);
  drop_graph(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (cudaStream_t& st : c->pipe_stream)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t ev : c->pipe_ev) cudaEventDestroy(ev);
  for (cudaEvent_t& ev : c->pipe_mark)
    if (ev) cudaEventDestroy(ev);
  cudaFree(c->d_ident);
  cudaFree(c->d_pipe_out);
  cudaFree(c->d_pipe_dt);
  cudaFree(c->d_pipe_int);
  for (cudaEvent_t ev : c->ev) cudaEventDestroy(ev);
  delete c;
  return GBH_OK;
}

const char* gbh_last_error(const gbh_ctx* c) { return c ? c->err : g_create_err; }

long long gbh_state_bytes(const gbh_ctx* c) {
  return c ? (long long)sizeof(double) * state_elems(c->lay) : -1;
}

int hydro_fill_guardcells(gbh_ctx* c, double* U, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U || !aligned8(U)) return set_err(c, GBH_ERR_INVAL, "U must be a non-null 8-byte aligned device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->refined && (rc = cuda_err(c, gbh::launch_restrict(U, c->amr, s), "restrict launch"))) return rc;
  gbh::FillArgs A{U, c->d_nbr, c->d_face, c->lay};
  if ((rc = cuda_err(c, gbh::launch_fill(A, s), "fill kernel launch"))) return rc;
  if (c->refined) return cuda_err(c, gbh::launch_prolong(U, c->amr, c->lay.g, false, s), "prolong launch");
  return GBH_OK;
}

int hydro_compute_dt(gbh_ctx* c, const double* U, double* dt_dev, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U || !dt_dev || !aligned8(U) || !aligned8(dt_dev)) return set_err(c, GBH_ERR_INVAL, "null or misaligned pointer");
  return reduce_dt(c, U, dt_dev, nullptr, (cudaStream_t)stream);
}

static int stage_common(gbh_ctx* c, const double* Uin, const double* Un, double* Uout, double dt, double a,
                        double b, bool gather, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (c->refined) return set_err(c, GBH_ERR_UNSUPPORTED, "single stages are not exposed on two-level contexts");
  if ((rc = check_dt(c, dt))) return rc;
  if (!Uin || !Uout || !aligned8(Uin) || !aligned8(Uout)) return set_err(c, GBH_ERR_INVAL, "null or misaligned state pointer");
  if (!std::isfinite(a) || !std::isfinite(b)) return set_err(c, GBH_ERR_INVAL, "a and b must be finite");
  const bool combine = !(a == 0.0 && b == 1.0);
  if (combine && (!Un || !aligned8(Un))) return set_err(c, GBH_ERR_INVAL, "Un is required when (a, b) != (0, 1)");
  const long long n = state_elems(c->lay);
  if (Uin < Uout + n && Uout < Uin + n) return set_err(c, GBH_ERR_INVAL, "Uout must not overlap Uin");
  return stage_launch(c, Uin, combine ? Un : nullptr, Uout, nullptr, dt, a, b, gather, false, (cudaStream_t)stream);
}

int hydro_stage(gbh_ctx* c, const double* Uin, const double* Un, double* Uout, double dt, double a, double b,
                void* stream) {
  return stage_common(c, Uin, Un, Uout, dt, a, b, true, stream);
}

int hydro_stage_guarded(gbh_ctx* c, const double* Uin, const double* Un, double* Uout, double dt, double a,
                        double b, void* stream) {
  return stage_common(c, Uin, Un, Uout, dt, a, b, false, stream);
}

int hydro_step(gbh_ctx* c, double* U, double dt, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = check_dt(c, dt))) return rc;
  if (!U || !aligned8(U)) return set_err(c, GBH_ERR_INVAL, "null or misaligned state pointer");
  cudaStream_t s = (cudaStream_t)stream;
  PrimChain pc;
  if (c->refined)
    return c->telescoping ? refined_telescoping_step(c, U, nullptr, dt, false, s)
                          : refined_step(c, U, nullptr, dt, false, s, &pc);
  return uniform_step(c, U, nullptr, dt, false, s, &pc);
}

int hydro_step_cfl(gbh_ctx* c, double* U, double* dt_dev, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U || !dt_dev || !aligned8(U) || !aligned8(dt_dev)) return set_err(c, GBH_ERR_INVAL, "null or misaligned pointer");
  PrimChain pc;
  return step_cfl(c, U, dt_dev, (cudaStream_t)stream, &pc);
}

int hydro_advance(gbh_ctx* c, double* U, int nsteps, double* dt_dev, double* dt_hist_dev, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (nsteps < 0) return set_err(c, GBH_ERR_INVAL, "nsteps must be >= 0");
  if (!U || !dt_dev || !aligned8(U) || !aligned8(dt_dev)) return set_err(c, GBH_ERR_INVAL, "null or misaligned pointer");
  cudaStream_t s = (cudaStream_t)stream;
  PrimChain pc;
  for (int n = 0; n < nsteps; ++n) {
    pc.last_out = n < nsteps - 1;
    if (dt_hist_dev) {
      rc = cuda_err(c, cudaMemcpyAsync(dt_hist_dev + (size_t)n * c->nproblems, dt_dev,
                                       sizeof(double) * c->nproblems, cudaMemcpyDeviceToDevice, s),
                    "dt history copy");
      if (rc) return rc;
    }
    rc = step_cfl(c, U, dt_dev, s, &pc);
    if (rc) return rc;
  }
  return GBH_OK;
}

// Doubles of one block in the interior-only layout [5][nz][ny][nx].
static long long interior_cells(const Layout& L) { return 5LL * L.nx * L.ny * L.nz; }

// The interior-only staging array of the host-buffer calls (allocated on first
// use).  Those calls write the interior of d_host_state alone: its guard cells
// get defined values once (the steps never read them).
static cudaError_t ensure_interior_staging(gbh_ctx* c) {
  if (c->d_pipe_int) return cudaSuccess;
  cudaError_t e = cudaMalloc(&c->d_pipe_int, sizeof(double) * interior_cells(c->lay) * c->lay.nblocks);
  if (e == cudaSuccess) e = cudaMemset(c->d_host_state, 0, sizeof(double) * state_elems(c->lay));
  return e;
}

// hydro_advance_host (interior = false: U_host in the padded state layout) and
// hydro_advance_host_interior (interior = true: [nblocks][5][nz][ny][nx], staged
// in d_pipe_int and scattered into / gathered from the padded device state).
static int advance_host(gbh_ctx* c, double* U_host, int nsteps, double* dt_hist_host, void* stream,
                        bool interior) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U_host || nsteps < 0) return set_err(c, GBH_ERR_INVAL, "U_host must be non-null and nsteps >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const Layout& L = c->lay;
  const size_t bytes = sizeof(double) * state_elems(L);
  const size_t ibytes = sizeof(double) * interior_cells(L) * L.nblocks;
  cudaError_t e = cudaSuccess;
  if (!c->d_host_state) e = cudaMalloc(&c->d_host_state, bytes);
  if (e == cudaSuccess && interior) e = ensure_interior_staging(c);
  if (e == cudaSuccess && !c->d_host_dt) e = cudaMalloc(&c->d_host_dt, sizeof(double) * c->nproblems);
  if (e == cudaSuccess && nsteps > c->host_hist_cap) {
    cudaFree(c->d_host_hist);
    c->d_host_hist = nullptr;
    e = cudaMalloc(&c->d_host_hist, sizeof(double) * nsteps * c->nproblems);
    if (e == cudaSuccess) c->host_hist_cap = nsteps;
  }
  if (e != cudaSuccess) return set_err(c, GBH_ERR_NOMEM, "device allocation failed: %s", cudaGetErrorString(e));
  if (interior) {
    e = cudaMemcpyAsync(c->d_pipe_int, U_host, ibytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = gbh::launch_interior_copy(c->d_host_state, c->d_pipe_int, L, 0, L.nblocks, true, s);
  } else {
    e = cudaMemcpyAsync(c->d_host_state, U_host, bytes, cudaMemcpyHostToDevice, s);
  }
  if ((rc = cuda_err(c, e, "H2D copy"))) return rc;
  if ((rc = hydro_compute_dt(c, c->d_host_state, c->d_host_dt, stream))) return rc;
  if ((rc = hydro_advance(c, c->d_host_state, nsteps, c->d_host_dt, nsteps ? c->d_host_hist : nullptr, stream)))
    return rc;
  if (interior) {
    e = gbh::launch_interior_copy(c->d_host_state, c->d_pipe_int, L, 0, L.nblocks, false, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(U_host, c->d_pipe_int, ibytes, cudaMemcpyDeviceToHost, s);
  } else {
    e = cudaMemcpyAsync(U_host, c->d_host_state, bytes, cudaMemcpyDeviceToHost, s);
  }
  if ((rc = cuda_err(c, e, "D2H copy"))) return rc;
  if (dt_hist_host && nsteps > 0 &&
      (rc = cuda_err(c, cudaMemcpyAsync(dt_hist_host, c->d_host_hist, sizeof(double) * nsteps * c->nproblems,
                                        cudaMemcpyDeviceToHost, s), "D2H dt copy")))
    return rc;
  return cuda_err(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
}

int hydro_advance_host(gbh_ctx* c, double* U_host, int nsteps, double* dt_hist_host, void* stream) {
  return advance_host(c, U_host, nsteps, dt_hist_host, stream, false);
}

int hydro_advance_host_interior(gbh_ctx* c, double* U_host, int nsteps, double* dt_hist_host, void* stream) {
  return advance_host(c, U_host, nsteps, dt_hist_host, stream, true);
}

// Buffers, chunks, streams and events of the pipelined host-buffer step.
static int pipe_setup(gbh_ctx* c, bool interior) {
  const size_t bytes = sizeof(double) * state_elems(c->lay);
  const int NB = c->lay.nblocks;
  cudaError_t e = cudaSuccess;
  if (!c->d_host_state) e = cudaMalloc(&c->d_host_state, bytes);
  if (e == cudaSuccess && interior) e = ensure_interior_staging(c);
  if (e == cudaSuccess && !c->d_host_dt) e = cudaMalloc(&c->d_host_dt, sizeof(double) * c->nproblems);
  if (e == cudaSuccess && !c->d_pipe_out) {
    e = cudaMalloc(&c->d_pipe_out, bytes);
    if (e == cudaSuccess) e = cudaMemset(c->d_pipe_out, 0, bytes);   // guard cells: defined, unspecified values
  }
  if (e == cudaSuccess && !c->d_pipe_dt) e = cudaMalloc(&c->d_pipe_dt, sizeof(double) * c->nproblems);
  if (e != cudaSuccess) return set_err(c, GBH_ERR_NOMEM, "host-step buffers: %s", cudaGetErrorString(e));
  if (c->pipe_chunks) return GBH_OK;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  // chunks of at most two resident CTAs per SM (one wave of the stage kernel; a
  // chunk a few CTAs larger would leave a nearly empty second wave), at most 64
  // chunks (or the count set)
  const int wave = 2 * (sms > 0 ? sms : 1);
  int K = c->pipe_chunks_wanted > 0 ? c->pipe_chunks_wanted : (NB + wave - 1) / wave;
  K = K < 1 ? 1 : (K > 64 ? 64 : (K > NB ? NB : K));
  c->pipe_first.resize(K + 1);
  for (int k = 0; k <= K; ++k) c->pipe_first[k] = (int)((long long)NB * k / K);
  if (c->pipe_chunks_wanted == 0 && (long long)wave * (K - 1) < NB && (K - 1) * wave > 0) {
    // whole waves, the remainder last
    for (int k = 0; k < K; ++k) c->pipe_first[k] = k * wave;
    c->pipe_first[K] = NB;
  }
  std::vector<int> chunk_of(NB);
  for (int k = 0; k < K; ++k)
    for (int b = c->pipe_first[k]; b < c->pipe_first[k + 1]; ++b) chunk_of[b] = k;
  c->pipe_need.assign(K, 0);
  for (int k = 0; k < K; ++k) {
    int m = k;
    for (int b = c->pipe_first[k]; b < c->pipe_first[k + 1]; ++b)
      for (int f = 0; f < 6; ++f) {
        const int nb = c->h_face[6 * (size_t)b + f];
        if (nb >= 0 && chunk_of[nb] > m) m = chunk_of[nb];
      }
    c->pipe_need[k] = m;
  }
  if (!c->d_ident) {
    std::vector<int> ident(NB);
    for (int b = 0; b < NB; ++b) ident[b] = b;
    e = cudaMalloc(&c->d_ident, sizeof(int) * NB);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_ident, ident.data(), sizeof(int) * NB, cudaMemcpyHostToDevice);
  }
  for (cudaStream_t& st : c->pipe_stream)
    if (e == cudaSuccess && !st) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  c->pipe_ev.assign(3 * (size_t)K, nullptr);
  for (cudaEvent_t& ev : c->pipe_ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  for (cudaEvent_t& ev : c->pipe_mark)
    if (e == cudaSuccess && !ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return set_err(c, GBH_ERR_CUDA, "host-step setup: %s", cudaGetErrorString(e));
  c->pipe_chunks = K;
  return GBH_OK;
}

// hydro_step_host (interior = false: U_host in the padded state layout) and
// hydro_step_host_interior (interior = true: U_host holds the interior cells
// only, [nblocks][5][nz][ny][nx]; each chunk is copied into the staging buffer
// d_pipe_int and scattered into the padded device state by a kernel on the
// copy stream, and gathered back the same way, so only interior bytes cross
// the host link).  The staging region of chunk k is read by its scatter
// before its stage-1 launch and written by its gather after its stage-2
// launch, which waits (through the stage-1 events) for that scatter: one
// buffer serves both directions.
static int host_step(gbh_ctx* c, double* U_host, double* dt_host, void* stream, bool interior) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U_host || !dt_host) return set_err(c, GBH_ERR_INVAL, "U_host and dt_host must be non-null");
  const bool given = dt_host[0] > 0.0;
  for (int p = 0; given && p < c->nproblems; ++p)
    if ((rc = check_dt(c, dt_host[p]))) return rc;
  if ((rc = pipe_setup(c, interior))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout& L = c->lay;
  const size_t bstride = sizeof(double) * (size_t)L.bstride;
  const long long cells = interior_cells(L);
  const size_t dtb = sizeof(double) * c->nproblems;
  double* U = c->d_host_state;
  // blocks [first, first + cnt) of the host state into the padded device state dst
  auto copy_in = [&](double* dst, int first, int cnt, cudaStream_t st) -> cudaError_t {
    if (!interior)
      return cudaMemcpyAsync(dst + (size_t)first * L.bstride, U_host + (size_t)first * L.bstride,
                             bstride * (size_t)cnt, cudaMemcpyHostToDevice, st);
    cudaError_t e = cudaMemcpyAsync(c->d_pipe_int + first * cells, U_host + first * cells,
                                    sizeof(double) * cells * cnt, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = gbh::launch_interior_copy(dst, c->d_pipe_int, L, first, cnt, true, st);
    return e;
  };
  // the same blocks of the padded device state src back into the host state
  auto copy_out = [&](double* src, int first, int cnt, cudaStream_t st) -> cudaError_t {
    if (!interior)
      return cudaMemcpyAsync(U_host + (size_t)first * L.bstride, src + (size_t)first * L.bstride,
                             bstride * (size_t)cnt, cudaMemcpyDeviceToHost, st);
    cudaError_t e = gbh::launch_interior_copy(src, c->d_pipe_int, L, first, cnt, false, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(U_host + first * cells, c->d_pipe_int + first * cells, sizeof(double) * cells * cnt,
                          cudaMemcpyDeviceToHost, st);
    return e;
  };
  cudaError_t e = cudaSuccess;
  if (c->refined || c->telescoping || c->nstages != 2) {
    // the other step forms exchange data across the whole state between their
    // stages: copy in, step, copy out
    e = copy_in(U, 0, L.nblocks, s);
    if (e == cudaSuccess && given) e = cudaMemcpyAsync(c->d_host_dt, dt_host, dtb, cudaMemcpyHostToDevice, s);
    if ((rc = cuda_err(c, e, "H2D copy"))) return rc;
    if (!given && (rc = reduce_dt(c, U, c->d_host_dt, nullptr, s))) return rc;
    PrimChain pc;
    rc = c->refined ? (c->telescoping ? refined_telescoping_step(c, U, c->d_host_dt, 0.0, true, s)
                                      : refined_step(c, U, c->d_host_dt, 0.0, true, s, &pc))
                    : uniform_step(c, U, c->d_host_dt, 0.0, true, s, &pc);
    if (!rc) rc = cuda_err(c, gbh::launch_dt_finalize(c->d_smax, c->cfl, c->d_pipe_dt, nullptr, s, c->nproblems),
                           "dt finalize launch");
    if (rc) return rc;
    e = copy_out(U, 0, L.nblocks, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dt_host, c->d_pipe_dt, dtb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_err(c, e, "host step");
  }
  // Pipelined SSP-RK2 step: chunk k's stage 1 starts once the chunks up to
  // need[k] are on the device (copies run in order), its stage 2 once stage 1
  // is done up to need[k]; stage 2 writes a separate state so that later
  // stage-1 launches still read U^n; chunk k goes back as soon as its stage 2
  // is done.  With dt given, copy-in, both stages and copy-out overlap.
  // The face pre-pass runs per chunk (stage_launch's block range): a chunk's
  // stage reads only slots written by the pre-pass of its own chunk or of an
  // earlier one on the same stream, and the stage-2 pre-pass of chunk k writes
  // only slots of blocks in chunks up to need[k], whose stage-1 launches it
  // waits for; in each stage every slot has exactly one writer.
  const int K = c->pipe_chunks;
  // stage 1 leaves the primitives of U(1) for stage 2 (chunk k's stage 2 reads
  // them only from the chunks whose stage 1 it waits for, like U(1) itself)
  double* W1 = c->prim_carry ? c->d_W[0] : nullptr;
  cudaStream_t sin = c->pipe_stream[0], s1 = c->pipe_stream[1], s2 = c->pipe_stream[2], sout = c->pipe_stream[3];
  cudaEvent_t* ev_in = &c->pipe_ev[0];
  cudaEvent_t* ev_s1 = &c->pipe_ev[K];
  cudaEvent_t* ev_s2 = &c->pipe_ev[2 * (size_t)K];
  e = cudaEventRecord(c->pipe_mark[0], s);
  for (cudaStream_t st : c->pipe_stream)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->pipe_mark[0], 0);
  if (e == cudaSuccess && given) e = cudaMemcpyAsync(c->d_host_dt, dt_host, dtb, cudaMemcpyHostToDevice, sin);
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    e = copy_in(U, c->pipe_first[k], c->pipe_first[k + 1] - c->pipe_first[k], sin);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[k], sin);
  }
  if ((rc = cuda_err(c, e, "H2D copies"))) return rc;
  if (!given) {
    if ((rc = cuda_err(c, cudaStreamWaitEvent(s1, ev_in[K - 1], 0), "event wait"))) return rc;
    if ((rc = reduce_dt(c, U, c->d_host_dt, nullptr, s1))) return rc;
  }
  for (int k = 0; k < K; ++k) {
    const int first = c->pipe_first[k], cnt = c->pipe_first[k + 1] - first;
    if ((rc = cuda_err(c, cudaStreamWaitEvent(s1, ev_in[c->pipe_need[k]], 0), "event wait"))) return rc;
    rc = stage_launch(c, U, nullptr, c->d_scratch, c->d_host_dt, 0.0, 0.0, 1.0, true, false, s1, 0, nullptr,
                      c->d_ident + first, cnt, nullptr, W1, first);
    if (rc) return rc;
    if ((rc = cuda_err(c, cudaEventRecord(ev_s1[k], s1), "event record"))) return rc;
  }
  for (int k = 0; k < K; ++k) {
    const int first = c->pipe_first[k], cnt = c->pipe_first[k + 1] - first;
    if ((rc = cuda_err(c, cudaStreamWaitEvent(s2, ev_s1[c->pipe_need[k]], 0), "event wait"))) return rc;
    rc = stage_launch(c, c->d_scratch, U, c->d_pipe_out, c->d_host_dt, 0.0, 0.5, 0.5, true, true, s2, 0, nullptr,
                      c->d_ident + first, cnt, W1, nullptr, first);
    if (rc) return rc;
    if ((rc = cuda_err(c, cudaEventRecord(ev_s2[k], s2), "event record"))) return rc;
  }
  if ((rc = cuda_err(c, gbh::launch_dt_finalize(c->d_smax, c->cfl, c->d_pipe_dt, nullptr, s2, c->nproblems),
                     "dt finalize launch")))
    return rc;
  e = cudaEventRecord(c->pipe_mark[1], s2);
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    e = cudaStreamWaitEvent(sout, ev_s2[k], 0);
    if (e == cudaSuccess) e = copy_out(c->d_pipe_out, c->pipe_first[k], c->pipe_first[k + 1] - c->pipe_first[k], sout);
  }
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, c->pipe_mark[1], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dt_host, c->d_pipe_dt, dtb, cudaMemcpyDeviceToHost, sout);
  if (e == cudaSuccess) e = cudaEventRecord(c->pipe_mark[2], sout);
  for (cudaStream_t st : {sin, s1}) {
    // join the remaining streams too, so that the caller's stream orders after all of them
    if (e != cudaSuccess) break;
    e = cudaEventRecord(c->pipe_mark[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->pipe_mark[0], 0);
  }
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->pipe_mark[2], 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_err(c, e, "host step");
}

int hydro_step_host(gbh_ctx* c, double* U_host, double* dt_host, void* stream) {
  return host_step(c, U_host, dt_host, stream, false);
}

int hydro_step_host_interior(gbh_ctx* c, double* U_host, double* dt_host, void* stream) {
  return host_step(c, U_host, dt_host, stream, true);
}

int hydro_check_state(gbh_ctx* c, const double* U, long long* nbad_host, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!U || !aligned8(U) || !nbad_host) return set_err(c, GBH_ERR_INVAL, "null or misaligned pointer");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long h = 0;
  if ((rc = cuda_err(c, cudaMemsetAsync(c->d_words + 2, 0, sizeof(unsigned long long), s), "memset"))) return rc;
  if ((rc = cuda_err(c, gbh::launch_check(U, c->lay, c->eos, c->d_words + 2, s), "check kernel launch"))) return rc;
  if ((rc = cuda_err(c, cudaMemcpyAsync(&h, c->d_words + 2, sizeof(h), cudaMemcpyDeviceToHost, s), "D2H copy")))
    return rc;
  if ((rc = cuda_err(c, cudaStreamSynchronize(s), "cudaStreamSynchronize"))) return rc;
  *nbad_host = (long long)h;
  if (h) return set_err(c, GBH_ERR_UNPHYSICAL, "%llu interior cells are unphysical or non-finite", h);
  return GBH_OK;
}

int hydro_floor_hits(gbh_ctx* c, long long* hits_host, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!hits_host) return set_err(c, GBH_ERR_INVAL, "hits_host is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long h = 0;
  if ((rc = cuda_err(c, cudaMemcpyAsync(&h, c->d_words + 1, sizeof(h), cudaMemcpyDeviceToHost, s), "D2H copy")))
    return rc;
  if ((rc = cuda_err(c, cudaMemsetAsync(c->d_words + 1, 0, sizeof(h), s), "memset"))) return rc;
  if ((rc = cuda_err(c, cudaStreamSynchronize(s), "cudaStreamSynchronize"))) return rc;
  *hits_host = (long long)h;
  return GBH_OK;
}

int gbh_set_kernel_timing(gbh_ctx* c, int enable) {
  if (!c) return set_err(nullptr, GBH_ERR_INVAL, "null context");
  c->timing = enable != 0;
  c->ev_used = 0;
  return GBH_OK;
}

int gbh_stage_kernel_time(gbh_ctx* c, double* ms_host, long long* launches_host, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!ms_host || !launches_host) return set_err(c, GBH_ERR_INVAL, "null output pointer");
  if ((rc = cuda_err(c, cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize"))) return rc;
  double total = 0.0;
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    if ((rc = cuda_err(c, cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]), "cudaEventElapsedTime"))) return rc;
    total += ms;
  }
  *ms_host = total;
  *launches_host = (long long)(c->ev_used / 2);
  c->ev_used = 0;
  return GBH_OK;
}

int gbh_fp64_probe(int blocks, int threads, int iters, int lanes, int form, double* out_dev, void* stream) {
  if (blocks < 1 || threads < 1 || threads > 1024 || iters < 1 || lanes < 1 || lanes > 32 || form < 0 ||
      form > 4 || !out_dev)
    return set_err(nullptr, GBH_ERR_INVAL, "invalid probe arguments");
  cudaError_t e = gbh::launch_fp64_probe(blocks, threads, iters, lanes, form, out_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_err(nullptr, GBH_ERR_CUDA, "probe launch: %s", cudaGetErrorString(e));
  return GBH_OK;
}

int gbh_op_count_probe(int fn, int blocks, int threads, int iters, double* io_dev, void* stream) {
  if (fn < 0 || fn >= GBH_OPCOUNT_FNS || blocks < 1 || threads < 1 || threads > 1024 || iters < 1 || !io_dev)
    return set_err(nullptr, GBH_ERR_INVAL, "invalid probe arguments");
  gbh_params p{};
  p.gamma = 1.4;
  p.small_rho = 1e-12;
  p.small_p = 1e-14;
  gbh::Layout L;
  gbh::Eos eos;
  gbh::layout_from_params(&p, &L, &eos);
  cudaError_t e = gbh::launch_op_count(fn, blocks, threads, iters, eos, io_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_err(nullptr, GBH_ERR_CUDA, "probe launch: %s", cudaGetErrorString(e));
  return GBH_OK;
}

int gbh_fastmath_selftest(const double* x_dev, double* out_dev, long long n, void* stream) {
  if (!x_dev || !out_dev || n < 1) return set_err(nullptr, GBH_ERR_INVAL, "invalid self-test arguments");
  cudaError_t e = gbh::launch_fastmath_selftest(x_dev, out_dev, n, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_err(nullptr, GBH_ERR_CUDA, "self-test launch: %s", cudaGetErrorString(e));
  return GBH_OK;
}

int gbh_bits_selftest(const double* x_dev, const double* y_dev, double* out_dev, long long n, void* stream) {
  if (!x_dev || !y_dev || !out_dev || n < 1) return set_err(nullptr, GBH_ERR_INVAL, "invalid self-test arguments");
  cudaError_t e = gbh::launch_bits_selftest(x_dev, y_dev, out_dev, n, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_err(nullptr, GBH_ERR_CUDA, "self-test launch: %s", cudaGetErrorString(e));
  return GBH_OK;
}

int gbh_check_violations(long long* count_host) {
  if (!count_host) return set_err(nullptr, GBH_ERR_INVAL, "count_host is NULL");
#ifdef GBH_CHECK
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_err(nullptr, GBH_ERR_CUDA, "cudaDeviceSynchronize: %s", cudaGetErrorString(e));
  const long long parts[4] = {gbh::check_take_stage(), gbh::check_take_aux(), gbh::check_take_amr(),
                              gbh::check_take_adjoint()};
  long long total = 0;
  for (long long v : parts) {
    if (v < 0) return set_err(nullptr, GBH_ERR_CUDA, "reading the check counters failed");
    total += v;
  }
  *count_host = total;
  return GBH_OK;
#else
  *count_host = 0;
  return set_err(nullptr, GBH_ERR_UNSUPPORTED, "not a checked build (compile with -DGBH_CHECK)");
#endif
}

int gbh_check_selftest(long long* count_host) {
  if (!count_host) return set_err(nullptr, GBH_ERR_INVAL, "count_host is NULL");
#ifdef GBH_CHECK
  const long long n = gbh::check_selftest();
  if (n < 0) return set_err(nullptr, GBH_ERR_CUDA, "check self-test failed");
  *count_host = n;
  return GBH_OK;
#else
  *count_host = 0;
  return set_err(nullptr, GBH_ERR_UNSUPPORTED, "not a checked build (compile with -DGBH_CHECK)");
#endif
}

int gbh_device_sm_count(void) {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GBH_ERR_CUDA;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GBH_ERR_CUDA;
  return n;
}

}  // extern "C"
