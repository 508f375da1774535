/*
 * gbhydro.h -- C ABI of libgbhydro.so: the per-block finite-volume update of
 * the compressible Euler equations on a block-structured mesh, on one GB300
 * GPU (sm_103a), in FP64.
 *
 * The paper (CG-Kit, Flash-X Spark variants) describes the work as a
 * block-structured grid of equal blocks, each surrounded by guard cells
 * (Sec. 2.2), advanced by an SSP Runge-Kutta time stepper that fills the
 * guard cells before every stage and then runs, on every block, the
 * intra-stage calculations calcLims -> calcFlux -> updSoln -> calcEos
 * (Sec. 4.2, non-telescoping listing; Alg. "Intra stage calculations for
 * Spark"; Alg. "Block initializations for Spark").  The paper names neither
 * the reconstruction, the Riemann solver, the RK order nor the time-step
 * rule.  This library uses piecewise-linear reconstruction of primitive
 * variables with the monotonized-central limiter, the HLLC flux with
 * Einfeldt / Roe-average wave speeds, two-stage SSP-RK (Shu-Osher), and the
 * CFL rule dt = cfl / max_cells sum_d (|u_d| + c) / dx_d.
 *
 * Conventions shared by every entry point:
 *  - Return value: GBH_OK (0) or a negative GBH_ERR_* code; gbh_last_error()
 *    gives a message.  Nothing throws or aborts across this boundary.
 *  - State arrays are caller-owned DEVICE pointers to FP64 data laid out as
 *        U[nblocks][5][nzb + 2*gz][nyb + 2*ng][nxb + 2*ng]   (x fastest)
 *    with variables (rho, rho*u, rho*v, rho*w, E), gz = ng in 3-D, 0 in 2-D.
 *    Pointers must be 8-byte aligned; distinct arrays must not overlap unless
 *    an entry point says so.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it and the call returns without synchronising, except where
 *    an entry point says it synchronises.
 *  - Interior cells are the result.  After hydro_step / hydro_step_cfl /
 *    hydro_advance the guard cells of U hold unspecified (stale) values;
 *    call hydro_fill_guardcells if they are wanted.
 *  - A context is used from one host thread and one stream at a time.
 */
#ifndef GBHYDRO_H
#define GBHYDRO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBH_OK 0
#define GBH_ERR_INVAL (-1)        /* bad argument: sizes, nguard < 2, dt <= 0 or non-finite, table entry out of range */
#define GBH_ERR_CUDA (-2)         /* a CUDA launch or runtime call failed; the message keeps the CUDA error string */
#define GBH_ERR_UNPHYSICAL (-3)   /* density or pressure at/below its floor, or a non-finite value */
#define GBH_ERR_NOMEM (-4)        /* device or host allocation failed */
#define GBH_ERR_UNSUPPORTED (-5)  /* valid request that this build does not implement (e.g. block shape) */

/* Neighbour-table code for a block face on the domain boundary with a
 * zero-gradient (outflow) condition.  Periodic boundaries are expressed by
 * the caller as the id of the wrapped block. */
#define GBH_BC_OUTFLOW (-1)

/* Neighbour-table code of a fine block whose region at that offset lies on
 * the next coarser level (two-level composite grids, gbh_create_refined):
 * the guard cells there are filled by prolongation from the parent level. */
#define GBH_NBR_COARSER (-2)

typedef struct gbh_ctx gbh_ctx;

typedef struct gbh_params {
  int ndim;               /* 2 or 3 */
  int nxb, nyb, nzb;      /* interior cells per block; this build supports nxb == nyb in {4, 8, 16},
                             nzb == 1 when ndim == 2, nzb >= 2 when ndim == 3 */
  int nguard;             /* guard cells per side, >= 2 and <= min(nxb, nyb[, nzb]) (4 in the standard setups) */
  int nblocks;            /* >= 1 */
  double gamma;           /* ratio of specific heats, > 1 */
  double cfl;             /* Courant number for hydro_compute_dt / hydro_step_cfl, in (0, 1] */
  double small_rho;       /* density floor used when converting conserved -> primitive (e.g. 1e-12), >= 1e-150 */
  double small_p;         /* pressure floor, same use (e.g. 1e-14) */
  const int32_t *nbr;     /* HOST [nblocks][3^ndim]: block id (>= 0) of the neighbour at lattice offset
                             (ox, oy[, oz]) in {-1,0,1}^ndim, entry index (oz+1)*9 + (oy+1)*3 + (ox+1)
                             (2-D: (oy+1)*3 + (ox+1)); the centre entry is the block itself; GBH_BC_OUTFLOW
                             where the offset leaves the domain.  Copied at gbh_create. */
  const double *dx;       /* HOST [nblocks][3]: cell widths of each block (dz ignored in 2-D), > 0.  Copied. */
} gbh_params;

/* Create a context for one block-structured grid of equal blocks with guard
 * cells (Sec. 2.2 of the paper): validates params (GBH_ERR_INVAL,
 * GBH_ERR_UNSUPPORTED), copies the tables to the current CUDA device and
 * allocates the stage scratch (one state-sized buffer) and a few device
 * words.  Synchronous.  *out is set to NULL on failure. */
int gbh_create(const gbh_params *params, gbh_ctx **out);

/* Two-level composite grids (refinement ratio 2, one dt for all levels).
 * Sec. 4.2 of the paper, all-levels variant: every leaf block of every level
 * is advanced in one sweep, then the fluxes through coarse-fine boundaries are
 * communicated and the coarse side corrected.  params describes all blocks of
 * both levels in one state array (same padded block shape); nbr entries of a
 * fine block whose region lies on the coarser level are GBH_NBR_COARSER; dx of
 * a fine block is half its parent's.  The tables (HOST, copied):
 *   parent   [nblocks][4]: parent block id and the offset of this block's
 *            origin in parent cells (0 or n/2 per dimension); (-1,0,0,0) on
 *            level 0;
 *   children [nblocks][8]: the 2^ndim children of a covered (refined) block in
 *            octant order x + 2y + 4z (x fastest), -1 elsewhere.
 * On such a context every stage restricts the covered blocks (mean of their
 * children), prolongs into the fine guard cells facing the coarser level
 * (u_c + sum_d s_d sigma_d / 4, MC slopes of the conserved coarse variables),
 * updates the leaf blocks and replaces the coarse flux through each face on
 * the fine-region boundary by the mean of the fine fluxes through it.
 * hydro_step / hydro_step_cfl / hydro_advance[_host] end with a restriction;
 * hydro_compute_dt uses leaf cells only; hydro_fill_guardcells restricts and
 * then fills every guard cell (prolongation where the region is coarser).
 * hydro_stage / hydro_stage_guarded return GBH_ERR_UNSUPPORTED on such a
 * context.  The refined coarse blocks may form any region (a box, an L, a
 * notch, separate boxes): a coarse cell next to several refined faces of its
 * block takes every face's correction, in the face order x-, x+, y-, y+, z-,
 * z+.  Supported: exactly two levels, cubic (3-D) or square (2-D) blocks of
 * even size, fine blocks not on the domain boundary. */
typedef struct gbh_refinement {
  const int32_t *parent;
  const int32_t *children;
} gbh_refinement;

int gbh_create_refined(const gbh_params *params, const gbh_refinement *refinement, gbh_ctx **out);

/* Batched ensembles: many independent problems in one context and one state
 * array, advanced together (the concurrent-data pattern of Sec. 3.2 of the
 * paper; independent simulations instead of blocks of one domain).
 * problem[b] (HOST, [nblocks], copied) is the problem id (0..nproblems-1) of
 * block b; the neighbour table must not connect blocks of different problems
 * (GBH_ERR_INVAL).  Every problem has its own CFL time step: on such a
 * context hydro_compute_dt, hydro_step_cfl, hydro_advance[_graph] read and
 * write dt_dev[nproblems], hydro_advance's history is [nsteps][nproblems],
 * and hydro_advance_host's is too; hydro_step / hydro_stage apply their one
 * host dt to all problems.  The paper has no batched mode. */
int gbh_create_batched(const gbh_params *params, const int32_t *problem, int nproblems, gbh_ctx **out);

/* Batched two-level ensembles: independent two-level composite grids (each
 * with the tables gbh_create_refined takes, block ids offset so that they
 * index the concatenated arrays) in one context, advanced together with one
 * launch per kernel for all problems and all levels.  problem[b] is as for
 * gbh_create_batched; neither a neighbour entry nor a parent may connect
 * blocks of different problems (GBH_ERR_INVAL).  The time-step rules of
 * gbh_create_batched apply (dt_dev[nproblems]); the flux correction at each
 * problem's fine-coarse faces uses that problem's dt.  Everything else is as
 * for gbh_create_refined.  The paper has no batched mode. */
int gbh_create_refined_batched(const gbh_params *params, const gbh_refinement *refinement, const int32_t *problem,
                               int nproblems, gbh_ctx **out);

/* Work decomposition of the stage kernel (how the concurrent-data pattern of
 * Sec. 3.2 maps blocks onto CTAs; not a choice the paper makes): kchunk = z planes per work item
 * (3-D; 0 or nzb = the whole block) and items_per_cta = consecutive work
 * items one CTA processes (1 = a CTA per item; a grid of about two CTAs per
 * SM makes the kernel persistent).  A third choice is the tile: the plane
 * tile of a work item (the nxb x nyb block plane, widened by the ring in the
 * telescoping mode) can be cut into ysplit row bands, one CTA each, so a CTA
 * has 1/ysplit of the threads and shared memory (twice as many CTAs fit on
 * an SM) at the cost of the halo rows and faces both bands form at the cut;
 * gbh_set_tile_split(ctx, ring, ysplit) sets it per ring width (0: the
 * interior stage; 2, 4: the ring stages of the telescoping mode), ysplit 1,
 * or 2 for blocks of at least 8 cells per side.  Results do not depend on
 * any of these (bitwise).  gbh_autotune times the candidates on U (stage
 * launches into the context's scratch; U is not modified; synchronises the
 * stream; clears the floor counter) and keeps the fastest: kchunk x
 * items_per_cta x ysplit for the interior stage, and, in the telescoping
 * mode, ysplit for each ring stage.  gbh_set_decomposition sets kchunk and
 * items_per_cta directly.  The chosen kchunk and items_per_cta are written to
 * *kchunk_out / *items_out if not NULL; gbh_get_tile_split reads a split.
 * GBH_ERR_INVAL: a ring other than 0, 2, 4 or an unsupported ysplit. */
int gbh_autotune(gbh_ctx *ctx, const double *U, int *kchunk_out, int *items_out, void *stream);
int gbh_set_decomposition(gbh_ctx *ctx, int kchunk, int items_per_cta);
int gbh_set_tile_split(gbh_ctx *ctx, int ring, int ysplit);
int gbh_get_tile_split(gbh_ctx *ctx, int ring, int *ysplit);

/* Time-stepping mode (Sec. 4.2, the telescoping variant of the SSP-RK
 * stepper).  enable = 0 (the default): non-telescoping, the guard cells are
 * refilled before every stage (fused into the stage kernel as a gather from
 * the neighbours).  enable != 0: telescoping, one guard fill per step (all 4
 * guard layers, edges and corners included, written into U's guard cells),
 * then the first stage updates the interior widened by 2 cells on every side
 * from U's own guard cells and the second stage reads that ring of the
 * intermediate state instead of exchanging halos.  Where a neighbour block
 * supplies the halo the result is the non-telescoping one; at an outflow
 * domain edge the first stage evolves the zero-gradient copies, so the 2
 * cells next to that edge differ.
 * On a two-level context (gbh_create_refined) the mode is the paper's
 * level-by-level telescoping variant (Fig. "Level-by-levels, Telescoping"):
 * one fill for both levels (restriction, same-level copies, prolongation of
 * all guard layers from the coarser level), both stages of every leaf block
 * from its own guard data with the fluxes through coarse-fine faces of each
 * stage kept, then the coarse side of the fine region corrected once with
 * weight 1/2 per stage, and the restriction.
 * Applies to hydro_step, hydro_step_cfl, hydro_advance(_graph/_host) and, on
 * uniform contexts, hydro_step_adjoint (the adjoint of the telescoping step);
 * not to single stages, hydro_stage_vjp, hydro_step_static or
 * hydro_step_adjoint_stored.
 * Errors: GBH_ERR_INVAL if nguard < 4; GBH_ERR_NOMEM if the second set of
 * flux registers (two-level contexts) cannot be allocated.  Drops a captured
 * graph. */
int gbh_set_telescoping(gbh_ctx *ctx, int enable);

/* Number of SSP-RK stages (Sec. 4.2 names SSP-RK, multistage, without an
 * order): 2 (the default; Shu-Osher SSP-RK2) or 3 (Shu-Osher SSP-RK3:
 * U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1)); U^{n+1} = 1/3 U +
 * 2/3 (U2 + dt L(U2))).  Applies to every step path of the context:
 * non-telescoping (a halo gather per stage), telescoping (ring widths 4, 2, 0;
 * needs nguard >= 6), two-level all-levels (correction every stage with its
 * b) and level-by-level telescoping (correction weights 1/6, 1/6, 2/3).
 * Allocates a second scratch state (and flux registers) on first use.
 * Errors: GBH_ERR_INVAL for other values or too few guard cells for the
 * telescoping mode; GBH_ERR_NOMEM.  hydro_step_adjoint follows the stage
 * count; hydro_step_adjoint_stored is of the two-stage non-telescoping step
 * only.  Drops a
 * captured graph. */
int gbh_set_rk_stages(gbh_ctx *ctx, int nstages);

/* Primitive variables carried from stage to stage (Alg. "Intra stage
 * calculations for Spark": calcEos runs once per stage, after updSoln, and
 * its primitives are what the next stage's calcLims reads).  With the carry
 * on, every stage of a call except its last leaves the primitive variables
 * (rho, u, v, w, p, floors applied) of its output in one of two
 * context-owned arrays of the state's size, and the next stage reads them
 * instead of converting its input again; the first stage of a call converts
 * the caller's state.  Within one call of hydro_step / hydro_step_cfl the
 * first stage hands its primitives to the second; hydro_advance,
 * hydro_advance_graph and hydro_advance_host carry them across their steps,
 * and hydro_step_host from stage 1 to stage 2.  Results, dt and floor
 * counts are bit for bit those of the carry off (a floor is counted by the
 * stage whose output it is found in, once per interior cell and stage, as
 * when the next stage converted).  On two-level contexts (all-levels steps)
 * the restriction, the prolongation and the flux correction also write the
 * primitives of the cells they write (the correction counts the floors of the
 * corrected value in place of the uncorrected one).  Applies to uniform,
 * batched and two-level contexts in the non-telescoping mode; telescoping
 * steps, single stages, the adjoint and hydro_step_static always convert.
 * Every gbh_create* allocates the arrays (2 x gbh_state_bytes) and switches
 * the carry on; if that allocation fails the carry stays off and the context
 * is created all the same.  gbh_set_prim_carry(ctx, 0) frees the arrays
 * (synchronises the device); enable != 0 allocates them again
 * (GBH_ERR_NOMEM if it cannot).  gbh_get_prim_carry writes 1 to *enabled
 * when the carry is on.  Drops a captured graph. */
int gbh_set_prim_carry(gbh_ctx *ctx, int enable);
int gbh_get_prim_carry(gbh_ctx *ctx, int *enabled);

/* Face pre-pass (not a choice the paper makes; how the blocks of the
 * concurrent-data pattern, Sec. 3.2, share their boundary work).  Each
 * interior stage that gathers its halo (ring 0, one row band, whole blocks;
 * uniform, batched and two-level contexts, all-levels steps) first runs a kernel
 * that solves the flux through every block face once: the block on the high
 * side of a face solves it for both blocks, and a block solves its low face
 * itself only where it has no face neighbour (an outflow edge, a face onto
 * the coarser level).  The stage kernel then reads those fluxes
 * instead of solving each shared face in both blocks.  Results, dt and
 * floor counts are bit for bit those without it (the same face states and
 * HLLC arithmetic).  Every gbh_create* allocates its buffer ([nblocks][6]
 * [5][nxb max(nxb, nzb)] doubles) and switches it on for 3-D contexts (off
 * if that allocation fails); 2-D contexts start with it off (enable
 * allocates [nblocks][6][5][nxb] doubles).  enable = 0 switches it off (the
 * buffer stays).  GBH_ERR_NOMEM if enable != 0 and the buffer cannot be
 * allocated.  Drops a captured graph. */
int gbh_set_face_prepass(gbh_ctx *ctx, int enable);
int gbh_get_face_prepass(gbh_ctx *ctx, int *enabled);

/* (No counterpart in the paper: launch batching.)
 * nsteps calls of hydro_step_cfl captured once into a CUDA graph (on a
 * private stream; re-captured when U, dt_dev or nsteps change, or the
 * decomposition changes) and launched on `stream` as one graph.  Kernel
 * timing must be off.  The first call captures: make it outside any capture
 * of the caller's own. */
int hydro_advance_graph(gbh_ctx *ctx, double *U, int nsteps, double *dt_dev, void *stream);

/* Adjoint (vector-Jacobian products) for gradients of a loss of the final
 * state with respect to the initial fields.  Conventions: dt is held fixed
 * (a constant of each step), and every branch keeps the decision the forward
 * evaluation took (floors, MC limiter case, HLLC side and fan, the min / max
 * of the wave-speed bounds).  Uniform single-problem contexts only
 * (GBH_ERR_UNSUPPORTED otherwise).  All arrays are DEVICE state arrays; only
 * interior cells are read or written.  The paper has no adjoint.
 *
 * hydro_stage_vjp: out = cA*A + cB*B + J_L(U)^T (scale*M), L the stage's
 *   flux-difference operator evaluated at U (guard data gathered from the
 *   neighbours as in hydro_stage).  A and B may be NULL; out may equal A or B
 *   but must not overlap U or M.
 * hydro_step_adjoint: given lam_next = dJ/dU^{n+1} of one hydro_step(Un, dt)
 *   with the context's stage count (2 or 3) and mode, writes lam_prev =
 *   dJ/dU^n: the Shu-Osher recursion run backwards,
 *   lam_{s-1} = b_s lam_s + J_L(U(s-1))^T (b_s dt lam_s), with U^n also
 *   collecting a_s lam_s from every stage (recomputes the intermediate
 *   stages; lam_prev may equal lam_next, must not overlap Un).  In the
 *   telescoping mode (Sec. 4.2) the recursion runs over the ring stages'
 *   boxes on the filled state, and ends with the reverse of the one fill of
 *   all guard layers: every guard cell's adjoint goes to the interior cell it
 *   was copied from (a neighbour's, or the block's own at an outflow edge).
 * hydro_prim_to_cons: U = conserved(W) on interior cells, W = (rho, u, v, w, p)
 *   in the state layout; hydro_prim_to_cons_vjp: lamW = (dU/dW)^T lamU. */
int hydro_stage_vjp(gbh_ctx *ctx, const double *U, const double *M, double scale, const double *A, double cA,
                    const double *B, double cB, double *out, void *stream);
int hydro_step_adjoint(gbh_ctx *ctx, const double *Un, double dt, const double *lam_next, double *lam_prev,
                       void *stream);

/* The same with the first-stage state U1 = Un + dt L(Un) of that step given
 * (DEVICE, e.g. kept while recomputing a checkpointed segment with
 * hydro_stage), which saves the stage the call would otherwise recompute.
 * U1 is read only; lam_prev must not overlap Un or U1.  Two-stage contexts
 * only, non-telescoping (GBH_ERR_UNSUPPORTED otherwise). */
int hydro_step_adjoint_stored(gbh_ctx *ctx, const double *Un, const double *U1, double dt, const double *lam_next,
                              double *lam_prev, void *stream);
/* Conserved variables from primitive ones, the inverse of the calcEos
 * conversion (Alg. "Intra stage calculations for Spark"): U = (rho, rho u,
 * rho v, rho w, p/(gamma-1) + rho |u|^2 / 2) from W = (rho, u, v, w, p), on
 * interior cells of DEVICE state arrays; and its VJP, lamW = (dU/dW)^T lamU
 * on interior cells (overwritten; the paper has no adjoint).  GBH_ERR_INVAL
 * for null or misaligned pointers. */
int hydro_prim_to_cons(gbh_ctx *ctx, const double *W, double *U, void *stream);
int hydro_prim_to_cons_vjp(gbh_ctx *ctx, const double *W, const double *lamU, double *lamW, void *stream);

/* Release everything gbh_create allocated.  Synchronises the device.  NULL is a no-op. */
int gbh_destroy(gbh_ctx *ctx);

/* Message of the last error on ctx (or of the last failed gbh_create when ctx is NULL). */
const char *gbh_last_error(const gbh_ctx *ctx);

/* Bytes of one state array U for this context's layout. */
long long gbh_state_bytes(const gbh_ctx *ctx);

/* fill_guardcells (Sec. 4.2, called before every RK stage in the
 * non-telescoping variant): every guard cell of every block is set, in place,
 * from the neighbour block's interior; at an outflow domain edge the nearest
 * interior value is copied, dimension by dimension in the order x, y, z (so
 * edge and corner guards are defined too).  Reads interior cells only. */
int hydro_fill_guardcells(gbh_ctx *ctx, double *U, void *stream);

/* CFL time step of the state U (interior cells of all blocks; leaf cells on
 * two-level grids): *dt_dev = cfl / max sum_d (|u_d| + c) / dx_d, written to
 * the DEVICE double dt_dev (one per problem on batched contexts).  The paper
 * gives no time-step rule; this unsplit-sum CFL form is the library's reading.
 * No synchronisation. */
int hydro_compute_dt(gbh_ctx *ctx, const double *U, double *dt_dev, void *stream);

/* One RK stage in Shu-Osher form on the interior of every block (a stage of
 * the paper's multistage SSP-RK stepper, Sec. 4.2):
 *     Uout = a * Un + b * (Uin + dt * L(Uin)),
 * L = the flux-difference operator of the intra-stage calculations (calcLims,
 * calcFlux, updSoln; Alg. "Intra stage calculations for Spark").  With a == 0 and b == 1 this is Uin + dt L(Uin) and Un
 * is not read (may be NULL).  Guard data of Uin are gathered from the
 * neighbour blocks' interiors through the neighbour table (Uin's own guard
 * cells are not read).  Uout may equal Un but must not overlap Uin.
 * dt must be finite and > 0. */
int hydro_stage(gbh_ctx *ctx, const double *Uin, const double *Un, double *Uout, double dt, double a,
                double b, void *stream);

/* The same stage, but reading the guard data from Uin's own guard cells
 * (for callers that filled them, e.g. with hydro_fill_guardcells). */
int hydro_stage_guarded(gbh_ctx *ctx, const double *Uin, const double *Un, double *Uout, double dt,
                        double a, double b, void *stream);

/* One full SSP-RK2 step in place with a host-given dt (the paper's
 * non-telescoping stepper, Sec. 4.2, with two Shu-Osher stages):
 *     U1 = U + dt L(U);   U <- 1/2 U + 1/2 (U1 + dt L(U1)).
 * U1 lives in the context's scratch buffer.  GBH_ERR_INVAL for dt <= 0 or
 * non-finite, or a null / misaligned U. */
int hydro_step(gbh_ctx *ctx, double *U, double dt, void *stream);

/* One SSP-RK2 step in place, as hydro_step, for callers that cannot
 * allocate device memory (a host whose memory manager owns the device pool,
 * a plug-in in a process that forbids cudaMalloc/cudaFree after start-up):
 * no context is created and nothing is allocated.  The intermediate stage,
 * the face-neighbour table and the inverse cell widths live in one fixed
 * file-scope device array of 40 MiB + 385 KiB that every GPU loading the
 * library holds until the process exits.  params is read as in gbh_create
 * (HOST tables); U is the caller's DEVICE state.  Rejected with
 * GBH_ERR_INVAL: a state larger than 40 MiB (41,943,040 bytes) or more than
 * 8192 blocks.  Every call looks up the array's device address for the
 * current device; the first call on a device also loads the library's
 * kernels there, so it should come before any stream capture.  All calls
 * share the array and leave their data in it: calls that may overlap on the
 * GPU race and must be serialised by the caller.  The floors are applied as
 * in hydro_step but not counted (no floor hits are reported).  The paper has
 * no counterpart of this entry point.  Errors are reported through
 * gbh_last_error(NULL). */
int hydro_step_static(const gbh_params *params, double *U, double dt, void *stream);

/* One SSP-RK2 step in place whose dt is read from the DEVICE double *dt_dev
 * (which must hold the CFL time step of U, e.g. from hydro_compute_dt or the
 * previous call); on return the stream holds work that overwrites *dt_dev
 * with the CFL time step of the new state (computed in the second stage's
 * epilogue).  No host synchronisation: the loop can be captured or pipelined. */
int hydro_step_cfl(gbh_ctx *ctx, double *U, double *dt_dev, void *stream);

/* nsteps calls of hydro_step_cfl.  If dt_hist_dev is not NULL it receives the
 * dt used by each step (DEVICE array of nsteps doubles). */
int hydro_advance(gbh_ctx *ctx, double *U, int nsteps, double *dt_dev, double *dt_hist_dev, void *stream);

/* Host-buffer variant for callers whose state lives in host memory (the
 * paper's heterogeneous case, where host-device movement adds to the cost of
 * every exchange, Sec. 4.2; the entry point itself has no counterpart there):
 * copies U_host (pinned or pageable, one state array) to a context-owned
 * device buffer (allocated on first use), computes dt, advances nsteps, and
 * copies the interior-updated state back into U_host and the dt of each step
 * into dt_hist_host (nsteps doubles, may be NULL).  Synchronises the stream. */
int hydro_advance_host(gbh_ctx *ctx, double *U_host, int nsteps, double *dt_hist_host, void *stream);

/* hydro_advance_host for a host state of the interior cells only, laid out
 * as in hydro_step_host_interior (U_host[nblocks][5][nzb][nyb][nxb], HOST,
 * in and out): copied into the context-owned interior-only staging array,
 * scattered into the padded device state, advanced, gathered and copied
 * back.  Arguments, errors and synchronisation otherwise as
 * hydro_advance_host; the interior results are the same bits. */
int hydro_advance_host_interior(gbh_ctx *ctx, double *U_host, int nsteps, double *dt_hist_host, void *stream);

/* One step of a state in HOST memory with the copies overlapped with the
 * stages (one hydro_step_cfl in effect).  dt_host (HOST, [nproblems]) is in
 * and out: if dt_host[0] > 0 it is the step's time step (every entry must be
 * finite and > 0), typically the value the previous call returned;
 * otherwise the CFL time step of U_host is computed first.  On return U_host
 * holds the new state (interior; guard cells are overwritten with
 * unspecified values) and dt_host the CFL time step of the new state.
 * The state is split into chunks of consecutive blocks: a chunk's first
 * stage starts as soon as the chunks its face neighbours live in are on the
 * device, its second stage writes a separate device state, and the chunk is
 * copied back as soon as that is done, so the copies in both directions
 * overlap the stages (U_host should be pinned for that).  Two-level
 * contexts, the telescoping mode and three stages run the same step
 * unpipelined.  Uses context-owned device buffers (three states, allocated
 * on first use) and streams; synchronises the stream.  The results equal
 * hydro_step_cfl's bit for bit. */
int hydro_step_host(gbh_ctx *ctx, double *U_host, double *dt_host, void *stream);

/* hydro_step_host for a host state that holds the interior cells only:
 * U_host (HOST, pinned or pageable) is laid out as
 *     U_host[nblocks][5][nzb][nyb][nxb]   (x fastest)
 * with the variables of the state layout, and is replaced by the new state in
 * the same layout.  Guard cells are not inputs of a step (every stage fills
 * them from neighbour interiors or the boundary conditions), so only interior
 * bytes cross the host link: at 16^3 blocks with 4 guard cells 4096 of 13824
 * cells per variable.  Each chunk of blocks is copied into a context-owned
 * device staging buffer (one interior-sized array, allocated on first use)
 * and scattered into the padded device state by a kernel on the copy stream;
 * the new state is gathered and copied back the same way.  dt_host, the
 * chunks, the step forms that run unpipelined, errors and synchronisation are
 * those of hydro_step_host, and the interior results equal hydro_step_cfl's
 * bit for bit. */
int hydro_step_host_interior(gbh_ctx *ctx, double *U_host, double *dt_host, void *stream);

/* Number of block chunks hydro_step_host pipelines (1..64); 0 (the default)
 * picks the fewest chunks of at most two resident CTAs per SM, one wave of the
 * stage kernel each.  GBH_ERR_INVAL outside [0, 64]. */
int gbh_set_host_pipeline(gbh_ctx *ctx, int chunks);

/* Failure check for the floors of the calcEos conversion (no counterpart in
 * the paper).  Scan the interior of U: counts cells whose density <= small_rho, pressure
 * <= small_p, or any variable is non-finite.  Synchronises the stream, writes
 * the count to *nbad_host and returns GBH_ERR_UNPHYSICAL if it is non-zero. */
int hydro_check_state(gbh_ctx *ctx, const double *U, long long *nbad_host, void *stream);

/* Number of floor applications (small_rho / small_p) on interior cells during
 * stages since the last call; resets the counter.  Synchronises the stream. */
int hydro_floor_hits(gbh_ctx *ctx, long long *hits_host, void *stream);

/* Kernel timing for measurement: when enabled, CUDA events are recorded on
 * the stream around every stage-kernel launch.  gbh_stage_kernel_time
 * synchronises the stream, returns the summed stage-kernel time (ms) and
 * launch count since the previous call, and clears them. */
int gbh_set_kernel_timing(gbh_ctx *ctx, int enable);
int gbh_stage_kernel_time(gbh_ctx *ctx, double *ms_host, long long *launches_host, void *stream);

/* FP64 throughput probe (not part of the method): launches blocks x threads
 * threads; in every warp the first `lanes` (1..32) lanes run 8 independent
 * chains of iters FP64 operations, the others none.  form selects the
 * operation: 0 = fused multiply-add with two compile-time constant operands,
 * 1 = fused multiply-add with all three operands in per-thread registers,
 * 2 = add, 3 = multiply (operands in per-thread registers), 4 = fused
 * multiply-add with two warp-uniform register operands.  Writes one double per thread to
 * out_dev (blocks*threads doubles).  FP64 operations executed =
 * 8 * iters * blocks * (threads/32) * lanes for threads a multiple of 32
 * (x2 flops for forms 0, 1 and 4).  GBH_ERR_INVAL for out-of-range arguments. */
int gbh_fp64_probe(int blocks, int threads, int iters, int lanes, int form, double *out_dev, void *stream);

/* FP64 instruction-count probe of the stage kernel's arithmetic building
 * blocks (not part of the method; for ncu's per-kernel instruction counters).
 * fn: 0 = conserved -> primitive conversion of one cell, 1 = one x/y slope
 * work item (three cells' MC slopes and face states) of one variable, 2 = one
 * HLLC face, 3 = the 3-D flux-difference update of one variable, 4 = the
 * second SSP-RK stage's combine of one variable, 5 = the CFL epilogue of one
 * cell (conversion and 3-D signal speed), 6 = the z march's next slope and
 * face states of one variable, 7 = the two face states of a block-boundary
 * face, one variable.  Each of blocks*threads threads makes iters dependent
 * calls on its 10 DEVICE doubles io_dev[10 t .. 10 t + 9] (a conserved state,
 * or two primitive states for fn 2, and any finite values for the rest;
 * overwritten with the chain's last inputs, which differ from the first ones
 * in the last mantissa bit at most), chained through integer operations only, so
 * the FP64 instructions of a launch divided by blocks*threads*iters are those
 * of one call.  GBH_ERR_INVAL for out-of-range arguments. */
#define GBH_OPCOUNT_FNS 8
int gbh_op_count_probe(int fn, int blocks, int threads, int iters, double *io_dev, void *stream);

/* Self-test of the FP64 reciprocal / reciprocal-square-root / square-root
 * building blocks the kernels use (hardware seed + one refinement step):
 * for n positive, normal, finite DEVICE doubles x_dev writes 6*n DEVICE
 * doubles out_dev = [refined 1/x | IEEE 1/x | refined 1/sqrt(x) |
 * IEEE 1/sqrt(x) | refined sqrt(x) | IEEE sqrt(x)].  Not part of the method. */
int gbh_fastmath_selftest(const double *x_dev, double *out_dev, long long n, void *stream);

/* Self-test of the integer-pipe helpers of the stage kernel (not part of the
 * method): for n finite DEVICE doubles x_dev, y_dev writes 6*n DEVICE doubles
 * out_dev = [x/2 | x/4 (both from the exponent field, exact for normal
 * results) | half the MC-limited slope from the differences x, y (dm, dp) |
 * 1 if x >= 0 (also -0) else 0 | min(x, y) | max(x, y) (bit-pattern order)].
 * GBH_ERR_INVAL for null pointers or n < 1. */
int gbh_bits_selftest(const double *x_dev, const double *y_dev, double *out_dev, long long n, void *stream);

/* Number of SMs of the current device (for sizing probes), or a negative error. */
int gbh_device_sm_count(void);

/* Checked build (libgbhydro_check.so, compiled with -DGBH_CHECK): every
 * computed global and shared-memory index of the kernels is compared with
 * its buffer's length; an index outside the buffer is counted and the
 * access redirected to the buffer's first element, so no access leaves its
 * buffer (the stand-in for a memory checker, which this build does not
 * use).  gbh_check_violations synchronises the device, writes the number of
 * such indices since the previous call to *count_host and clears it.
 * gbh_check_selftest runs one kernel that computes an index one past a
 * 4-element buffer and writes the count it produced (1 when the checks work).
 * In the normal build both return GBH_ERR_UNSUPPORTED with *count_host = 0.
 * The paper has no counterpart. */
int gbh_check_violations(long long *count_host);
int gbh_check_selftest(long long *count_host);

#ifdef __cplusplus
}
#endif

#endif /* GBHYDRO_H */
