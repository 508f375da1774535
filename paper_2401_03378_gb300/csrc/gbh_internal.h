// gbh_internal.h -- launch interfaces shared by the translation units of
// libgbhydro.so (not part of the public ABI; see include/gbhydro.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbhydro.h"

namespace gbh {

// Face order used by the compact face-neighbour table: x-, x+, y-, y+, z-, z+.
enum { FACE_XM = 0, FACE_XP, FACE_YM, FACE_YP, FACE_ZM, FACE_ZP };

struct Layout {
  int ndim;
  int nx, ny, nz;        // interior cells per block
  int g, gz;             // guard widths (gz = g in 3-D, 0 in 2-D)
  int nxp, nyp, nzp;     // padded extents
  int nblocks;
  long long vstride;     // nzp*nyp*nxp
  long long bstride;     // 5*vstride
};

// The FP64 constants 1 and -0: a + b = fma(a, one, b), a - b = fma(-b, one, a)
// and a * b = fma(a, b, nz) give exactly the results of the plain operations
// (gbh_fastmath.cuh).
struct Rk {
  double one, nz;
};

struct Eos {
  double gamma, gm1, inv_gm1, g_gm1, small_rho, small_p;  // g_gm1 = gamma / (gamma - 1)
  double hgm1;                                            // (gamma - 1) / 2
  Rk k;                                                   // {1, -0}
  long long opaque;                                       // 0 (see reg_eos)
};

// Arguments of one RK-stage launch: Uout = a*Un + b*(Uin + dt*L(Uin)).
struct StageArgs {
  const double* Uin;
  const double* Un;      // may alias Uout (read and written by the same thread)
  double* Uout;
  const int* face_nbr;   // [nblocks][6]
  const double* inv_dx;  // [nblocks][3]
  const double* dt_dev;  // if non-null, dt = *dt_dev
  double dt;
  double a, b;
  int combine;           // 0: Uout = Uin + dt*L; 1: a*Un + b*(Uin + dt*L); 2: the same with a = b = 1/2
  int gather;            // 1: halo from neighbour interiors; 0: from Uin's own guard cells
  int kchunk, nchunks;   // z planes per work item (3-D), work items per block
  int items_per_cta;     // consecutive work items processed by one CTA (>= 1)
  int ysplit;            // row bands per plane tile, one CTA each (1, or 2 for nx >= 8)
  const int* problem;    // [nblocks] problem of each block (batched ensembles), or null
                         // (then dt_dev and smax_acc have one entry)
  Layout lay;
  Eos eos;
  unsigned long long* smax_acc;     // if non-null: max signal-speed sum of Uout (bit pattern)
  unsigned long long* floor_count;  // floor applications on interior cells
  // primitive variables carried from stage to stage (uniform grids, halo
  // gathered; the layout of the state, interior cells only)
  // the fluxes through the blocks' faces, formed before the stage by the face
  // pre-pass ([nblocks][6][5][NF], NF = N max(N, nz) in 3-D and N in 2-D,
  // tangential index fastest: x faces j + N k, y faces i + N k, z faces
  // i + N j); null: the stage forms them
  const double* bflux;
  const double* Win;                // if non-null: the primitives of Uin (no floor counted on reading them)
  double* Wout;                     // if non-null: the epilogue writes the primitives of Uout (and counts
                                    // their floors)
  // two-level composite grids (all null on a uniform grid)
  const int* block_list;            // blocks to update (leaf blocks); null = all blocks
  int nlist;                        // entries of block_list
  const int* flux_slot;             // [nblocks][6] flux-register slot of a face, or -1
  double* flux_reg;                 // [slots][5][n_t2][N] face fluxes (t1 fastest)
  long long flux_reg_len;           // doubles in flux_reg (checked build)
};

// One coarse face on the boundary of the fine region: the coarse block, its
// face (2*dim + side), its flux-register slot and the slots of the 2^(d-1)
// fine faces covering it (quadrant index q1 + 2*q2 of the tangential halves).
struct RefluxEntry {
  int block, face, coarse_slot;
  int fine_slot[4];
};

struct AmrArgs {
  Layout lay;
  const int* nbr;        // [nblocks][3^ndim]
  const int* parent;     // [nblocks][4]: parent id, offset in parent cells (x, y, z)
  const int* children;   // [nblocks][8]
  const int* covered;    // covered (non-leaf) coarse blocks
  int ncovered;
  const int* fine;       // fine blocks with at least one region on the coarser level
  int nfine;
  const int2* cf_faces;  // (fine block, face) pairs whose face neighbour is on the coarser level
  int ncf_faces;
  const RefluxEntry* reflux;
  const int* reflux_of;  // [nblocks][6]: entry of a coarse block's face in reflux, or -1
  int nreflux;
  double* flux_reg;
  long long flux_reg_len;  // doubles in flux_reg (checked build)
  const double* inv_dx;
  const int* problem;      // [nblocks] problem of each block (batched two-level ensembles), or null
  Eos eos;                 // for the CFL signal speed of corrected cells
  unsigned long long* floor_count;  // the stage kernel's floor counter
};

// W: if non-null, a primitive array of the state's layout; each launch also
// writes the primitives of the cells it writes there.
cudaError_t launch_restrict(double* U, const AmrArgs& a, cudaStream_t s, double* W = nullptr);
cudaError_t launch_prolong(double* U, const AmrArgs& a, int depth, bool faces_only, cudaStream_t s,
                           double* W = nullptr);
// smax_acc: if non-null, the max CFL signal-speed sum of the corrected cells
// (after their correction) goes into smax_acc[problem] (bit pattern), the part
// of the step's CFL reduction that the stage kernel's epilogue leaves out.
cudaError_t launch_reflux(double* U, const AmrArgs& a, const double* dt_dev, double dt, double coef,
                          unsigned long long* smax_acc, cudaStream_t s, double* W = nullptr);

cudaError_t launch_stage(const StageArgs& a, cudaStream_t s);
// The face pre-pass of an interior stage (uniform grid, halo gathered): the
// fluxes through every block face, each face solved once, into out ([nblocks]
// [6][5][NF] as StageArgs::bflux); the stage then reads them through a.bflux.
// Blocks [lo, hi) (hi < 0: all): the faces of a stage over that range of a
// sequence of such ranges in block order.  A block's low face is solved by its
// neighbour, as that block's high face, when the neighbour is below hi (in
// this range or an earlier one), else by the block itself; a high face is
// written into the neighbour's slot when the neighbour is at or above lo.
cudaError_t launch_face_fluxes(const StageArgs& a, double* out, cudaStream_t s, int lo = 0, int hi = -1);

// Telescoping mode (Sec. 4.2): a stage that updates the interior widened by
// `ring` cells (0, 2 or 4) from the block's own guard cells (gather = 0),
// which must hold ring + 2 cells.  No dt epilogue; combine and flux registers
// as in launch_stage.  kchunk/nchunks split the nz + 2*ring planes.
cudaError_t launch_stage_ring(const StageArgs& a, int ring, cudaStream_t s);

// Host helpers shared by the entry points (gbh_abi.cu).
int validate_params(const gbh_params* p, bool allow_coarser);  // GBH_OK or an error code; message in gbh_last_error(NULL)
void layout_from_params(const gbh_params* p, Layout* L, Eos* e);
void face_table_from_params(const gbh_params* p, long long b, int face[6], double inv_dx[3]);
void stage_args_common(StageArgs* A, const Layout& L, const Eos& e);
int set_create_error(int code, const char* msg);
size_t stage_smem_bytes(int nx);
cudaError_t stage_prepare(int nx, int ndim);  // opt-in to the dynamic shared memory size

struct FillArgs {
  double* U;
  const int* nbr;        // [nblocks][3^ndim]
  const int* face_nbr;   // [nblocks][6]
  Layout lay;
};
cudaError_t launch_fill(const FillArgs& a, cudaStream_t s);

struct DtArgs {
  const double* U;
  const double* inv_dx;
  Layout lay;
  Eos eos;
  unsigned long long* smax_acc;
  const int* block_list;   // blocks to include (null = all)
  int nlist;
};
cudaError_t launch_dt_reduce(const DtArgs& a, cudaStream_t s);
cudaError_t launch_dt_finalize(unsigned long long* acc, double cfl, double* dt_out, double* hist,
                               cudaStream_t s, int n = 1);
cudaError_t launch_dt_reduce_blocks(const DtArgs& a, const int* problem, cudaStream_t s);

cudaError_t launch_check(const double* U, Layout lay, Eos eos, unsigned long long* count,
                         cudaStream_t s);

// Interior cells of blocks [b0, b0 + nb) between the padded state layout and
// the interior-only layout [nblocks][5][nz][ny][nx] (the same block origin b0
// in both): to_padded = true scatters `interior` into the interior cells of
// `padded`, false gathers them.  Guard cells are neither read nor written.
cudaError_t launch_interior_copy(double* padded, double* interior, const Layout& L, int b0, int nb,
                                 bool to_padded, cudaStream_t s);

size_t stage_vjp_scratch_doubles(const Layout& L, int ring = 0);   // face-slot buffer of a (box) stage VJP
cudaError_t launch_stage_vjp(const StageArgs& a, const double* M, double scale, const double* A, double cA,
                             const double* B, double cB, double* C, double* Wp, double* out, cudaStream_t s);
// VJP of a stage of ring width `ring` that reads the block's own padded cells
// (a.gather = 0, the telescoping mode): out = J_L(Uin)^T (scale M), with M
// read on the box of that ring, plus nterms linear terms c_t X_t, each on the
// box of ring width rings[t]; every padded cell of out is written.  C: face
// slots (stage_vjp_scratch_doubles(L, ring)); Wp: a state-sized buffer.
cudaError_t launch_stage_vjp_box(const StageArgs& a, int ring, const double* M, double scale, const double* const X[3],
                                 const double c[3], const int rings[3], int nterms, double* C, double* Wp, double* out,
                                 cudaStream_t s);
// Reverse of the full guard fill: out = lam + the adjoints of the guard cells
// the fill copies each interior cell into (interior cells of out only).
cudaError_t launch_fill_vjp(const Layout& L, const int* nbr, const int* face_nbr, const double* lam, double* out,
                            cudaStream_t s);
cudaError_t launch_axpby(const Layout& L, double a, const double* X, double b, const double* Y, double* out,
                         cudaStream_t s);   // out = a X + b Y on interior cells
cudaError_t launch_prim_to_cons(const Layout& L, const Eos& e, const double* W, double* U, const double* lamU,
                                double* lamW, cudaStream_t s);
cudaError_t launch_fastmath_selftest(const double* x, double* out, long long n, cudaStream_t s);
cudaError_t launch_bits_selftest(const double* x, const double* y, double* out, long long n, cudaStream_t s);

// Checked build (-DGBH_CHECK, gbh_check.cuh): per translation unit, read and
// clear the count of out-of-range indices (0 in the normal build, -1 if the
// read failed); the self-test plants one index past a 4-element buffer and
// returns the count it produced (checked build only).
long long check_take_stage();
long long check_take_aux();
long long check_take_amr();
long long check_take_adjoint();
long long check_selftest();
cudaError_t launch_fp64_probe(int blocks, int threads, int iters, int lanes, int form, double* out, cudaStream_t s);
cudaError_t launch_op_count(int fn, int blocks, int threads, int iters, const Eos& e, double* io, cudaStream_t s);

}  // namespace gbh
