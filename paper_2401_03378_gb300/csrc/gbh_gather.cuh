// gbh_gather.cuh -- reading a block's cells and its 2-deep face halo.
//
// The guard-cell fill before every stage (Sec. 4.2) is fused into the stage
// kernels: a halo cell across a face is read from the face neighbour's
// interior, from the nearest interior cell at an outflow domain edge, or from
// the block's own (prolonged) guard cells across a coarse-fine boundary.
// Shared by the forward stage kernel and the adjoint kernels so that both
// see exactly the same halo.
#pragma once

#include <cuda_runtime.h>

#include "gbh_check.cuh"
#include "gbh_device.cuh"
#include "gbh_internal.h"

namespace gbh {

// Offset (in doubles, relative to the array base) of cell (i, j, k) of block
// b, given in interior coordinates that may lie outside the block in at most
// one dimension by at most 2 cells.  In gather mode such a cell is read from
// the face neighbour's interior, or, at an outflow edge (GBH_BC_OUTFLOW), from
// the nearest interior cell of b, or, across a coarse-fine boundary
// (GBH_NBR_COARSER), from b's own (prolonged) guard cells; in guard mode
// always from b's own guard cells.
template <int N>
__device__ __forceinline__ long long cell_offset(const StageArgs& a, int b, int i, int j, int k) {
  const Layout& L = a.lay;
  int blk = b;
  if (a.gather) {
    int f = -1;
    if (i < 0) f = FACE_XM;
    else if (i >= N) f = FACE_XP;
    else if (j < 0) f = FACE_YM;
    else if (j >= N) f = FACE_YP;
    else if (k < 0) f = FACE_ZM;
    else if (k >= L.nz) f = FACE_ZP;
    if (f >= 0) {
      const int nb = __ldg(a.face_nbr + 6 * b + f);
      if (nb >= 0) {
        blk = nb;
        switch (f) {
          case FACE_XM: i += N; break;
          case FACE_XP: i -= N; break;
          case FACE_YM: j += N; break;
          case FACE_YP: j -= N; break;
          case FACE_ZM: k += L.nz; break;
          default: k -= L.nz; break;
        }
      } else if (nb == GBH_BC_OUTFLOW) {
        switch (f) {
          case FACE_XM: i = 0; break;
          case FACE_XP: i = N - 1; break;
          case FACE_YM: j = 0; break;
          case FACE_YP: j = N - 1; break;
          case FACE_ZM: k = 0; break;
          default: k = L.nz - 1; break;
        }
      }
      // GBH_NBR_COARSER: the region lies on the coarser level; b's own guard
      // cells hold the prolonged data

    }
  }
  const long long o = (long long)blk * L.bstride + ((long long)(k + L.gz) * L.nyp + (j + L.g)) * L.nxp + (i + L.g);
  return GBH_IX(o, (long long)L.nblocks * L.bstride - 4 * L.vstride);   // o + v*vstride, v < 5, in the state
}

// Primitives of a cell (cell_offset's addressing); e: a.eos, or its
// register copy (reg_eos).
template <int N>
__device__ __forceinline__ int load_prim(const StageArgs& a, const Eos& e, int b, int i, int j, int k, double W[5]) {
  const long long o = cell_offset<N>(a, b, i, j, k);
  double U[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) U[v] = __ldg(a.Uin + o + v * a.lay.vstride);
  return cons_to_prim(U, W, e);
}


}  // namespace gbh
