// gbh_static.cu -- hydro_step_static: one SSP-RK2 step that allocates nothing.
//
// Some callers cannot allocate device memory: a host application whose
// memory manager owns the whole device pool, or a plug-in loaded into a
// process that forbids cudaMalloc/cudaFree after start-up (an allocation
// there would synchronise the device or fragment the pool).  For them this
// entry point keeps everything the step needs beyond the caller's state --
// the intermediate stage U1, the face-neighbour table, the inverse cell
// widths and a discard word for the stage kernel's floor counter -- in ONE
// file-scope __device__ array of fixed size.  The array exists on every GPU
// that loads the library, for the life of the process.
//
// Limits: the state array (all blocks, guard cells included) must fit the
// U1 region (kU1Bytes = 40 MiB, e.g. a 2-D 128^2 problem of 64 blocks of
// 16^2 + 4 guards, or a 3-D 64^3 problem of 64 blocks of 16^3 + 4 guards)
// and nblocks <= kMaxBlocks = 8192; larger requests are rejected with
// GBH_ERR_INVAL.  Every call shares the array and leaves its contents in it,
// so calls that can overlap on the GPU (different streams without ordering,
// or different host threads) race and must not be issued concurrently.
// Nothing in the array has to start at zero: U1 and the tables are written
// in full before they are read, and the floor counter is never read, so
// this entry point reports no floor hits (the floors are still applied).
//
// Device address: in host code g_static_scratch names a host-side stand-in,
// not device memory, so every call looks the array's device address up with
// cudaGetSymbolAddress, with the caller's device current, and sets the stage
// kernel's shared-memory attribute.  Both are host-side calls that allocate
// nothing; doing them on every call (instead of caching them per device
// index) keeps the address right when the caller's context changes, e.g.
// after cudaDeviceReset or under a non-primary context.  The first call on a
// device loads the library's kernels and the array there, so that first call
// should come before any stream capture.  Each call then copies the tables
// (from host memory, staged by the runtime before cudaMemcpyAsync returns)
// and launches the two stage kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/gbhydro.h"
#include "gbh_internal.h"

namespace {

constexpr size_t kU1Bytes = 40ull << 20;                 // intermediate stage U1
constexpr int kMaxBlocks = 8192;
constexpr size_t kFaceOffset = kU1Bytes;                  // int [kMaxBlocks][6]
constexpr size_t kInvDxOffset = kFaceOffset + sizeof(int) * 6 * kMaxBlocks;      // double [kMaxBlocks][3]
constexpr size_t kWordsOffset = kInvDxOffset + sizeof(double) * 3 * kMaxBlocks;  // unsigned long long (discard)
constexpr size_t kStaticBytes = kWordsOffset + 256;

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_mutex;   // guards the host staging buffers below

// host staging of the per-call tables (copied with cudaMemcpyAsync from
// pageable memory, which the runtime stages before returning)
int g_face_host[6 * kMaxBlocks];
double g_inv_host[3 * kMaxBlocks];

int fail(int code, const char* fmt, long long a = 0, long long b = 0) {
  char buf[256];
  snprintf(buf, sizeof(buf), fmt, a, b);
  return gbh::set_create_error(code, buf);
}

int cuda_fail(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return gbh::set_create_error(GBH_ERR_CUDA, buf);
}

}  // namespace

extern "C" int hydro_step_static(const gbh_params* params, double* U, double dt, void* stream) {
  int rc = gbh::validate_params(params, false);
  if (rc) return rc;
  if (!U || ((uintptr_t)U & 7u)) return fail(GBH_ERR_INVAL, "U must be a non-null 8-byte aligned device pointer");
  if (!std::isfinite(dt) || !(dt > 0.0)) return fail(GBH_ERR_INVAL, "dt must be finite and > 0");
  gbh::Layout L;
  gbh::Eos eos;
  gbh::layout_from_params(params, &L, &eos);
  const long long bytes = (long long)sizeof(double) * L.nblocks * L.bstride;
  if (bytes > (long long)kU1Bytes)
    return fail(GBH_ERR_INVAL, "state of %lld bytes exceeds the %lld-byte static scratch of hydro_step_static",
                bytes, (long long)kU1Bytes);
  if (params->nblocks > kMaxBlocks)
    return fail(GBH_ERR_INVAL, "nblocks %lld exceeds the static limit of %lld", params->nblocks, kMaxBlocks);

  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_mutex);
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
  e = gbh::stage_prepare(L.nx, L.ndim);
  if (e != cudaSuccess) return cuda_fail(e, "stage kernel attribute");
  unsigned char* base = (unsigned char*)ptr;
  double* U1 = (double*)base;
  int* face = (int*)(base + kFaceOffset);
  double* inv = (double*)(base + kInvDxOffset);
  unsigned long long* words = (unsigned long long*)(base + kWordsOffset);

  for (long long b = 0; b < params->nblocks; ++b)
    gbh::face_table_from_params(params, b, &g_face_host[6 * b], &g_inv_host[3 * b]);
  e = cudaMemcpyAsync(face, g_face_host, sizeof(int) * 6 * params->nblocks, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(inv, g_inv_host, sizeof(double) * 3 * params->nblocks, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "table upload");

  gbh::StageArgs A{};
  gbh::stage_args_common(&A, L, eos);
  A.face_nbr = face;
  A.inv_dx = inv;
  A.dt = dt;
  A.gather = 1;
  A.floor_count = words;   // discard word: this entry point reports no floor hits
  A.smax_acc = nullptr;
  // stage 1: U1 = U + dt L(U)
  A.Uin = U;
  A.Un = nullptr;
  A.Uout = U1;
  A.a = 0.0;
  A.b = 1.0;
  A.combine = 0;
  if ((e = gbh::launch_stage(A, s)) != cudaSuccess) return cuda_fail(e, "stage 1 launch");
  // stage 2: U = 1/2 U + 1/2 (U1 + dt L(U1))
  A.Uin = U1;
  A.Un = U;
  A.Uout = U;
  A.a = 0.5;
  A.b = 0.5;
  A.combine = 2;   // a = b = 1/2
  if ((e = gbh::launch_stage(A, s)) != cudaSuccess) return cuda_fail(e, "stage 2 launch");
  return GBH_OK;
}
