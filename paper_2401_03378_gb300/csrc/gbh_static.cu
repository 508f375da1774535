// gbh_static.cu -- hydro_step_static: one SSP-RK2 step that allocates nothing.
//
// Some callers cannot allocate device memory: a host application whose
// memory manager owns the whole device pool, a plug-in loaded into a process
// that forbids cudaMalloc/cudaFree after start-up (allocation there would
// synchronise the device or fragment the pool), or code running inside a
// captured region that must not change the allocation state.  For them this
// entry point keeps everything the step needs beyond the caller's state --
// the intermediate stage U1, the face-neighbour table, the inverse cell
// widths and a counter -- in ONE file-scope __device__ array of fixed size.
// The array exists on every GPU that loads the library, for the life of the
// process.
//
// Limits: the state array (all blocks, guard cells included) must fit the
// U1 region (kU1Bytes = 40 MiB, e.g. a 2-D 128^2 problem of 64 blocks of
// 16^2 + 4 guards, or a 3-D 64^3 problem of 64 blocks of 16^3 + 4 guards)
// and nblocks <= kMaxBlocks = 8192; larger requests are rejected with
// GBH_ERR_INVAL.  Every call shares the array and leaves its contents in it,
// so calls that can overlap on the GPU (different streams without ordering,
// or different host threads) race and must not be issued concurrently.
//
// Set-up: the first call on a device (with that device current) looks up
// the array's device address with cudaGetSymbolAddress and sets the stage
// kernel's shared-memory attribute; that first call should therefore come
// before any stream capture.  Later calls only copy the tables (from host
// memory, staged synchronously by the runtime) and launch the two stage
// kernels.
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
constexpr size_t kWordsOffset = kInvDxOffset + sizeof(double) * 3 * kMaxBlocks;  // unsigned long long [4]
constexpr size_t kStaticBytes = kWordsOffset + 256;

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_base[kMaxDevices] = {nullptr};   // device address of g_static_scratch per device
unsigned g_prepared[kMaxDevices] = {0};           // bit per (nx, ndim) stage kernel attribute set

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

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(GBH_ERR_UNSUPPORTED, "device index %lld out of range", dev);
  cudaStream_t s = (cudaStream_t)stream;

  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_base[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    g_base[dev] = (unsigned char*)ptr;
  }
  const unsigned bit = 1u << ((L.nx == 4 ? 0 : L.nx == 8 ? 1 : 2) * 2 + (L.ndim == 3 ? 1 : 0));
  if (!(g_prepared[dev] & bit)) {
    e = gbh::stage_prepare(L.nx, L.ndim);
    if (e != cudaSuccess) return cuda_fail(e, "stage kernel attribute");
    g_prepared[dev] |= bit;
  }
  unsigned char* base = g_base[dev];
  double* U1 = (double*)base;
  int* face = (int*)(base + kFaceOffset);
  double* inv = (double*)(base + kInvDxOffset);
  unsigned long long* words = (unsigned long long*)(base + kWordsOffset);

  for (long long b = 0; b < params->nblocks; ++b)
    gbh::face_table_from_params(params, b, &g_face_host[6 * b], &g_inv_host[3 * b]);
  e = cudaMemcpyAsync(face, g_face_host, sizeof(int) * 6 * params->nblocks, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(inv, g_inv_host, sizeof(double) * 3 * params->nblocks, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(words, 0, sizeof(unsigned long long) * 4, s);   // floor counter
  if (e != cudaSuccess) return cuda_fail(e, "table upload");

  gbh::StageArgs A{};
  gbh::stage_args_common(&A, L, eos);
  A.face_nbr = face;
  A.inv_dx = inv;
  A.dt = dt;
  A.gather = 1;
  A.floor_count = words + 1;
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
