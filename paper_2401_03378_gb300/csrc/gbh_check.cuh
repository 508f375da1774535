// gbh_check.cuh -- index checks of the checked build (compiled with -DGBH_CHECK).
//
// GBH_IX(i, n) is the index i of a buffer of n elements.  In the checked
// build an index outside [0, n) is counted in a device word of the
// translation unit and replaced by 0, so the access stays inside the buffer
// and the kernel neither faults nor stops; the host reads and clears the
// count with the function GBH_CHECK_TAKE defines (gbh_check_violations sums
// them over all translation units).  The normal build compiles GBH_IX(i, n)
// to i.
#pragma once

#include <cuda_runtime.h>

namespace gbh {

#ifdef GBH_CHECK
static __device__ unsigned long long g_check_count;   // one per translation unit

__device__ __forceinline__ long long check_index(long long i, long long n) {
  if ((unsigned long long)i < (unsigned long long)n) return i;
  atomicAdd(&g_check_count, 1ULL);
  return 0;
}

#define GBH_IX(i, n) ::gbh::check_index((long long)(i), (long long)(n))
#define GBH_CHECK_TAKE(fn)                                                          \
  long long fn() {                                                                  \
    unsigned long long h = 0, z = 0;                                                \
    if (cudaMemcpyFromSymbol(&h, g_check_count, sizeof(h)) != cudaSuccess) return -1; \
    if (cudaMemcpyToSymbol(g_check_count, &z, sizeof(z)) != cudaSuccess) return -1;   \
    return (long long)h;                                                            \
  }
#else
#define GBH_IX(i, n) (i)
#define GBH_CHECK_TAKE(fn) \
  long long fn() { return 0; }
#endif

}  // namespace gbh
