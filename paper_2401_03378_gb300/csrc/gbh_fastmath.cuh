// gbh_fastmath.cuh -- FP64 building blocks that keep work off the FP64 pipe.
//
// On GB300 the FP64 pipe retires 2 lanes per SM per clock while the integer
// and FP32 pipes retire 64-128; the stage kernel is bound by FP64 issue.  So:
//  * reciprocal and (reciprocal) square root start from the hardware's
//    documented approximations (PTX rcp.approx.ftz.f64, rsqrt.approx.ftz.f64)
//    and are refined by ONE third-order Newton-Raphson / series step (the
//    classical iteration for 1/x and 1/sqrt(x), see e.g. Muller et al.,
//    Handbook of Floating-Point Arithmetic, ch. 5): with the residual
//    e = 1 - x y0 (resp. 1 - x y0^2),
//        1/x       = y0 (1 + e + e^2 + ...)
//        1/sqrt(x) = y0 (1 + e/2 + 3 e^2/8 + ...),
//    truncated after the quadratic term, so the relative error of the seed
//    is cubed; the results are within a few ulp of the correctly rounded
//    ones (not bit-identical to IEEE division / sqrt).  Valid for positive,
//    normal, finite inputs -- what the scheme feeds them.
//  * comparisons, min / max and sign tests of doubles are done on the bit
//    patterns with 64-bit integer operations (ALU pipe), which give the same
//    decisions as the IEEE comparisons for non-NaN values.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbh {

__device__ __forceinline__ double rcp_approx(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

__device__ __forceinline__ double rsqrt_approx(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

// 1/x: 3 FP64 operations after the seed.
__device__ __forceinline__ double rcp_nr(double x) {
  const double y = rcp_approx(x);
  const double e = fma(-x, y, 1.0);
  const double t = fma(e, e, e);
  return fma(y, t, y);
}

// 1/sqrt(x): 5 FP64 operations after the seed.
__device__ __forceinline__ double rsqrt_nr(double x) {
  const double y = rsqrt_approx(x);
  const double t = x * y;
  const double e = fma(-t, y, 1.0);
  const double q = e * fma(e, 0.375, 0.5);
  return fma(y, q, y);
}

// sqrt(x) = x / sqrt(x), refined the same way: 5 FP64 operations after the seed.
__device__ __forceinline__ double sqrt_nr(double x) {
  const double y = rsqrt_approx(x);
  const double t = x * y;
  const double e = fma(-t, y, 1.0);
  const double q = e * fma(e, 0.375, 0.5);
  return fma(t, q, t);
}

// ---- integer-domain comparisons -------------------------------------------

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double bitsd(long long b) { return __longlong_as_double(b); }

// Key whose signed-integer order is the numeric order of non-NaN doubles
// (negative values have their magnitude bits flipped).
__device__ __forceinline__ long long order_key(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

__device__ __forceinline__ double min_d(double a, double b) { return order_key(b) < order_key(a) ? b : a; }
__device__ __forceinline__ double max_d(double a, double b) { return order_key(a) < order_key(b) ? b : a; }
__device__ __forceinline__ bool less_d(double a, double b) { return order_key(a) < order_key(b) && ((dbits(a) | dbits(b)) << 1) != 0; }

// x >= 0 (true for +0 and -0), x < 0, x > 0.  (-0 is tested by its exact bit
// pattern: a test of the bits below the sign against zero is turned into an
// FP64 compare by the compiler.)
__device__ __forceinline__ bool ge0(double x) {
  const long long b = dbits(x);
  return b >= 0 || b == (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool lt0(double x) { return !ge0(x); }
__device__ __forceinline__ bool gt0(double x) { return dbits(x) > 0; }

__device__ __forceinline__ double sel(bool c, double a, double b) { return c ? a : b; }

}  // namespace gbh
