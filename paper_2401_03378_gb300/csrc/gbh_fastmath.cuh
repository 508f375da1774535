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
//  * in the stage kernel every FP64 add and multiply is an FMA whose three
//    operands are per-thread registers: a + b = fma(a, 1, b), a - b =
//    fma(-b, 1, a), a * b = fma(a, b, -0), the same results as the plain
//    operations (the product is exact inside the FMA, and x + (-0) = x for
//    every x, zeros included).  Measured on GB300 (gbh_fp64_probe): such an
//    FMA issues at 1.99 lanes per SM clock, while DADD, DMUL and an FMA with
//    a constant-bank, immediate or warp-uniform operand issue at 1.68.  The
//    constants (1, -0, the equation-of-state constants, dt/dx) get there
//    through reg_const: their bit patterns OR-ed with a run-time zero that
//    depends on the thread index, so the compiler can neither fold them into
//    constant operands nor keep them in uniform registers.  With the
//    compile-time constants of plain_rk() the same code compiles to the
//    ordinary DADD / DMUL.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbh_internal.h"

namespace gbh {

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double bitsd(long long b) { return __longlong_as_double(b); }

__device__ __forceinline__ double add(double a, double b, const Rk& k) { return fma(a, k.one, b); }
__device__ __forceinline__ double sub(double a, double b, const Rk& k) { return fma(-b, k.one, a); }
__device__ __forceinline__ double mul(double a, double b, const Rk& k) { return fma(a, b, k.nz); }

__device__ __forceinline__ Rk plain_rk() { return Rk{1.0, -0.0}; }

// A run-time zero that depends on the thread index (p.opaque is 0).
__device__ __forceinline__ long long thread_zero(const Eos& p) { return p.opaque & (long long)threadIdx.x; }

// x in a per-thread register (z = thread_zero(...)).
__device__ __forceinline__ double reg_const(double x, long long z) { return bitsd(dbits(x) | z); }

// The constants of e in per-thread registers.
__device__ __forceinline__ Eos reg_eos(const Eos& p, long long z) {
  Eos e = p;
  e.gamma = reg_const(p.gamma, z);
  e.gm1 = reg_const(p.gm1, z);
  e.g_gm1 = reg_const(p.g_gm1, z);
  e.hgm1 = reg_const(p.hgm1, z);
  e.k.one = reg_const(p.k.one, z);
  e.k.nz = reg_const(p.k.nz, z);
  return e;
}

// Magnitudes and signs of doubles on the integer pipe.  The magnitude key is
// the bit pattern shifted left by one (the sign bit drops out): magnitudes of
// doubles order like these unsigned integers.  Masking the sign bit off with
// an AND would say the same, but the compiler turns that pattern into an FP64
// absolute-value operation (a DADD on the FP64 pipe, the resource this kernel
// is bound by), and it does not do so for the shift.
__device__ __forceinline__ unsigned long long mag_key(double x) { return (unsigned long long)dbits(x) << 1; }
__device__ __forceinline__ unsigned long long sign_bit(double x) {
  return ((unsigned long long)dbits(x) >> 63) << 63;
}

// x / 2 for any finite x on the integer pipe: one off the exponent field when
// |x| >= 2^-1021, else the magnitude bits shifted right (exact except that
// the last bit of a subnormal result is truncated)
__device__ __forceinline__ double half_any(double x) {
  const unsigned long long m2 = mag_key(x);
  return bitsd(m2 >= (4ULL << 52) ? dbits(x) - (1LL << 52) : (long long)(sign_bit(x) | (m2 >> 2)));
}

// x / 4 for any finite x on the integer pipe: two off the exponent field when
// |x| >= 2^-1020, else the magnitude bits shifted right by two (which moves
// the result by less than 2^-1022)
__device__ __forceinline__ double quarter_any(double x) {
  const unsigned long long m2 = mag_key(x);
  return bitsd(m2 >= (6ULL << 52) ? dbits(x) - (2LL << 52) : (long long)(sign_bit(x) | (m2 >> 3)));
}

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
__device__ __forceinline__ double rcp_nr(double x, const Rk& k) {
  const double y = rcp_approx(x);
  const double e = fma(-x, y, k.one);
  const double t = fma(e, e, e);
  return fma(y, t, y);
}

// The series term e/2 + 3e^2/8 of the square-root refinements, as h + (3/2) h^2
// with h = e/2 (exponent decrement on the integer pipe): 2 FP64 operations.
__device__ __forceinline__ double rsqrt_corr(double e, const Rk& k) {
  const double h = half_any(e);
  return fma(add(h, half_any(h), k), h, h);
}

// 1/sqrt(x): 5 FP64 operations after the seed.
__device__ __forceinline__ double rsqrt_nr(double x, const Rk& k) {
  const double y = rsqrt_approx(x);
  const double t = mul(x, y, k);
  const double e = fma(-t, y, k.one);
  return fma(y, rsqrt_corr(e, k), y);
}

// sqrt(x) = x / sqrt(x), refined the same way: 5 FP64 operations after the seed.
__device__ __forceinline__ double sqrt_nr(double x, const Rk& k) {
  const double y = rsqrt_approx(x);
  const double t = mul(x, y, k);
  const double e = fma(-t, y, k.one);
  return fma(t, rsqrt_corr(e, k), t);
}

__device__ __forceinline__ double rcp_nr(double x) { return rcp_nr(x, plain_rk()); }
__device__ __forceinline__ double rsqrt_nr(double x) { return rsqrt_nr(x, plain_rk()); }
__device__ __forceinline__ double sqrt_nr(double x) { return sqrt_nr(x, plain_rk()); }

// ---- integer-domain comparisons -------------------------------------------

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
