// kp_dd.cuh -- double-float ("dd") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats (about 48 significant
// bits).  GB300 issues about 2 FP64 operations per clock per SM against 128
// FP32 ones, so the solvers' high-precision true residuals run in this form:
// a dd add or multiply costs 7-11 FP32 instructions, several times less issue
// time than one FP64 instruction.
//
// The building blocks are the classical error-free transformations:
//  * TwoSum (Knuth): s = fl(a + b) and the exact error e, a + b = s + e;
//  * Fast-TwoSum (Dekker), for |a| >= |b|: the same in three operations;
//  * TwoProduct with a fused multiply-add: p = fl(a b), e = fma(a, b, -p).
// dd_add is the "sloppy" sum (hi parts by TwoSum, lo parts added, one
// renormalisation): its error is bounded by a few units of 2^-44 times
// |x| + |y|, i.e. relative to the operands, not to the result -- the bound a
// residual b - A x needs, whose accuracy is judged against ||b||.
//
// FP64 <-> dd conversions: dd_from_double splits the FP64 bit pattern with
// integer operations (no FP64 instruction): hi = x truncated to 24
// significant bits, lo = the remaining 29 bits rounded to 24; |x| < 2^-74 maps
// to (hi, 0) and below 2^-100 to zero, far under any quantity the solvers
// compare.  dd_to_double is exact (hi + lo has at most 48 significant bits).
#pragma once

#include <cuda_runtime.h>

namespace kp {

struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ dd dd_add(dd x, dd y) {
  dd s = dd_two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return dd_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd{-y.hi, -y.lo}); }

__device__ __forceinline__ dd dd_add_f(dd x, float y) {
  dd s = dd_two_sum(x.hi, y);
  s.lo += x.lo;
  return dd_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return dd_fast_two_sum(p, e);
}

__device__ __forceinline__ dd dd_from_double(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int uh = (unsigned int)(u >> 32), ul = (unsigned int)u;
  const unsigned int sign = uh & 0x80000000u;
  const int e = (int)((uh >> 20) & 0x7FFu);          // biased FP64 exponent
  if (e < 1023 - 100) return {0.f, 0.f};
  // top 24 significant bits -> float (exponent rebiased by 1023 - 127 = 896)
  const float hi = __uint_as_float(sign | ((unsigned int)(e - 896) << 23) | ((uh & 0xFFFFFu) << 3) | (ul >> 29));
  if (e < 949) return {hi, 0.f};
  // the 29 bits below: an integer times 2^(e - 1075)
  const float scale = __uint_as_float(sign | ((unsigned int)(e - 948) << 23));
  return {hi, __uint2float_rn(ul & 0x1FFFFFFFu) * scale};
}

__device__ __forceinline__ double dd_to_double(dd x) { return (double)x.hi + (double)x.lo; }

// The FP32 value nearest to x (ties to even) by integer operations on its bit
// pattern -- the top 24 significant bits, rounded on the 29 below -- for x in
// the normal FP32 range; other values go through the conversion instruction.
__device__ __forceinline__ float f32_nearest(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int uh = (unsigned int)(u >> 32), ul = (unsigned int)u;
  const int e = (int)((uh >> 20) & 0x7FFu);
  if (e < 897 || e > 1150) return __double2float_rn(x);
  unsigned int f = (uh & 0x80000000u) | ((unsigned int)(e - 896) << 23) | ((uh & 0xFFFFFu) << 3) | (ul >> 29);
  const unsigned int rem = ul & 0x1FFFFFFFu;
  f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
  return __uint_as_float(f);
}

}  // namespace kp
