// Double-float ("ff") arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  Built from
// the error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2,
// 4.2.2): TwoSum, FastTwoSum and the FMA form of TwoProduct.  All operations
// use the _rn intrinsics so that the compiler neither contracts nor
// reassociates them (either would break the error-free steps).
//
// Used by the FP64X output kernel, which reaches FP64-level accuracy on the
// FP32 and integer pipes (GB300 issues FP32 FMA about 70x faster than FP64).
#pragma once
#include <cstdint>

namespace emrifd {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float hi, float lo) { ff r; r.hi = hi; r.lo = lo; return r; }

// |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  return ff_make(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v)));
}

__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff_make(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ ff ff_neg(ff x) { return ff_make(-x.hi, -x.lo); }

__device__ __forceinline__ ff ff_add(ff x, ff y) {
  const ff s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

// running sum acc += y without renormalising: the high words by TwoSum, their error and
// the low words added into acc.lo (renormalise with fast_two_sum before other use);
// |acc.lo| stays a few hundred ulps of acc.hi over the few hundred terms of a tile
__device__ __forceinline__ ff ff_acc(ff acc, ff y) {
  const ff s = two_sum(acc.hi, y.hi);
  return ff_make(s.hi, __fadd_rn(acc.lo, __fadd_rn(s.lo, y.lo)));
}

// ff + float
__device__ __forceinline__ ff ff_add_f(ff x, float y) {
  const ff s = two_sum(x.hi, y);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

// ff * float
__device__ __forceinline__ ff ff_mul_f(ff x, float y) {
  const float p = __fmul_rn(x.hi, y);
  float e = __fmaf_rn(x.hi, y, -p);
  e = __fmaf_rn(x.lo, y, e);
  return fast_two_sum(p, e);
}

// ff from a double (prep time only: uses the FP64 pipe)
__device__ __forceinline__ ff ff_from_double(double x) {
  const float hi = __double2float_rn(x);
  return ff_make(hi, __double2float_rn(x - (double)hi));
}

__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

// frac(x) of a float x in turns, as Q0.64 (exact: a float has 24 significant bits)
__device__ __forceinline__ unsigned long long q64_of_float(float x) {
  const unsigned u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xFF);
  if (e == 0) return 0ull;
  const unsigned long long m = (unsigned long long)((u & 0x7FFFFFu) | 0x800000u);
  const int sh = e - 150 + 64;            // value * 2^64 = m * 2^sh
  unsigned long long r;
  if (sh >= 64) r = 0ull;
  else if (sh >= 0) r = m << sh;
  else if (sh > -64) r = m >> (-sh);
  else r = 0ull;
  return (u >> 31) ? (0ull - r) : r;
}

__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

}  // namespace emrifd
