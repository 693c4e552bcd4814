// Float-float arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits,
// computed on the float32 pipes.  Built from error-free transformations: Knuth's TwoSum
// (a + b = s + e exactly for any a, b), Dekker's FastTwoSum (the same when |a| >= |b|) and the
// product error fma(a, b, -a b); sums and products follow the usual double-word algorithms
// (accurate sum of both words, renormalised).  The _rn intrinsics keep the compiler from
// contracting or reordering the compensated steps.
#pragma once
#include <cuda_runtime.h>

namespace dh {

struct ff2 {
  float hi, lo;
};

__device__ __forceinline__ ff2 ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff2{s, e};
}

__device__ __forceinline__ ff2 ff_fast_two_sum(float a, float b) {  // requires |a| >= |b|
  const float s = __fadd_rn(a, b);
  return ff2{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff2 ff_add(ff2 x, ff2 y) {
  ff2 s = ff_two_sum(x.hi, y.hi);
  const ff2 t = ff_two_sum(x.lo, y.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = ff_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return ff_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff2 ff_neg(ff2 x) { return ff2{-x.hi, -x.lo}; }

__device__ __forceinline__ ff2 ff_sub(ff2 x, ff2 y) { return ff_add(x, ff_neg(y)); }

// x * y (both float-float)
__device__ __forceinline__ ff2 ff_mul(ff2 x, ff2 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return ff_fast_two_sum(p, e);
}

// x * b for a float b
__device__ __forceinline__ ff2 ff_mul_f(ff2 x, float b) {
  const float p = __fmul_rn(x.hi, b);
  const float e = __fmaf_rn(x.hi, b, -p);
  return ff_fast_two_sum(p, __fmaf_rn(x.lo, b, e));
}

// x + b for a float b
__device__ __forceinline__ ff2 ff_add_f(ff2 x, float b) {
  const ff2 s = ff_two_sum(x.hi, b);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

// Compensated running sum (Neumaier): hi carries the float32 sum, lo gathers the exact rounding
// error of every addition; hi + lo is the sum to about eps32^2 times the sum of |terms| plus
// eps32 times |lo|.  Not renormalised per step.
__device__ __forceinline__ void ff_acc(ff2& acc, float x) {
  const ff2 s = ff_two_sum(acc.hi, x);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, s.lo);
}

__host__ __device__ __forceinline__ ff2 ff_from_double(double v) {
  const float hi = (float)v;
  return ff2{hi, (float)(v - (double)hi)};
}

__device__ __forceinline__ ff2 ff_from(float v) { return ff2{v, 0.0f}; }
__device__ __forceinline__ ff2 ff_from(double v) { return ff_from_double(v); }

__host__ __device__ __forceinline__ double ff_to_double(ff2 x) { return (double)x.hi + (double)x.lo; }

// planar storage: n hi floats, then n lo floats
__device__ __forceinline__ ff2 ff_load(const float* __restrict__ p, long long n, long long i) {
  return ff2{p[i], p[n + i]};
}
__device__ __forceinline__ void ff_store(float* __restrict__ p, long long n, long long i, ff2 v) {
  p[i] = v.hi;
  p[n + i] = v.lo;
}

}  // namespace dh
