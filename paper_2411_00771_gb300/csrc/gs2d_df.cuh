// Double-float arithmetic on the FP32 pipes (device only).
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The preprocess carries the geometry that decides
// where a surfel lands on screen in this form instead of FP64, whose pipe runs
// at a small fraction of the FP32 rate on this GPU.
//
// Methods (all published):
//   - TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly;
//   - Fast2Sum (Dekker 1971): the same when |a| >= |b|, used to renormalise;
//   - exact product with one fused multiply-add: a b = p + fma(a, b, -p);
//   - sums and products of two double-floats as in Dekker's 1971 paper
//     ("A floating-point technique for extending the available precision"):
//     the high parts combined exactly, the low-order terms added once;
//   - reciprocal, square root and reciprocal square root: one Newton step in
//     double-float from the FP32 result, which doubles the number of correct
//     bits (quadratic convergence).
// Every operation is written with explicit round-to-nearest intrinsics so
// that the compiler cannot contract or reorder the error terms away.
#pragma once

#include <cuda_runtime.h>

namespace gs2d {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return {a, 0.f}; }
__device__ __forceinline__ df df_make(float hi, float lo) { return {hi, lo}; }
__device__ __forceinline__ float df_float(df a) { return __fadd_rn(a.hi, a.lo); }

// Knuth's TwoSum
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// Dekker's Fast2Sum (|a| >= |b|)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// exact product
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df operator+(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  df r = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(r.hi, __fadd_rn(r.lo, t.lo));
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator+(df a, float b) {
  const df s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ df operator-(df a, float b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ df operator*(df a, float b) {
  const df p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ df operator*(float a, df b) { return b * a; }

// Sign tests and ordering (hi carries the sign unless hi = 0).
__device__ __forceinline__ bool df_pos(df a) { return a.hi > 0.f || (a.hi == 0.f && a.lo > 0.f); }
__device__ __forceinline__ bool df_nonzero(df a) { return a.hi != 0.f || a.lo != 0.f; }
__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ df df_min(df a, df b) { return df_lt(b, a) ? b : a; }
__device__ __forceinline__ df df_max(df a, df b) { return df_lt(a, b) ? b : a; }

// 1 / b: x = 1/b.hi in FP32, then one Newton step x + x (1 - b x).
__device__ __forceinline__ df df_rcp(df b) {
  const float x = __frcp_rn(b.hi);
  const df r = df_make(1.f) - b * x;  // residual, about 2^-24
  return df_make(x) + r * x;
}
__device__ __forceinline__ df operator/(df a, df b) { return a * df_rcp(b); }

// 1 / sqrt(a) for a > 0: y = rsqrt(a.hi), then y + y (1 - a y^2) / 2.
__device__ __forceinline__ df df_rsqrt(df a) {
  const float y = rsqrtf(a.hi);
  const df r = df_make(1.f) - a * two_prod(y, y);
  return df_make(y) + r * (0.5f * y);
}
// sqrt(a) for a >= 0: s = a * rsqrt(a), then s + (a - s^2) / (2 s).
__device__ __forceinline__ df df_sqrt(df a) {
  if (!(a.hi > 0.f)) return df_make(0.f);
  const float s = __fsqrt_rn(a.hi);
  const df r = a - two_prod(s, s);
  return df_make(s) + r * __frcp_rn(2.f * s);
}

// floor and ceil of hi + lo: when hi is not an integer, |lo| <= ulp(hi)/2
// cannot carry the sum across one.
__device__ __forceinline__ float df_floor(df a) {
  const float f = floorf(a.hi);
  return f != a.hi ? f : f + floorf(a.lo);
}
__device__ __forceinline__ float df_ceil(df a) {
  const float c = ceilf(a.hi);
  return c != a.hi ? c : c + ceilf(a.lo);
}

}  // namespace gs2d
