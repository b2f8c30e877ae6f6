// Double-float arithmetic: a value held as an unevaluated sum of two FP32
// terms, x = hi + lo with |lo| <= ulp(hi) / 2 (about 48 significant bits).
//
// GB300 issues FP64 arithmetic (and FP64 conversions) at 1/64 of its FP32
// rate, so on the element-wise paths of the refined form every FP64
// operation per vector entry costs about as much as a gather. The refined
// form therefore keeps its FP64-accurate quantities (the outer iterate, the
// refinement residual, the outer Lanczos basis) as two FP32 terms and works
// on them with FP32 instructions only, through the error-free transforms
// below:
//   two_sum  (Knuth):   s + e == a + b exactly, any a, b
//   quick_two_sum (Dekker): the same when |a| >= |b| (or a == 0)
//   two_prod (FMA):     p + e == a * b exactly
// The compound operations (add, mul) are the usual "sloppy" double-float
// forms: their error is about 2^-46 of the operands' magnitudes, which is
// what an absolute residual or a normalised Lanczos vector needs.
#pragma once
#include <cuda_runtime.h>

namespace wl {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_norm(float s, float e) { return quick_two_sum(s, e); }

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return two_sum(s.hi, e);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df{-b.hi, -b.lo}); }

__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  return two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.lo, p.lo);
  e = __fmaf_rn(a.lo, b.hi, e);
  return quick_two_sum(p.hi, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  return quick_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// running sum (s, c) += a with the rounding error of every add kept in c
__device__ __forceinline__ void df_acc(float& s, float& c, float a) {
  const df t = two_sum(s, a);
  s = t.hi;
  c = __fadd_rn(c, t.lo);
}

// running sum (s, c) += a (double-float)
__device__ __forceinline__ void df_acc2(float& s, float& c, df a) {
  const df t = two_sum(s, a.hi);
  s = t.hi;
  c = __fadd_rn(c, __fadd_rn(t.lo, a.lo));
}

// host/device split of an FP64 constant
__host__ __device__ inline df df_from_double(double x) {
  const float h = (float)x;
  return df{h, (float)(x - (double)h)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace wl
