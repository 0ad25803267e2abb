// Double-float ("FP32 pair") arithmetic for the FP64-accurate steps of the
// mixed-precision solve.
//
// GB300 executes FP64 FMA at about 1/63 of its FP32 rate (measured 1.19 vs
// 74.6 TFLOP/s), so the steps that must be accurate beyond FP32 -- the
// right-hand side, the true residual and W = U_K Wbar -- are computed with
// unevaluated sums hi + lo of two FP32 numbers (a 48-bit significand) using
// the error-free transformations
//   TwoSum  (Knuth):  s = a + b, e = (a - (s - bb)) + (b - bb), bb = s - a,
//                     with s + e = a + b exactly;
//   TwoProd (with a fused multiply-add): p = a b, e = fma(a, b, -p),
//                     with p + e = a b exactly;
// and the compensated dot-product scheme of Ogita, Rump and Oishi ("Accurate
// sum and dot product", SIAM J. Sci. Comput. 26, 2005): products are split
// exactly, their high parts summed with TwoSum, and every rounding error is
// collected in the low word.  A sum of k products is then as accurate as if
// computed with a 48-bit significand (error ~ k 2^-48 of the sum of the
// magnitudes), far below any residual tolerance the solver is asked for.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#include <cuda_runtime.h>
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

// The transformations are exact only if every product and sum below is
// rounded on its own; the device compiler would otherwise fuse a product and
// a following sum into one FMA.  The _rn intrinsics are never fused.  Host
// builds (the CPU unit test) must use -ffp-contract=off.
#if defined(__CUDA_ARCH__)
#define DF_MUL(a, b) __fmul_rn((a), (b))
#define DF_ADD(a, b) __fadd_rn((a), (b))
#define DF_SUB(a, b) __fsub_rn((a), (b))
#else
#define DF_MUL(a, b) ((a) * (b))
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#endif

namespace cphifi {

struct df {
  float hi, lo;
};

// Split of a double into hi + lo with hi = fl32(x) and
// |x - hi - lo| <= 2^-48 |x| (for x in the normal FP32 range).
DF_HD df df_from_double(double x) {
  const float hi = (float)x;
  const float lo = (float)(x - (double)hi);
  return {hi, lo};
}

DF_HD double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (|a| >= |b| not required).
DF_HD df two_sum(float a, float b) {
  const float s = DF_ADD(a, b);
  const float bb = DF_SUB(s, a);
  const float e = DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb));
  return {s, e};
}

// s + e = a + b exactly when |a| >= |b|.
DF_HD df fast_two_sum(float a, float b) {
  const float s = DF_ADD(a, b);
  const float e = DF_SUB(b, DF_SUB(s, a));
  return {s, e};
}

// (hi + lo) of x * y, x and y double-float; the dropped term lo_x lo_y is
// below 2^-48 of the product.
DF_HD df df_mul(df x, df y) {
  const float p = DF_MUL(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

// Lazily normalised accumulator: a.hi carries the TwoSum chain of the product
// heads, a.lo collects every rounding error (Ogita-Rump-Oishi).  Normalise
// with df_norm before using the value.
DF_HD void df_acc_prod(df& a, df x, df y) {
  const float p = DF_MUL(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  const float s = DF_ADD(a.hi, p);
  const float bb = DF_SUB(s, a.hi);
  const float t = DF_ADD(DF_SUB(a.hi, DF_SUB(s, bb)), DF_SUB(p, bb));
  a.hi = s;
  a.lo = DF_ADD(a.lo, DF_ADD(t, e));
}

// Adds a double-float value to the accumulator (same lazy scheme).
DF_HD void df_acc_add(df& a, df x) {
  const float s = DF_ADD(a.hi, x.hi);
  const float bb = DF_SUB(s, a.hi);
  const float t = DF_ADD(DF_SUB(a.hi, DF_SUB(s, bb)), DF_SUB(x.hi, bb));
  a.hi = s;
  a.lo = DF_ADD(a.lo, DF_ADD(t, x.lo));
}

DF_HD df df_norm(df a) { return two_sum(a.hi, a.lo); }

// a + b for normalised double-float values.
DF_HD df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = DF_ADD(s.lo, DF_ADD(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}

}  // namespace cphifi
