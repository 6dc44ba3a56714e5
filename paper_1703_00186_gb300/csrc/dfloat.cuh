// Double-float ("double-word") arithmetic on the FP32 pipe.
//
// A value is hi + lo with two float32 words, |lo| <= ulp(hi) / 2, carrying
// about 48 significant bits.  The building blocks are the error-free
// transforms of Dekker (1971) and Knuth (TwoSum, Fast2Sum, and the exact
// product by FMA) and the double-word algorithms analysed by Joldes, Muller
// and Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44 (2017):
//   DWPlusFP, AccurateDWPlusDW, DWTimesFP (FMA variant), DWTimesDW (FMA
//   variant), each with a relative error of a few u^2, u = 2^-24.
// On GB300 the FP32 pipe issues 64 times the FP64 rate, so a handful of
// float32 operations per emulated operation is still far cheaper.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ DF df_two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ DF df_from(float a) { return {a, 0.f}; }

// DWPlusFP: x + y for a double-word x and a float y.
__device__ __forceinline__ DF df_add(DF x, float y) {
  const DF s = df_two_sum(x.hi, y);
  return df_fast_two_sum(s.hi, x.lo + s.lo);
}

// AccurateDWPlusDW: x + y for double-words.
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = df_two_sum(x.hi, y.hi);
  const DF t = df_two_sum(x.lo, y.lo);
  const DF v = df_fast_two_sum(s.hi, s.lo + t.hi);
  return df_fast_two_sum(v.hi, t.lo + v.lo);
}

__device__ __forceinline__ DF df_neg(DF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ DF df_sub(DF x, DF y) { return df_add(x, df_neg(y)); }

// DWTimesFP (FMA variant): x * y for a double-word x and a float y.
__device__ __forceinline__ DF df_mul(DF x, float y) {
  const DF c = df_two_prod(x.hi, y);
  return df_fast_two_sum(c.hi, fmaf(x.lo, y, c.lo));
}

// DWTimesDW (FMA variant): x * y for double-words.
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const DF c = df_two_prod(x.hi, y.hi);
  const float t = fmaf(x.hi, y.lo, x.lo * y.hi);
  return df_fast_two_sum(c.hi, c.lo + t);
}

// x * y + z
__device__ __forceinline__ DF df_fma(DF x, DF y, DF z) { return df_add(df_mul(x, y), z); }

// 1 / x: float reciprocal seed refined by one Newton step in double-word,
// r <- r + r (1 - x r).
__device__ __forceinline__ DF df_rcp(DF x) {
  const float r = 1.0f / x.hi;
  const DF e = df_add(df_neg(df_mul(x, r)), 1.0f);   // 1 - x r
  return df_add(df_mul(e, r), r);
}

// Round a float64 to a double-word (two float64 -> float32 conversions).
__device__ __forceinline__ DF df_from_double(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ double df_to_double(DF x) { return (double)x.hi + (double)x.lo; }

}  // namespace lbm
