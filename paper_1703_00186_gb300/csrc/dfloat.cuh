// Double-float ("double-word") arithmetic on the FP32 pipe.
//
// A value is hi + lo with two float32 words, |lo| <= ulp(hi) / 2, carrying
// about 48 significant bits.  The building blocks are the error-free
// transforms of Dekker (1971) and Knuth (TwoSum, Fast2Sum, and the exact
// product by FMA) and the double-word algorithms analysed by Joldes, Muller
// and Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44 (2017):
//   DWPlusFP, AccurateDWPlusDW, SloppyDWPlusDW, DWTimesFP (FMA variant),
//   DWTimesDW (FMA variant), each with a relative error of a few u^2,
//   u = 2^-24 (SloppyDWPlusDW: relative to |x| + |y|).
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

// SloppyDWPlusDW (same paper): x + y for double-words in 11 operations.  Its
// error is a few u^2 relative to |x| + |y| (not to |x + y|), so it is used
// only where the sum does not cancel: adding a smaller correction to a
// dominant term of the equilibrium polynomial.
__device__ __forceinline__ DF df_add_fast(DF x, DF y) {
  const DF s = df_two_sum(x.hi, y.hi);
  return df_fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
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

// float64 -> double-word without the FP64 pipe: integer arithmetic on the bit
// pattern.  hi is x rounded to float32 (half-up on the 29 dropped mantissa
// bits; the carry runs into the exponent field); the remainder x - hi is an
// exact integer multiple of 2^(e - 1075), |multiple| <= 2^28, and lo is its
// float32 rounding.  Representation error <= 2^-48 |x| for |x| >= 2^-74; below
// that lo would be subnormal and is dropped (error <= 2^-24 |x|, at most
// 2^-98 in absolute terms).  |x| < 2^-126 gives 0; |x| >= 2^128 (beyond
// float32) or non-finite x gives NaN, so a diverged state stays visible.
__device__ __forceinline__ DF df_from_double_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)(mag >> 52);
  const unsigned long long H = (mag + (1ull << 28)) & ~((1ull << 29) - 1ull);
  const int hbits = (int)(H >> 29) - (896 << 23);
  const long long D = (long long)(mag - H);  // exact, |D| <= 2^28
  const float scale = __int_as_float(max(e - 948, 1) << 23);
  float lo = (float)(int)D * scale;
  float hi = __int_as_float(hbits);
  if (e < 897) { hi = 0.f; lo = 0.f; }
  if (e > 1150) { hi = __int_as_float(0x7fc00000); lo = 0.f; }
  if (e < 949) lo = 0.f;
  return {__int_as_float(__float_as_int(hi) | (int)sign), __int_as_float(__float_as_int(lo) ^ (int)sign)};
}

// float32 -> float64 by bit arithmetic (exact for normal floats; zero and
// subnormals give 0; NaN/Inf stay NaN/Inf).
__device__ __forceinline__ double f32_to_f64_bits(float v) {
  const unsigned int u = (unsigned int)__float_as_int(v);
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  const unsigned long long ex = e == 255u ? 0x7FFull : (unsigned long long)(e + 896u);
  const unsigned long long bits = e == 0u ? sign : (sign | (ex << 52) | m);
  return __longlong_as_double((long long)bits);
}

// double-word -> float64: two exact conversions and one float64 add.
__device__ __forceinline__ double df_to_double_bits(DF v) { return f32_to_f64_bits(v.hi) + f32_to_f64_bits(v.lo); }

// x * k for a small integer k (exact scaling for powers of two).
__device__ __forceinline__ DF df_mul_int(DF x, int k) {
  if (k == 1) return x;
  if (k == -1) return df_neg(x);
  if (k == 2 || k == -2 || k == 4 || k == -4 || k == 8 || k == -8) return {x.hi * (float)k, x.lo * (float)k};
  return df_mul(x, (float)k);
}

}  // namespace lbm
