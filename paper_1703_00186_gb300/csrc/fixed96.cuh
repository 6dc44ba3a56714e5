// 96-bit two's-complement fixed-point numbers on the 2^-82 grid, for exact
// sums of float64 values on the integer pipe.
//
// GB300 executes float64 arithmetic at 1/64 of the float32 rate while its
// integer pipe is nearly idle in the float64 step, so the moment sums of the
// float64 collide are formed here: every population is converted exactly to
// fixed point (shifts of its mantissa), the sums are exact integer sums with
// carries, and each sum is rounded once to float64 (round to nearest even).
// The result is the correctly rounded exact sum whenever no summand has bits
// below 2^-82 (every |v| >= 2^-30 qualifies); smaller summands lose those
// bits, an error below 2^-76 per sum before the rounding.  Either way it is at
// least as accurate as any float64 summation order.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct Fix96 {
  unsigned w0, w1, w2;  // value = (w2:w1:w0, two's complement) * 2^-82
};

// Fixed-point grid: value = M * 2^(e - 1075) = (M << (e - kFixE0)) * 2^-82 for
// a float64 with biased exponent e and 53-bit significand M.
constexpr int kFixE0 = 993;
// Largest biased exponent converted exactly with a left shift of at most 31
// (|v| < 4); sums of up to 37 such values with weights up to 10 stay below
// 2^11, well inside the 2^13 range of the format.
constexpr int kFixEMax = kFixE0 + 31;

__device__ __forceinline__ Fix96 fix_add(Fix96 a, Fix96 b) {
  Fix96 r;
  asm("add.cc.u32 %0, %3, %6;\n\t"
      "addc.cc.u32 %1, %4, %7;\n\t"
      "addc.u32 %2, %5, %8;"
      : "=&r"(r.w0), "=&r"(r.w1), "=&r"(r.w2)
      : "r"(a.w0), "r"(a.w1), "r"(a.w2), "r"(b.w0), "r"(b.w1), "r"(b.w2));
  return r;
}

__device__ __forceinline__ Fix96 fix_sub(Fix96 a, Fix96 b) {
  Fix96 r;
  asm("sub.cc.u32 %0, %3, %6;\n\t"
      "subc.cc.u32 %1, %4, %7;\n\t"
      "subc.u32 %2, %5, %8;"
      : "=&r"(r.w0), "=&r"(r.w1), "=&r"(r.w2)
      : "r"(a.w0), "r"(a.w1), "r"(a.w2), "r"(b.w0), "r"(b.w1), "r"(b.w2));
  return r;
}

// acc + c a for an unsigned 32-bit multiplier c (modulo 2^96, so exact
// two's-complement arithmetic while the true result fits).
__device__ __forceinline__ Fix96 fix_mad(Fix96 acc, Fix96 a, unsigned c) {
  Fix96 r;
  asm("mad.lo.cc.u32 %0, %3, %6, %7;\n\t"
      "madc.lo.cc.u32 %1, %4, %6, %8;\n\t"
      "madc.lo.u32 %2, %5, %6, %9;\n\t"
      "mad.hi.cc.u32 %1, %3, %6, %1;\n\t"
      "madc.hi.u32 %2, %4, %6, %2;"
      : "=&r"(r.w0), "=&r"(r.w1), "=&r"(r.w2)
      : "r"(a.w0), "r"(a.w1), "r"(a.w2), "r"(c), "r"(acc.w0), "r"(acc.w1), "r"(acc.w2));
  return r;
}

// acc + k a for a small integer k of either sign (a constant after unrolling,
// so the branches fold away).
__device__ __forceinline__ Fix96 fix_axpy(Fix96 acc, Fix96 a, int k) {
  if (k == 0) return acc;
  if (k == 1) return fix_add(acc, a);
  if (k == -1) return fix_sub(acc, a);
  if (k > 0) return fix_mad(acc, a, (unsigned)k);
  return fix_sub(acc, fix_mad(Fix96{0u, 0u, 0u}, a, (unsigned)(-k)));
}

// Exact conversion of a float64 with biased exponent <= kFixEMax (|v| < 4).
// Values below 2^-30 keep their bits down to 2^-82 (the rest, < 2^-82, is
// dropped); zero and subnormals give 0.  `ok` is cleared for |v| >= 4,
// infinities and NaNs, which the format does not hold.
__device__ __forceinline__ Fix96 to_fix(double v, bool& ok) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7ffu);
  ok = ok && e <= kFixEMax;
  const unsigned m1 = (hi & 0xfffffu) | (e != 0 ? 0x100000u : 0u);  // top 21 significand bits
  const int s = e - kFixE0;
  Fix96 r;
  if (s >= 0) {
    const int t = s & 31;
    r.w0 = lo << t;
    r.w1 = __funnelshift_l(lo, m1, t);
    r.w2 = __funnelshift_l(m1, 0u, t);
  } else {
    const int t = -s;  // right shift of the 53-bit significand
    r.w0 = t < 32 ? __funnelshift_r(lo, m1, t) : (t < 53 ? m1 >> (t - 32) : 0u);
    r.w1 = t < 32 ? m1 >> t : 0u;
    r.w2 = 0u;
  }
  if (hi >> 31) r = fix_sub(Fix96{0u, 0u, 0u}, r);
  return r;
}

// to_fix for |v| < 2^(EMAX - 1022), EMAX <= kFixE0 + 42 (|v| < 2^12): the
// significand may also move past the first word (left shifts of 32 to 42).
// `ok` is cleared above that bound, for infinities and for NaNs.  Used for
// the coefficients of a polynomial whose evaluated sums the caller keeps
// inside the format's range by choosing EMAX per coefficient.
template <int EMAX>
__device__ __forceinline__ Fix96 to_fix_upto(double v, bool& ok) {
  static_assert(EMAX <= kFixE0 + 42, "the significand must stay below the sign bit");
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7ffu);
  ok = ok && e <= EMAX;
  const unsigned m1 = (hi & 0xfffffu) | (e != 0 ? 0x100000u : 0u);
  const int s = e - kFixE0;
  Fix96 r;
  if (s >= 32) {
    const int t = min(s - 32, 10);
    r.w0 = 0u;
    r.w1 = lo << t;
    r.w2 = __funnelshift_l(lo, m1, t);
  } else if (s >= 0) {
    const int t = s;
    r.w0 = lo << t;
    r.w1 = __funnelshift_l(lo, m1, t);
    r.w2 = __funnelshift_l(m1, 0u, t);
  } else {
    const int t = -s;
    r.w0 = t < 32 ? __funnelshift_r(lo, m1, t) : (t < 53 ? m1 >> (t - 32) : 0u);
    r.w1 = t < 32 ? m1 >> t : 0u;
    r.w2 = 0u;
  }
  if (hi >> 31) r = fix_sub(Fix96{0u, 0u, 0u}, r);
  return r;
}

// Block scaling for values of no fixed magnitude (cotangents): a per-site
// exponent D moves the whole set onto the grid, v 2^-D in fixed point and a
// fixed-point sum s back as s 2^D.  Both are exact exponent shifts (integer
// operations only).

// Biased exponent field of a float64.
__device__ __forceinline__ int exp_field(double v) { return (int)(((unsigned)__double2hiint(v) >> 20) & 0x7ffu); }

// to_fix of v 2^-D for a v whose biased exponent is at most kFixEMax + D
// (|v 2^-D| < 4), which the caller guarantees (D from the largest exponent
// of the set).  Bits below 2^(D - 82) are dropped, subnormals give 0.
__device__ __forceinline__ Fix96 to_fix_scaled(double v, int D) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned m1 = (hi & 0xfffffu) | 0x100000u;
  const int s = e - D - kFixE0;  // <= 31
  Fix96 r;
  if (e == 0) {
    r = Fix96{0u, 0u, 0u};
  } else if (s >= 0) {
    r.w0 = lo << s;
    r.w1 = __funnelshift_l(lo, m1, s);
    r.w2 = __funnelshift_l(m1, 0u, s);
  } else {
    const int t = -s;
    r.w0 = t < 32 ? __funnelshift_r(lo, m1, t) : (t < 53 ? m1 >> (t - 32) : 0u);
    r.w1 = t < 32 ? m1 >> t : 0u;
    r.w2 = 0u;
  }
  if (hi >> 31) r = fix_sub(Fix96{0u, 0u, 0u}, r);
  return r;
}

// Exact conversion of a float32 with |v| < 4 (biased exponent <= 128):
// v = M 2^(e - 150) for the 24-bit significand M, i.e. M shifted left by
// e - 68 <= 60 places on the 2^-82 grid.  Values below 2^-58 keep their bits
// down to 2^-82 (the rest is dropped); zero gives 0.  `ok` is cleared for
// |v| >= 4, infinities and NaNs.  Integer operations only.
__device__ __forceinline__ Fix96 to_fix_f32(float v, bool& ok) {
  const unsigned b = __float_as_uint(v);
  const int e = (int)((b >> 23) & 0xffu);
  ok = ok && e <= 128;
  const unsigned m = (b & 0x7fffffu) | (e != 0 ? 0x800000u : 0u);
  const int s = (e != 0 ? e : 1) - 68;
  Fix96 r;
  if (s >= 32) {
    const int t = min(s - 32, 31);  // t <= 28 while ok
    r.w0 = 0u;
    r.w1 = m << t;
    r.w2 = __funnelshift_l(m, 0u, t);
  } else if (s >= 0) {
    r.w0 = m << s;
    r.w1 = __funnelshift_l(m, 0u, s);
    r.w2 = 0u;
  } else {
    const int t = -s;
    r.w0 = t < 24 ? m >> t : 0u;
    r.w1 = 0u;
    r.w2 = 0u;
  }
  if (b >> 31) r = fix_sub(Fix96{0u, 0u, 0u}, r);
  return r;
}

// Round a 2^D (a fixed-point value) to the nearest float64 (ties to even).
// The magnitude is below 2^95; the caller keeps the result's exponent in
// the normal range (D = 0 always does).
__device__ __forceinline__ double fix_to_double_scaled(Fix96 a, int D) {
  const unsigned sign = a.w2 & 0x80000000u;
  if (sign) a = fix_sub(Fix96{0u, 0u, 0u}, a);
  if ((a.w0 | a.w1 | a.w2) == 0u) return 0.0;
  // word-align the leading word, then bit-align the leading one to bit 95
  unsigned n2 = a.w2, n1 = a.w1, n0 = a.w0;
  int lz = 0;
  if (n2 == 0u) {
    n2 = n1;
    n1 = n0;
    n0 = 0u;
    lz = 32;
    if (n2 == 0u) {
      n2 = n1;
      n1 = 0u;
      lz = 64;
    }
  }
  const int b = __clz(n2);
  n2 = __funnelshift_l(n1, n2, b);
  n1 = __funnelshift_l(n0, n1, b);
  n0 = n0 << b;  // b <= 31
  lz += b;
  // significand: bits 95..43 (n2 and the top 21 bits of n1); the rest rounds
  unsigned long long m = ((unsigned long long)n2 << 21) | (n1 >> 11);
  const unsigned rest = n1 & 0x7ffu;
  const bool up = rest > 0x400u || (rest == 0x400u && (n0 != 0u || (m & 1ull)));
  m += up ? 1ull : 0ull;
  // value = m 2^(13 - lz - 52); the implicit bit of m adds one to the
  // exponent field, and a carry out of the rounding adds one more
  const unsigned long long bits =
      ((unsigned long long)(13 - lz + 1022 + D) << 52) + m + ((unsigned long long)sign << 32);
  return __longlong_as_double((long long)bits);
}

// Round to the nearest float64 (ties to even).  The magnitude is below 2^95.
__device__ __forceinline__ double fix_to_double(Fix96 a) { return fix_to_double_scaled(a, 0); }

}  // namespace lbm
