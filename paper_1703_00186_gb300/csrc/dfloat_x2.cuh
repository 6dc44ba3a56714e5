// Two double-words side by side in the lanes of packed float32 instructions
// (f32x2.cuh): the algorithms of dfloat.cuh (Dekker, Knuth; Joldes, Muller
// and Popescu, ACM TOMS 44, 2017) with every float32 operation replaced by
// its packed form, so each lane's result is bit-identical to the scalar
// double-word operation on that lane's operands.
//
// There is no packed negation.  The exact product's error term needs -p for
// p = a * b; it is formed as a * (-b) (or (-a) * b), which equals -p exactly
// under round-to-nearest, so every product takes the negated high word of one
// of its factors, and p itself is never formed: p + t is computed as t - (-p).
#pragma once

#include "dfloat.cuh"
#include "f32x2.cuh"

namespace lbm {

struct DF2 {
  float2 hi, lo;
};

__device__ __forceinline__ DF2 df2_bcast(DF x) { return {f2s(x.hi), f2s(x.lo)}; }
__device__ __forceinline__ DF df2_lane0(DF2 x) { return {x.hi.x, x.lo.x}; }
__device__ __forceinline__ DF df2_lane1(DF2 x) { return {x.hi.y, x.lo.y}; }

// SloppyDWPlusDW per lane (df_add_fast).
__device__ __forceinline__ DF2 df2_add_fast(DF2 x, DF2 y) {
  const float2 s = add2(x.hi, y.hi);
  const float2 bb = sub2(s, x.hi);
  const float2 e = add2(sub2(x.hi, sub2(s, bb)), sub2(y.hi, bb));
  const float2 v = add2(e, add2(x.lo, y.lo));
  const float2 r = add2(s, v);
  return {r, sub2(v, sub2(r, s))};
}

// df_add_fast(x, df_neg(y)) per lane, without forming -y: with y' = -y,
// y'.hi - bb = -(y.hi + bb) and x.lo + y'.lo = x.lo - y.lo exactly.
__device__ __forceinline__ DF2 df2_sub_fast(DF2 x, DF2 y) {
  const float2 s = sub2(x.hi, y.hi);
  const float2 bb = sub2(s, x.hi);
  const float2 e = sub2(sub2(x.hi, sub2(s, bb)), add2(y.hi, bb));
  const float2 v = add2(e, sub2(x.lo, y.lo));
  const float2 r = add2(s, v);
  return {r, sub2(v, sub2(r, s))};
}

// DWTimesFP (df_mul(DF, float)) per lane, given ny = -y.
__device__ __forceinline__ DF2 df2_mul_f(DF2 x, float2 y, float2 ny) {
  const float2 np = mul2(x.hi, ny);    // -p, p = x.hi y rounded
  const float2 e = fma2(x.hi, y, np);  // x.hi y - p, exact
  const float2 t = fma2(x.lo, y, e);
  const float2 s = sub2(t, np);        // p + t
  return {s, sub2(t, add2(s, np))};    // t - (s - p)
}

// DWTimesDW (df_mul(DF, DF)) per lane, given nyh = -y.hi.
__device__ __forceinline__ DF2 df2_mul_ny(DF2 x, DF2 y, float2 nyh) {
  const float2 np = mul2(x.hi, nyh);
  const float2 e = fma2(x.hi, y.hi, np);
  const float2 t = fma2(x.hi, y.lo, mul2(x.lo, y.hi));
  const float2 b = add2(e, t);
  const float2 s = sub2(b, np);
  return {s, sub2(b, add2(s, np))};
}

// DWTimesDW per lane, given nxh = -x.hi.
__device__ __forceinline__ DF2 df2_mul_nx(DF2 x, DF2 y, float2 nxh) {
  const float2 np = mul2(nxh, y.hi);
  const float2 e = fma2(x.hi, y.hi, np);
  const float2 t = fma2(x.hi, y.lo, mul2(x.lo, y.hi));
  const float2 b = add2(e, t);
  const float2 s = sub2(b, np);
  return {s, sub2(b, add2(s, np))};
}

// -x.hi per lane (an exact multiplication by -1).
__device__ __forceinline__ float2 df2_neg_hi(DF2 x) { return mul2(x.hi, f2s(-1.0f)); }

}  // namespace lbm
