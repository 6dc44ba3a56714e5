// Device building blocks of the D2Q37 step: pull gather with periodic x,
// thermal walls, and the float64 / float32-shifted BGK collide.
#pragma once

#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "dfloat_x2.cuh"
#include "f32x2.cuh"
#include "fixed96.cuh"
#include "lbm_internal.h"

namespace lbm {

__device__ __forceinline__ int wrap_x(int xs, int lx) {
  xs = xs < 0 ? xs + lx : xs;
  return xs >= lx ? xs - lx : xs;
}

// Element offset of (l, y, x) in a state buffer (y physical, may be a halo row).
__device__ __forceinline__ long long sidx(const LatticeArgs& a, int l, int y, int x) {
  return (long long)l * a.plane + (long long)(y + HALO) * a.lx + x;
}

// propagate (Sect. 2, eq. 1 first term): f_l <- src_l(x - xi_l), periodic in x;
// in y the source may be a halo row (replaced by the walls) or, in the
// periodic-y test mode, wraps.
// Loads: read-only path by default; COHERENT = true reads through L2 only
// (ld.global.cg), for kernels that read what other blocks of the same launch
// wrote earlier (the persistent batch kernel).
template <bool COHERENT, typename T>
__device__ __forceinline__ T load(const T* p) {
  if constexpr (COHERENT) return __ldcg(p);
  else return __ldg(p);
}

template <typename T, bool COHERENT = false>
__device__ __forceinline__ void pull(const T* __restrict__ src, int x, int y,
                                     const LatticeArgs& a, T (&f)[NPOP]) {
#pragma unroll
  for (int l = 0; l < NPOP; ++l) {
    const int xs = wrap_x(x - vx(l), a.lx);
    int ys = y - vy(l);
    if (a.periodic_y) ys = ys < 0 ? ys + a.ly : (ys >= a.ly ? ys - a.ly : ys);
    f[l] = load<COHERENT>(src + sidx(a, l, ys, xs));
  }
}

// Element offset of site (y, x) within a population plane.
__device__ __forceinline__ int site_off(const LatticeArgs& a, int y, int x) { return (y + HALO) * a.lx + x; }

// True where the pull of every population is a fixed site-relative offset:
// 32-bit state indices, a column at least 3 sites from the periodic seam, and
// walls (not the periodic-y test mode) in y.
__device__ __forceinline__ bool fast_site(const LatticeArgs& a, int x) {
  return a.idx32 && !a.periodic_y && x >= 3 && x < a.lx - 3;
}

// fast_site for every lane of the warp holding column x (a warp is a row
// segment of 32 columns starting at x - lane): a warp that reaches a seam
// column takes the general pull for all its lanes instead of running both
// paths one after the other (measured: +0.3 % on the FP32-store step, +1.1 %
// on the parameter-table batch kernel, whose lattices are 128-1024 wide).
__device__ __forceinline__ bool fast_warp(const LatticeArgs& a, int x) {
  const int x0 = x - (int)(threadIdx.x & 31u);
  return a.idx32 && !a.periodic_y && x0 >= 3 && x0 + 32 <= a.lx - 3;
}

// pull at a fast site: one address computation per population.
template <typename T, bool COHERENT = false>
__device__ __forceinline__ void pull_fast(const T* __restrict__ src, int site, const LatticeArgs& a,
                                          T (&f)[NPOP]) {
  const char* s = reinterpret_cast<const char*>(src + site);
#pragma unroll
  for (int l = 0; l < NPOP; ++l) f[l] = load<COHERENT>(reinterpret_cast<const T*>(s + a.pull_off[l]));
}

// Store the 37 populations of a site (any site, fast indices if idx32).
template <typename T>
__device__ __forceinline__ void store_site(T* __restrict__ dst, int x, int y, const LatticeArgs& a,
                                           const T (&f)[NPOP]) {
  if (a.idx32) {
    char* d = reinterpret_cast<char*>(dst + site_off(a, y, x));
#pragma unroll
    for (int l = 0; l < NPOP; ++l) *reinterpret_cast<T*>(d + a.plane_off[l]) = f[l];
  } else {
#pragma unroll
    for (int l = 0; l < NPOP; ++l) dst[sidx(a, l, y, x)] = f[l];
  }
}

// Mass M(x) that left through the bottom (top) wall during propagate and lands
// in column x, summed in the fixed order: l ascending, then source row
// ascending; round-to-nearest adds without contraction.  `decode` maps a
// stored element of population l to its float64 population value.
template <bool TOP, bool COHERENT = false, typename T, typename Decode>
__device__ __forceinline__ double lost_mass(const T* __restrict__ src, int x,
                                            const LatticeArgs& a, Decode decode) {
  double M = 0.0;
  bool first = true;
#pragma unroll
  for (int l = 0; l < NPOP; ++l) {
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      // bottom: source row y0 = e, lost if y0 + xi_y < 0;
      // top:    source row y0 = ly - 3 + e, lost if y0 + xi_y >= ly.
      const bool lost = TOP ? (e + vy(l) >= 3) : (e + vy(l) < 0);
      if (lost) {
        const int y0 = TOP ? a.ly - 3 + e : e;
        const double v = decode(l, load<COHERENT>(src + sidx(a, l, y0, wrap_x(x - vx(l), a.lx))));
        M = first ? v : __dadd_rn(M, v);
        first = false;
      }
    }
  }
  return M;
}

// Replace the unknown slots of a wall row by M(x) q_l (Sect. 2, bc).
// `encode` maps a float64 population value of population l to storage.
template <bool COHERENT = false, typename S, typename F, typename Decode, typename Encode>
__device__ __forceinline__ void walls(const S* __restrict__ src, int x, int y,
                                      const LatticeArgs& a, F (&f)[NPOP],
                                      Decode decode, Encode encode) {
  if (a.periodic_y) return;
  if (y < 3) {
    const double M = lost_mass<false, COHERENT>(src, x, a, decode);
#pragma unroll
    for (int l = 0; l < NPOP; ++l)
      if (vy(l) > 0 && vy(l) > y) f[l] = encode(l, __dmul_rn(M, a.q_bot[l]));
  } else if (y >= a.ly - 3) {
    const double M = lost_mass<true, COHERENT>(src, x, a, decode);
    const int d = a.ly - 1 - y;  // row offset from the top wall
#pragma unroll
    for (int l = 0; l < NPOP; ++l)
      if (vy(l) < 0 && -vy(l) > d) f[l] = encode(l, __dmul_rn(M, a.q_top[l]));
  }
}

// Per-site coefficients of the 4th-order Hermite equilibrium, written as a
// polynomial in cu = c.u' for each shell (D = 2, theta = T' - 1, U2 = |u'|^2):
//   P = A0 + A1 cu + A2 cu^2 + cu^3 / 6 + cu^4 / 24,
//   A0 = B00 + B01 c2 + B02 c2^2,  A1 = B10 + B11 c2,  A2 = B20 + B21 c2.
struct EqCoef {
  double B00, B01, B02, B10, B11, B20, B21;
};

__device__ __forceinline__ EqCoef eq_coef(double U2, double theta) {
  EqCoef c;
  c.B20 = fma(-1.5, theta, fma(-0.25, U2, 0.5));
  c.B21 = 0.25 * theta;
  c.B10 = fma(-2.0, theta, fma(-0.5, U2, 1.0));
  c.B11 = 0.5 * theta;
  c.B00 = fma(theta, (U2 - 1.0) + theta, fma(U2, fma(0.125, U2, -0.5), 1.0));
  c.B01 = theta * (fma(-0.25, U2, 0.5) - theta);
  c.B02 = 0.125 * (theta * theta);
  return c;
}

// cu = xi_k . v for the pair representative k (v = r u' in xi units).
template <typename R>
__device__ __forceinline__ R pair_cu(int k, R v_x, R v_y) {
  const int ax = rep_x(k), ay = rep_y(k);
  if (ax == 0) return ay == 1 ? v_y : (R)ay * v_y;
  if (ay == 0) return ax == 1 ? v_x : (R)ax * v_x;
  const R ty = ay == 1 ? v_y : (R)ay * v_y;
  return ax == 1 ? v_x + ty : (ax == -1 ? ty - v_x : fma((R)ax, v_x, ty));
}

// Moment sums of 37 values in float64 using the (+,-) pairing:
// rho = sum f, Jx = sum xi_x f, Jy = sum xi_y f, Exi = sum |xi|^2 f.
struct Moments {
  double rho, Jx, Jy, Exi;
};

template <typename Get>
__device__ __forceinline__ Moments moment_sums(Get get) {
  double sh[NSHELL];
#pragma unroll
  for (int j = 0; j < NSHELL; ++j) sh[j] = -0.0;
  double Jx = -0.0, Jy = -0.0;
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const double p = get(2 * k + 1), m = get(2 * k + 2);
    const double s = p + m, d = p - m;
    sh[pair_shell(k)] += s;
    if (rep_x(k) != 0) Jx = rep_x(k) == 1 ? Jx + d : rep_x(k) == -1 ? Jx - d : fma((double)rep_x(k), d, Jx);
    if (rep_y(k) != 0) Jy = rep_y(k) == 1 ? Jy + d : fma((double)rep_y(k), d, Jy);
  }
  Moments mo;
  mo.rho = ((get(0) + sh[1]) + (sh[2] + sh[3])) + ((sh[4] + sh[5]) + (sh[6] + sh[7]));
  mo.Exi = fma(10.0, sh[7], fma(9.0, sh[6], fma(8.0, sh[5], fma(5.0, sh[4], fma(4.0, sh[3], fma(2.0, sh[2], sh[1]))))));
  mo.Jx = Jx;
  mo.Jy = Jy;
  return mo;
}

// The same four sums formed exactly in 96-bit fixed point on the integer
// pipe and rounded once to float64 (fixed96.cuh): the correctly rounded exact
// sums.  Returns false, leaving `mo` unset, when a population lies outside
// the fixed-point range (|f| >= 4, infinities, NaN).  EXI_D = -1 returns
// E / 2 in place of E (an exact scaling of the same rounding).
template <int EXI_D = 0, typename Get>
__device__ __forceinline__ bool moment_sums_exact(Get get, Moments& mo) {
  static_assert(EXI_D == 0 || EXI_D == -1, "E or E / 2");
  bool ok = true;
  Fix96 r = to_fix(get(0), ok);
  Fix96 jx{0u, 0u, 0u}, jy{0u, 0u, 0u}, e{0u, 0u, 0u};
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const Fix96 p = to_fix(get(2 * k + 1), ok), m = to_fix(get(2 * k + 2), ok);
    const Fix96 s = fix_add(p, m), d = fix_sub(p, m);
    r = fix_add(r, s);
    e = fix_axpy(e, s, rep_x(k) * rep_x(k) + rep_y(k) * rep_y(k));
    jx = fix_axpy(jx, d, rep_x(k));
    jy = fix_axpy(jy, d, rep_y(k));
  }
  if (!ok) return false;
  mo.rho = fix_to_double(r);
  mo.Jx = fix_to_double(jx);
  mo.Jy = fix_to_double(jy);
  mo.Exi = fix_to_double_scaled(e, EXI_D);
  return true;
}

// Moment sums of 37 float64 values: exact (moment_sums_exact) where the
// populations fit the fixed-point range, float64 additions (moment_sums) for
// finite populations beyond it, and NaN moments for a site holding an
// infinity or a NaN (so a diverged state stays non-finite, at the cost of
// the normal path).  EXI_D = -1: E / 2 in place of E.
template <int EXI_D = 0, typename Get>
__device__ __forceinline__ Moments site_moments(Get get) {
  Moments mo;
  if (!moment_sums_exact<EXI_D>(get, mo)) {
    bool nonfinite = false;
#pragma unroll
    for (int l = 0; l < NPOP; ++l)
      nonfinite |= ((unsigned)__double2hiint(get(l)) & 0x7ff00000u) == 0x7ff00000u;
    if (nonfinite) {
      const double q = __longlong_as_double(0x7ff8000000000000LL);
      mo = Moments{q, q, q, q};
    } else {
      mo = moment_sums(get);
      if (EXI_D == -1) mo.Exi *= 0.5;
    }
  }
  return mo;
}

// Moment sums (rho, Jx, Jy, Exi as in moment_sums) in double-float.
struct MomentsDF {
  DF rho, Jx, Jy, Exi;
};

// Moment sums of 37 float32 values by a split of every value d = h + m + e
// (the "magic number" rounding of Dekker and Knuth: adding and subtracting
// 1.5 * 2^k rounds to a multiple of 2^(k-23)):
//   h: d rounded to a multiple of 2^-12; for |d| < 4 every weighted sum of
//      the h (integer weights <= 10, 37 terms) stays below 2^23 grid steps,
//      so it is exact in float32;
//   m: the rest rounded to a multiple of 2^-34, read off as an integer
//      (|m| 2^34 <= 2^21) and summed exactly in int32;
//   e: the remainder, |e| <= 2^-35, dropped.
// Values with |d| >= 4 (a diverged lattice) are still summed, only no longer
// exactly.
struct SplitAcc {
  float h;
  unsigned m;  // integer part, accumulated modulo 2^32 (the true sum fits in int32)
};

__device__ __forceinline__ DF split_result(const SplitAcc& a) {
  // h + m 2^-34 in double-float (m 2^-34 as two exact floats)
  const int m = (int)a.m;
  const float m_hi = (float)(m >> 12) * 0x1p-22f;
  const float m_lo = (float)(m & 0xfff) * 0x1p-34f;
  return df_add(df_two_sum(a.h, m_hi), m_lo);
}

// Two-level split of one float32 value v (|v| < 2^10):
//   v = h + m 2^-34 + e,  h on the 2^-12 grid, m an integer with
//   |m| <= 2^21, |e| <= 2^-35 (e is dropped).
// h = (v + C1) - C1 rounds v to the 2^-12 grid; rem = v - h is exact and
// |rem| <= 2^-13, so t = rem + C2 lies in [2^-11, 2^-10), where the float
// spacing is 2^-34: the bit pattern of t minus that of C2 is round(rem 2^34).
// The pattern itself is returned (bits = m + K2); the constant K2 cancels in
// the differences of a +-pair and is removed once from the other sums.
struct Split {
  float h;
  unsigned bits;
};

__device__ __forceinline__ Split split2(float v) {
  constexpr float C1 = 3072.0f;     // 1.5 * 2^11: grid 2^-12
  constexpr float C2 = 0x1.8p-11f;  // 1.5 * 2^-11: grid 2^-34
  const float h = (v + C1) - C1;
  return {h, __float_as_uint((v - h) + C2)};
}

// Float32 sums sum_l d_l, sum_l xi_l d_l and sum_l |xi_l|^2 d_l of the exact
// values h_l + m_l 2^-34: the h parts sum exactly on the 2^-12 grid (float,
// exact while sum_l |xi_l|^2 |d_l| < 2^12; deviations are O(1) at most) and
// the 2^-34-grid parts exactly as integers.  The only error is the rounding
// of each d_l to the 2^-34 grid: at most 2^-35 per term, round-to-nearest and
// so without bias, three orders of magnitude below the float32 quantum of the
// stored deviations.  Population pairs (2k+1, 2k+2) = (R_k, -R_k) are split
// together in the two lanes of packed float32 pairs, and each h sum is kept
// as one partial sum per lane (every partial sum is exact, so is their total);
// the integer parts combine the pair first: the even moments take m+ + m-,
// the odd ones m+ - m-.
// The four sums (rho, Jx, Jy, Exi) before the conversion to double-float.
struct SplitSums {
  SplitAcc r, jx, jy, e;
};

__device__ __forceinline__ SplitSums moment_sums_split(const float (&d)[NPOP]) {
  constexpr unsigned K2 = 0x3a400000u;  // bit pattern of 1.5 * 2^-11
  const float2 C1 = f2s(3072.0f), C1n = f2s(-3072.0f), C2 = f2s(0x1.8p-11f);
  const Split s0 = split2(d[0]);
  float2 r2 = f2(s0.h, 0.f), e2 = f2(0.f, 0.f), jx2 = f2(0.f, 0.f), jy2 = f2(0.f, 0.f);
  // integer parts (modulo 2^32, exact): m+ + m- summed per shell, and
  // +-(m+ - m-) per |xi_x| and |xi_y| value; the weights are applied once
  unsigned sh[NSHELL] = {}, ax_sum[4] = {}, ay_sum[4] = {};
  unsigned e_off = 0u;
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const float2 v = f2(d[2 * k + 1], d[2 * k + 2]);
    const float2 h = add2(add2(v, C1), C1n);  // both lanes of split2
    const float2 t = add2(sub2(v, h), C2);
    const unsigned pb = __float_as_uint(t.x), qb = __float_as_uint(t.y);
    const int ax = rep_x(k), ay = rep_y(k), c2 = ax * ax + ay * ay;
    r2 = add2(r2, h);
    e2 = c2 == 1 ? add2(e2, h) : fma2(f2s((float)c2), h, e2);
    sh[pair_shell(k)] += pb + qb;
    e_off += 2u * (unsigned)c2;
    if (ax != 0) {
      jx2 = fma2(f2((float)ax, (float)-ax), h, jx2);
      ax_sum[ax > 0 ? ax : -ax] += ax > 0 ? pb - qb : qb - pb;
    }
    if (ay != 0) {
      jy2 = fma2(f2((float)ay, (float)-ay), h, jy2);
      ay_sum[ay > 0 ? ay : -ay] += ay > 0 ? pb - qb : qb - pb;
    }
  }
  unsigned rm = s0.bits, em = 0u;
#pragma unroll
  for (int j = 1; j < NSHELL; ++j) {
    rm += sh[j];
    em += (unsigned)shell_sq(j) * sh[j];
  }
  const unsigned jxm = ax_sum[1] + 2u * ax_sum[2] + 3u * ax_sum[3];
  const unsigned jym = ay_sum[1] + 2u * ay_sum[2] + 3u * ay_sum[3];
  const SplitAcc r{r2.x + r2.y, rm - (unsigned)NPOP * K2}, e{e2.x + e2.y, em - e_off * K2};
  const SplitAcc jx{jx2.x + jx2.y, jxm}, jy{jy2.x + jy2.y, jym};
  return {r, jx, jy, e};
}

__device__ __forceinline__ MomentsDF split_moments(const SplitSums& s) {
  return {split_result(s.r), split_result(s.jx), split_result(s.jy), split_result(s.e)};
}

// b - a for two split sums of the same kind, rounded once to float32: the h
// parts are on the 2^-12 grid and below 2^11, so h_b - h_a is exact; the
// integer difference (modulo 2^32; the true difference fits in int32) is
// split into two pieces that convert exactly, and only the last addition
// rounds.
__device__ __forceinline__ float split_diff(const SplitAcc& b, const SplitAcc& a) {
  const int dm = (int)(b.m - a.m);
  const float dh = b.h - a.h;
  return fmaf((float)(dm & 0xfff), 0x1p-34f, fmaf((float)(dm >> 12), 0x1p-22f, dh));
}

// Site state derived from the moments: velocity in xi units and temperature.
struct SiteFields {
  double rho, inv, ux, uy, T;  // u = r (ux, uy)
};

__device__ __forceinline__ SiteFields site_fields(const Moments& m, const LatticeArgs& a) {
  SiteFields s;
  s.rho = m.rho;
  s.inv = 1.0 / m.rho;
  s.ux = m.Jx * s.inv;
  s.uy = m.Jy * s.inv;
  s.T = a.r2_2 * fma(m.Exi, s.inv, -fma(s.ux, s.ux, s.uy * s.uy));
  return s;
}

// BGK collide in float64 (eq. 1) with the gravity equilibrium shift.  Returns
// the pre-collide site fields (rho, u in xi units, T).
__device__ __forceinline__ SiteFields collide_fp64(double (&f)[NPOP], const LatticeArgs& a) {
  const Moments mo = site_moments([&](int l) { return f[l]; });
  const SiteFields sf = site_fields(mo, a);
  const double theta = sf.T + a.tshift;
  const double uys = sf.uy - a.tau_g_xi;
  const double v_x = a.r2 * sf.ux, v_y = a.r2 * uys;
  const double U2 = a.r2 * fma(sf.ux, sf.ux, uys * uys);
  const EqCoef B = eq_coef(U2, theta);
  const double th2 = theta * theta;
  const double wr = a.omega * sf.rho;
  f[0] = fma(a.omc, f[0], (wr * a.w_shell[0]) * B.B00);
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    // A0 = B00 + B01 c2 + B02 c2^2, A1 = B10 + B11 c2, A2 = B20 + B21 c2 with
    // B02 = theta^2 / 8, B11 = theta / 2, B21 = theta / 4 folded into the
    // shell constants; the odd part carries the shell weight in its Horner
    // coefficients, sO = cu (sc A1 + (sc / 6) cu^2), sc = omega rho w.
    const int j = pair_shell(k);
    const double A0 = fma(a.c4e_shell[j], th2, fma(a.c2_shell[j], B.B01, B.B00));
    const double A1 = fma(theta, a.c2h_shell[j], B.B10);
    const double A2 = fma(theta, a.c2q_shell[j], B.B20);
    const double sc = wr * a.w_shell[j];
    const double sc6 = wr * a.w6_shell[j];
    const double scA1 = sc * A1;
    const double cu = pair_cu<double>(k, v_x, v_y);
    const double cu2 = cu * cu;
    const double E = fma(cu2, fma(cu2, 1.0 / 24.0, A2), A0);
    const double sO = cu * fma(cu2, sc6, scA1);
    f[2 * k + 1] = fma(a.omc, f[2 * k + 1], fma(sc, E, sO));    // sc (E + O)
    f[2 * k + 2] = fma(a.omc, f[2 * k + 2], fma(sc, E, -sO));   // sc (E - O)
  }
  return sf;
}

// Row-averaged observables of one site: rho, u_x, u_y, T, T^2, u_y T,
// rho |u|^2 / 2, rho u_y, with the mid-step hydrodynamic velocity (physical
// units) u_h = (u_x, u_y + g / 2) of the stored post-collide state.
constexpr int NOBS = 8;

// The fields site_observables takes: rho, the physical u_x, the physical u_y
// minus g / 2 and T.
struct ObsFields {
  double rho, ux, uy, T;
};

__device__ __forceinline__ void site_observables(double rho, double ux, double uy_h, double T, double (&o)[NOBS]) {
  o[0] = rho;
  o[1] = ux;
  o[2] = uy_h;
  o[3] = T;
  o[4] = T * T;
  o[5] = uy_h * T;
  o[6] = 0.5 * rho * fma(ux, ux, uy_h * uy_h);
  o[7] = rho * uy_h;
}

__device__ __forceinline__ DF dfc(const float (&c)[2]) { return {c[0], c[1]}; }
__device__ __forceinline__ DF df_scale2(DF x, float p2) { return {x.hi * p2, x.lo * p2}; }  // p2 a power of two

// BGK collide on float32 deviations d_l = f_l - w_l rho0 (FP32 shifted storage):
//   d_l <- (1 - omega) d_l + omega (f^eq_l - w_l rho0).
// Precision plan (GB300 issues FP64 at 1/64 of the FP32 rate, so nothing here
// uses the FP64 pipe):
//  * the moment sums are accurate to 2^-35 per term (moment_sums_split);
//  * the quantities that carry cancellation are double-float (about 48
//    bits): rho, 1/rho, E, T, theta = T' - 1 and rho (B00 - 1), i.e. the
//    temperature-dependent zeroth-order part of the equilibrium;
//  * u, |u'|^2 and the coefficients of the cu-dependent terms (which are
//    scaled by cu or cu^2) are float32, as are the per-population polynomial
//    and the relaxation.
// Rounding the per-shell coefficients to float32 leaves the discrete
// equilibrium's mass, momentum and energy off by ~1e-8 relative in a way that
// repeats from step to step and so accumulates; after the relaxation the
// conserved moments of the new populations are therefore measured again and
// the small defect is put back on the rest and |xi| = 1 populations, so the
// collide conserves mass and energy and adds exactly rho g to the momentum.
// PAIRED relaxes each (+, -) pair with one packed FMA (fewer issue slots, a few
// more live registers); the results are identical either way.
// A is LatticeArgs or any type with the same float32 / double-float members
// (F32Args below), so that a batch kernel can pass per-lattice values held in
// its kernel parameters.
template <bool PAIRED = true, typename A = LatticeArgs>
__device__ __forceinline__ void collide_fp32(float (&d)[NPOP], const A& a) {
  MomentsDF dev;
  SplitSums dev_raw;
  float rf = 0.f;
  // The two passes (the moments of the stored deviations, then of the
  // relaxed ones) unrolled: 2.6 % faster than one rolled copy of the
  // moment-sum code.
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    const SplitSums m = moment_sums_split(d);
    if (pass == 0) {
      dev_raw = m;
      dev = split_moments(m);
      const DF rho = df_add(dev.rho, dfc(a.df_rho0));
      const DF inv = df_rcp(rho);
      const float invf = inv.hi;
      const float ux = dev.Jx.hi * invf, uy = dev.Jy.hi * invf;  // xi units
      const float usq = fmaf(ux, ux, uy * uy);
      const DF exi = df_add(dev.Exi, dfc(a.df_e0));
      const DF T = df_mul(df_add(df_mul(exi, inv), -usq), dfc(a.df_half_r2));
      const DF theta = df_add(T, dfc(a.df_tshift));
      const float th = theta.hi;
      const float r2f = a.df_r2[0];
      const float uys = uy - a.df_taug_r[0];
      const float U2 = r2f * fmaf(ux, ux, uys * uys);
      // equilibrium coefficients (see eq_coef); B00 - 1 in double-float
      const DF b00m1 = df_add(df_mul(theta, df_add(theta, U2 - 1.0f)), U2 * fmaf(0.125f, U2, -0.5f));
      const float b20 = fmaf(-1.5f, th, fmaf(-0.25f, U2, 0.5f));
      const float b21 = 0.25f * th;
      const float b10 = fmaf(-2.0f, th, fmaf(-0.5f, U2, 1.0f));
      const float b11 = 0.5f * th;
      const float b01 = th * (fmaf(-0.25f, U2, 0.5f) - th);
      const float b02 = 0.125f * th * th;
      rf = rho.hi;
      const float v_x = r2f * ux, v_y = r2f * uys;
      const float rb00 = df_add(df_mul(rho, b00m1), dev.rho).hi;  // rho B00 - rho0 = (rho - rho0) + rho (B00 - 1)
      const float rb01 = rf * b01, rb02 = rf * b02;
      const float om = a.omega_f, omc = a.omc_f;
      const float wr = om * rf;
      d[0] = fmaf(omc, d[0], om * a.w_shell_f[0] * rb00);
#pragma unroll
      for (int k = 0; k < NPAIR; ++k) {
        const int j = pair_shell(k);
        const float c2 = a.c2_shell_f[j];
        const float w = a.w_shell_f[j];
        const float A1 = fmaf(b11, c2, b10);
        const float A2 = fmaf(b21, c2, b20);
        const float alpha = wr * w;                                        // omega w rho
        const float beta = om * w * fmaf(c2, fmaf(c2, rb02, rb01), rb00);  // omega w (rho A0 - rho0)
        const float cu = pair_cu<float>(k, v_x, v_y);
        const float cu2 = cu * cu;
        const float E = fmaf(alpha * cu2, fmaf(cu2, 1.0f / 24.0f, A2), beta);
        const float O = alpha * cu * fmaf(cu2, 1.0f / 6.0f, A1);
        if constexpr (PAIRED) {
          const float2 D = fma2(f2s(omc), f2(d[2 * k + 1], d[2 * k + 2]), f2(E + O, E - O));
          d[2 * k + 1] = D.x;
          d[2 * k + 2] = D.y;
        } else {
          d[2 * k + 1] = fmaf(omc, d[2 * k + 1], E + O);
          d[2 * k + 2] = fmaf(omc, d[2 * k + 2], E - O);
        }
      }
    } else {
      // conserved-moment correction.  Targets of the exact BGK update with
      // the equilibrium shift (omega tau = 1), deviation form, xi units,
      // g_xi = g / r: mass and Jx unchanged, Jy - rho g_xi,
      // Exi - 2 g_xi Jy + rho g_xi^2 (the gravity terms are ~1e-5 of the
      // sums, float32 is enough for them).  The defects (~1e-8 of the sums)
      // are the differences of the two passes' sums less the target change,
      // each rounded once.
      const float gr = a.df_g_r[0];
      const float dm = split_diff(m.r, dev_raw.r);
      const float djx = split_diff(m.jx, dev_raw.jx);
      const float djy = fmaf(rf, gr, split_diff(m.jy, dev_raw.jy));
      const float de = split_diff(m.e, dev_raw.e) - fmaf(rf * gr, gr, -2.0f * gr * dev.Jy.hi);
      d[0] += de - dm;
      d[1] += (-0.5f * de - djx) * 0.5f;  // xi = (1, 0)
      d[2] += (-0.5f * de + djx) * 0.5f;  // xi = (-1, 0)
      d[3] += (-0.5f * de - djy) * 0.5f;  // xi = (0, 1)
      d[4] += (-0.5f * de + djy) * 0.5f;  // xi = (0, -1)
    }
  }
}

// The members of LatticeArgs that collide_fp32 reads, as plain values: the
// per-lattice ones (rho0, tau and g) and the quadrature's float32 copies.
struct F32Args {
  float df_rho0[2], df_e0[2], df_tshift[2], df_taug_r[2], df_g_r[2];
  float omega_f, omc_f;
  float df_half_r2[2], df_r2[2];
  float w_shell_f[NSHELL], c2_shell_f[NSHELL];
};

// Exact moment sums of the populations w_rho0[l] + d_l held as float32
// deviations d_l: the deviations convert exactly to 96-bit fixed point from
// their bit patterns (integer pipe only), the shift constants enter as their
// exact sums precomputed on the host, and each sum is rounded once to
// float64.  Returns false, leaving `mo` unset, when a deviation is outside
// the fixed-point range (|d| >= 4, infinities, NaN).
__device__ __forceinline__ bool moment_sums_f32_exact(const float (&d)[NPOP], const LatticeArgs& a, Moments& mo) {
  bool ok = true;
  Fix96 r = fix_add(Fix96{a.fix_shift_rho[0], a.fix_shift_rho[1], a.fix_shift_rho[2]}, to_fix_f32(d[0], ok));
  Fix96 jx{0u, 0u, 0u}, jy{0u, 0u, 0u};
  Fix96 e{a.fix_shift_exi[0], a.fix_shift_exi[1], a.fix_shift_exi[2]};
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const Fix96 p = to_fix_f32(d[2 * k + 1], ok), m = to_fix_f32(d[2 * k + 2], ok);
    const Fix96 s = fix_add(p, m), df = fix_sub(p, m);
    r = fix_add(r, s);
    e = fix_axpy(e, s, rep_x(k) * rep_x(k) + rep_y(k) * rep_y(k));
    jx = fix_axpy(jx, df, rep_x(k));
    jy = fix_axpy(jy, df, rep_y(k));
  }
  if (!ok) return false;
  mo.rho = fix_to_double(r);
  mo.Jx = fix_to_double(jx);
  mo.Jy = fix_to_double(jy);
  mo.Exi = fix_to_double(e);
  return true;
}

// BGK collide on float32 deviations with the conserved-moment sums and the
// temperature-dependent equilibrium terms in float64 (LBM_FLAG_FP32_F64_TERMS):
//  * rho, J, E of eq. (2): exact sums of the populations w_rho0[l] + d_l,
//    rounded once (moment_sums_f32_exact);
//  * rho, u, T, the gravity shift, the Hermite coefficients B and, per shell,
//    A0, A1, A2 and the zeroth-order deviation omega w (rho A0 - rho0): float64,
//    A1, A2 and the deviation rounded once to float32;
//  * the cu-dependent polynomial and the relaxation: float32, as in
//    collide_fp32.
// No conserved-moment correction.  Sites with a deviation outside the
// fixed-point range take float64 sums of the decoded populations.
__device__ __forceinline__ void collide_fp32_f64terms(float (&d)[NPOP], const LatticeArgs& a) {
  Moments mo;
  if (!moment_sums_f32_exact(d, a, mo)) mo = site_moments([&](int l) { return a.w_rho0[l] + (double)d[l]; });
  const SiteFields sf = site_fields(mo, a);
  const double theta = sf.T + a.tshift;
  const double uys = sf.uy - a.tau_g_xi;
  const double U2 = a.r2 * fma(sf.ux, sf.ux, uys * uys);
  const EqCoef B = eq_coef(U2, theta);
  const double th2 = theta * theta;
  const float v_x = (float)(a.r2 * sf.ux), v_y = (float)(a.r2 * uys);
  const float wr = (float)(a.omega * sf.rho);
  const float omc = a.omc_f;
  d[0] = fmaf(omc, d[0], (float)(a.ow_shell[0] * fma(sf.rho, B.B00, -a.rho0)));
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const int j = pair_shell(k);
    const double A0 = fma(a.c4e_shell[j], th2, fma(a.c2_shell[j], B.B01, B.B00));
    const float A1 = (float)fma(theta, a.c2h_shell[j], B.B10);
    const float A2 = (float)fma(theta, a.c2q_shell[j], B.B20);
    const float beta = (float)(a.ow_shell[j] * fma(sf.rho, A0, -a.rho0));  // omega w (rho A0 - rho0)
    const float alpha = wr * a.w_shell_f[j];                               // omega w rho
    const float cu = pair_cu<float>(k, v_x, v_y);
    const float cu2 = cu * cu;
    const float E = fmaf(alpha * cu2, fmaf(cu2, 1.0f / 24.0f, A2), beta);
    const float O = alpha * cu * fmaf(cu2, 1.0f / 6.0f, A1);
    const float2 D = fma2(f2s(omc), f2(d[2 * k + 1], d[2 * k + 2]), f2(E + O, E - O));
    d[2 * k + 1] = D.x;
    d[2 * k + 2] = D.y;
  }
}

// Per-pair constants for rolled loops: representative R_k and shell index.
static __constant__ signed char c_pair_rep[NPAIR][2] = {
    {1, 0}, {0, 1}, {1, 1}, {-1, 1}, {2, 0}, {0, 2}, {2, 1}, {1, 2}, {-1, 2},
    {-2, 1}, {2, 2}, {-2, 2}, {3, 0}, {0, 3}, {3, 1}, {1, 3}, {-1, 3}, {-3, 1}};
// The same representatives for pairs 2g and 2g+1 side by side, as float32
// lane pairs with their negations: rx, -rx, ry, -ry.
#define LBM_REP_X2(g)                                                                          \
  {(float)rep_x(2 * (g)), (float)rep_x(2 * (g) + 1), (float)-rep_x(2 * (g)), (float)-rep_x(2 * (g) + 1), \
   (float)rep_y(2 * (g)), (float)rep_y(2 * (g) + 1), (float)-rep_y(2 * (g)), (float)-rep_y(2 * (g) + 1)}
static __constant__ float c_pair_rep_x2[NPAIR / 2][8] = {LBM_REP_X2(0), LBM_REP_X2(1), LBM_REP_X2(2),
                                                         LBM_REP_X2(3), LBM_REP_X2(4), LBM_REP_X2(5),
                                                         LBM_REP_X2(6), LBM_REP_X2(7), LBM_REP_X2(8)};
#undef LBM_REP_X2
// first pair of shell j (j = 1..7), and one past the last
__host__ __device__ constexpr int shell_first_pair(int j) {
  return j == 1 ? 0 : j == 2 ? 2 : j == 3 ? 4 : j == 4 ? 6 : j == 5 ? 10 : j == 6 ? 12 : j == 7 ? 14 : 18;
}

#ifndef LBM_DF_GROUP_UNROLL
#define LBM_DF_GROUP_UNROLL 2  // unrolling of the double-float collide's loop over a shell's pair groups
#endif
constexpr int kDfGroupUnroll = LBM_DF_GROUP_UNROLL;

// BGK collide on float64 populations, balancing the FP64 and FP32 pipes
// (GB300 issues FP64 at 1/64 of the FP32 rate).  The moment sums, 1/rho, u and
// T are float64 exactly as in collide_fp64; the temperature-dependent
// coefficients and the per-population equilibrium polynomial run in
// double-float (about 48 significant bits) on the FP32 pipe; the relaxation is
// one float64 FMA, f <- (1 - omega) f + f^eq, with f^eq recombined from its two
// words by one float64 add.  The populations wait in shared memory for the
// relaxation.  The loop over a shell's pair groups (one or two) carries an
// unroll count of two: 4075 MLUPS against 3890 rolled and 3493 with a plain
// full-unroll pragma, as measured.  The results are written to dst directly.
template <int NT>
__device__ __forceinline__ void collide_fp64_df(double (&f)[NPOP], const LatticeArgs& a, double (*s_f)[NT],
                                                int tid, double* __restrict__ dst, int x, int y) {
  const Moments mo = site_moments([&](int l) { return f[l]; });
  const SiteFields sf = site_fields(mo, a);
#pragma unroll
  for (int l = 1; l < NPOP; ++l) s_f[l][tid] = f[l];
  const DF rho = df_from_double_bits(sf.rho);
  const DF ux = df_from_double_bits(sf.ux), uy = df_from_double_bits(sf.uy);
  const DF T = df_from_double_bits(sf.T);
  const DF theta = df_add(T, dfc(a.df_tshift));
  const DF uys = df_sub(uy, dfc(a.df_taug_r));
  const DF U2 = df_mul(df_add(df_mul(ux, ux), df_mul(uys, uys)), dfc(a.df_r2));
  const DF v_x = df_mul(ux, dfc(a.df_r2)), v_y = df_mul(uys, dfc(a.df_r2));
  const DF th2 = df_mul(theta, theta);
  const DF B20 = df_add(df_add(df_mul(U2, -0.25f), df_mul(theta, -1.5f)), 0.5f);
  const DF B21 = df_scale2(theta, 0.25f);
  const DF B10 = df_add(df_add(df_scale2(U2, -0.5f), df_scale2(theta, -2.0f)), 1.0f);
  const DF B11 = df_scale2(theta, 0.5f);
  const DF B00 = df_add(df_add(df_mul(U2, df_add(df_scale2(U2, 0.125f), -0.5f)),
                               df_mul(theta, df_add(df_add(U2, -1.0f), theta))), 1.0f);
  const DF B01 = df_mul(theta, df_sub(df_add(df_scale2(U2, -0.25f), 0.5f), theta));
  const DF B02 = df_scale2(th2, 0.125f);
  const DF wr = df_mul(rho, dfc(a.df_omega));
  dst[sidx(a, 0, y, x)] = fma(a.omc, f[0], df_to_double_bits(df_mul(df_mul(wr, dfc(a.df_w_shell[0])), B00)));
  const DF2 VX = df2_bcast(v_x), VY = df2_bcast(v_y);
  const DF2 C24 = df2_bcast(DF{0x1.555556p-5f, -0x1.555556p-30f}), C6 = df2_bcast(DF{0x1.555556p-3f, -0x1.555556p-28f});
  const float2 nC24 = f2s(-0x1.555556p-5f), nC6 = f2s(-0x1.555556p-3f);  // 1/24, 1/6
#pragma unroll
  for (int j = 1; j < NSHELL; ++j) {
    // Every sum below ends up in sc (E +- O) with E = A0 + O(cu^2) and
    // A0 = B00 + ... ~ 1, so what matters is each sum's absolute error
    // against that O(1) scale, not its relative error: the 11-operation
    // double-word addition (error a few u^2 of |x| + |y|) suffices.
    const DF c2 = dfc(a.df_c2_shell[j]);
    const DF A0 = df_add_fast(df_mul(df_add_fast(df_mul(B02, c2), B01), c2), B00);
    const DF A1 = df_add_fast(df_mul(B11, c2), B10);
    const DF A2 = df_add_fast(df_mul(B21, c2), B20);
    const DF sc = df_mul(wr, dfc(a.df_w_shell[j]));
    const DF2 A0v = df2_bcast(A0), A1v = df2_bcast(A1), A2v = df2_bcast(A2), scv = df2_bcast(sc);
    const float2 nsc = f2s(-sc.hi);
    // two pairs of the shell per iteration, one in each lane (every shell
    // holds an even number of pairs)
#pragma unroll kDfGroupUnroll
    for (int g = shell_first_pair(j) / 2; g < shell_first_pair(j + 1) / 2; ++g) {
      const float2 rx = f2(c_pair_rep_x2[g][0], c_pair_rep_x2[g][1]);
      const float2 nrx = f2(c_pair_rep_x2[g][2], c_pair_rep_x2[g][3]);
      const float2 ry = f2(c_pair_rep_x2[g][4], c_pair_rep_x2[g][5]);
      const float2 nry = f2(c_pair_rep_x2[g][6], c_pair_rep_x2[g][7]);
      const DF2 cu = df2_add_fast(df2_mul_f(VX, rx, nrx), df2_mul_f(VY, ry, nry));
      const float2 ncu = df2_neg_hi(cu);
      const DF2 cu2 = df2_mul_ny(cu, cu, ncu);
      const DF2 E1 = df2_add_fast(df2_mul_ny(cu2, C24, nC24), A2v);
      const DF2 E = df2_add_fast(df2_mul_ny(E1, cu2, df2_neg_hi(cu2)), A0v);
      const DF2 O = df2_mul_ny(df2_add_fast(df2_mul_ny(cu2, C6, nC6), A1v), cu, ncu);
      const DF2 sE = df2_mul_nx(scv, E, nsc), sO = df2_mul_nx(scv, O, nsc);
      const DF2 fp = df2_add_fast(sE, sO), fm = df2_sub_fast(sE, sO);  // sc (E + O), sc (E - O)
      const int lp = 4 * g + 1;  // populations 4g+1, 4g+2 (pair 2g) and 4g+3, 4g+4 (pair 2g+1)
      dst[sidx(a, lp, y, x)] = fma(a.omc, s_f[lp][tid], df_to_double_bits(df2_lane0(fp)));
      dst[sidx(a, lp + 1, y, x)] = fma(a.omc, s_f[lp + 1][tid], df_to_double_bits(df2_lane0(fm)));
      dst[sidx(a, lp + 2, y, x)] = fma(a.omc, s_f[lp + 2][tid], df_to_double_bits(df2_lane1(fp)));
      dst[sidx(a, lp + 3, y, x)] = fma(a.omc, s_f[lp + 3][tid], df_to_double_bits(df2_lane1(fm)));
    }
  }
}

__host__ __device__ constexpr int cpow(int v, int e) { return e == 0 ? 1 : v * cpow(v, e - 1); }

// Monomial moments N (order N00 N20 N02 N40 N22 N04 N10 N30 N12 N01 N03 N21 N11 N31 N13).
__device__ __forceinline__ void reg_moments_f64(const double (&f)[NPOP], double (&N)[15]) {
  double s[NPAIR], d[NPAIR];
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    s[k] = f[2 * k + 1] + f[2 * k + 2];
    d[k] = f[2 * k + 1] - f[2 * k + 2];
  }
  // monomial moments: even total degree from s, odd from d; the rest
  // population only enters N_00
  auto Nm = [&](int c, int e) -> double {
    const bool odd = ((c + e) & 1) != 0;
    double acc = (c == 0 && e == 0) ? f[0] : -0.0;
#pragma unroll
    for (int k = 0; k < NPAIR; ++k) {
      const int coef = cpow(rep_x(k), c) * cpow(rep_y(k), e);
      if (coef != 0) acc = fma((double)coef, odd ? d[k] : s[k], acc);
    }
    return acc;
  };
  const double N00 = Nm(0, 0), N20 = Nm(2, 0), N02 = Nm(0, 2), N40 = Nm(4, 0), N22 = Nm(2, 2), N04 = Nm(0, 4);
  const double N10 = Nm(1, 0), N30 = Nm(3, 0), N12 = Nm(1, 2);
  const double N01 = Nm(0, 1), N03 = Nm(0, 3), N21 = Nm(2, 1);
  const double N11 = Nm(1, 1), N31 = Nm(3, 1), N13 = Nm(1, 3);
  N[0] = N00; N[1] = N20; N[2] = N02; N[3] = N40; N[4] = N22; N[5] = N04;
  N[6] = N10; N[7] = N30; N[8] = N12; N[9] = N01; N[10] = N03; N[11] = N21;
  N[12] = N11; N[13] = N31; N[14] = N13;
}

// 1 / x by one third-order Newton-Raphson correction of a float32 seed
// (float64 FP-pipe work: three FMAs).  The seed y0 comes from x's top 23
// significand bits (integer operations), the approximate float32 reciprocal
// and an exact widening of its bits; with e = 1 - x y0 (|e| < 2^-21) the
// correction y0 (1 + e + e^2) = (1 - e^3) / x leaves a relative error below
// 2^-62 before the last rounding.  x outside [2^-125, 2^126) (zero,
// subnormals, infinities, NaN included) gives NaN.
__device__ __forceinline__ double rcp_nr(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int ex = (int)((hi >> 20) & 0x7ffu) - 1023;
  const unsigned xf = (hi & 0x80000000u) | ((unsigned)(ex + 127) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(xf)));
  const unsigned rb = __float_as_uint(rf);
  const unsigned yhi = (rb & 0x80000000u) | ((((rb >> 23) & 0xffu) + (1023u - 127u)) << 20) | ((rb & 0x7fffffu) >> 3);
  const double y0 = __hiloint2double((int)yhi, (int)(rb << 29));
  const double e = fma(-x, y0, 1.0);
  const double y = fma(y0, fma(e, e, e), y0);
  return (ex >= -125 && ex < 126) ? y : __longlong_as_double(0x7ff8000000000000LL);
}

// Coefficients P of the equilibrium polynomial (4th-order Hermite, with the
// gravity shift) in the integer-velocity monomials of degree <= 4:
// f^eq_l = w_l rho P(xi_l), P(xi) = sum_i P_i xi_x^(c_i) xi_y^(e_i), in the
// order of N (expanded from cu = xi . v and c2 = r^2 |xi|^2), straight from
// the moment sums (rho, J and E / 2) with the site fields folded in, and with
// P[12] halved (poly_to_fix<true> doubles it).  With s = r^2 / rho the
// shifted velocity is v = (J_x s, J_y s - r^2 tau g / r) = r^2 (u - (0,
// tau g / r)), and
//   theta = T + tshift,  T = (r^2 / 2) (E / rho - |u|^2),
//   (r^2 / 2) |u|^2 = U2 / 2 + (tau g / r) v_y + (r^2 / 2) (tau g / r)^2,
// so theta = (E / 2) s - U2 / 2 - (tau g / r) v_y + tshift_v, where the
// lattice constant tshift_v = tshift - (r^2 / 2) (tau g / r)^2.  Products
// of the theta multiples: theta^2 r^4 / 8 = t2 t4 and theta^2 r^4 / 4 = t2^2.
struct EqSite {
  double vx, vy, theta;  // r^2 u_x, r^2 (u_y - tau g / r), T + tshift
};

// VIA_V2: U2 enters only through multiples of v2 = |v|^2 (one product fewer;
// measured faster in the regularised collide, 0.3 % slower in the BGK step).
template <bool VIA_V2 = false>
__device__ __forceinline__ EqSite eq_monomials_moments(const Moments& mh, const LatticeArgs& a, double (&P)[15]) {
  const double s = a.r2 * rcp_nr(mh.rho);
  const double vx_ = mh.Jx * s, vy_ = fma(mh.Jy, s, -a.r2_tau_g_xi);
  const double vx2 = vx_ * vx_, vy2 = vy_ * vy_, vxy = vx_ * vy_;
  const double v2 = vx2 + vy2;
  double theta, h, h2, U2m1;  // h2 = 2 h exactly; U2m1 = U2 - 1
  if constexpr (VIA_V2) {
    theta = fma(mh.Exi, s, fma(-a.half_inv_r2, v2, fma(-a.tau_g_xi, vy_, a.tshift_v)));
    h = fma(-a.quarter_inv_r2, v2, 0.5);
    h2 = fma(-a.half_inv_r2, v2, 1.0);
    U2m1 = fma(a.inv_r2, v2, -1.0);
  } else {
    const double U2 = v2 * a.inv_r2;
    theta = fma(mh.Exi, s, fma(-0.5, U2, fma(-a.tau_g_xi, vy_, a.tshift_v)));
    h = fma(-0.25, U2, 0.5);
    h2 = fma(-0.5, U2, 1.0);
    U2m1 = U2 - 1.0;
  }
  const double B20 = fma(-1.5, theta, h);
  const double B10 = fma(-2.0, theta, h2);  // = 2 (h - theta), rounded once
  // 1 - U2 / 2 + U2^2 / 8 = 2 h^2 + 1/2
  const double B00 = fma(theta, U2m1 + theta, fma(h2, h, 0.5));
  const double t4 = theta * a.r2_4, t2 = theta * a.r2_2;
  const double B01r2 = t2 * B10;  // theta r^2 (h - theta)
  const double q8 = t2 * t4, q4 = t2 * t2;
  const double I = fma(vx2, 1.0 / 6.0, t2), J = fma(vy2, 1.0 / 6.0, t2);
  P[0] = B00;
  P[1] = fma(B20, vx2, B01r2);
  P[2] = fma(B20, vy2, B01r2);
  P[3] = fma(vx2, fma(vx2, 1.0 / 24.0, t4), q8);
  P[4] = fma(t4, v2, fma(0.25 * vxy, vxy, q4));
  P[5] = fma(vy2, fma(vy2, 1.0 / 24.0, t4), q8);
  P[6] = B10 * vx_;
  P[7] = vx_ * I;
  P[8] = vx_ * fma(0.5, vy2, t2);
  P[9] = B10 * vy_;
  P[10] = vy_ * J;
  P[11] = vy_ * fma(0.5, vx2, t2);
  P[12] = B20 * vxy;  // half
  P[13] = vxy * I;
  P[14] = vxy * J;
  return EqSite{vx_, vy_, theta};
}

// The regularised collide's coefficients R of the new populations
// f_l = w_l R(xi_l) from the monomial moments N (same order as N).
__device__ __forceinline__ void reg_coefficients(const double (&N)[15], const LatticeArgs& a, double (&Rv)[15]) {
  const double N00 = N[0], N20 = N[1], N02 = N[2], N40 = N[3], N22 = N[4], N04 = N[5];
  const double N10 = N[6], N30 = N[7], N12 = N[8], N01 = N[9], N03 = N[10], N21 = N[11];
  const double N11 = N[12], N31 = N[13], N13 = N[14];
  // the equilibrium's coefficients from rho, J and E / 2 (monomial moments);
  // Pm[12] holds half the xy coefficient
  double Pm[15];
  eq_monomials_moments<true>(Moments{N00, N10, N01, 0.5 * (N20 + N02)}, a, Pm);
  const double P00 = Pm[0], P20 = Pm[1], P02 = Pm[2], P40 = Pm[3], P22 = Pm[4], P04 = Pm[5];
  const double P10 = Pm[6], P30 = Pm[7], P12 = Pm[8], P01 = Pm[9], P03 = Pm[10], P21 = Pm[11];
  const double P11 = Pm[12], P31 = Pm[13], P13 = Pm[14];
  // relaxed projection coefficients (1 - omega) q = (1 - omega) G^-1 N, block
  // by block (the lattice constants hold (1 - omega) G^-1)
  const double* G = a.ginv;
  const double NE[6] = {N00, N20, N02, N40, N22, N04};
  double q[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) acc = fma(G[6 * i + j], NE[j], acc);
    q[i] = acc;
  }
  auto blk3 = [&](int off, double n0, double n1, double n2, double (&o)[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) o[i] = fma(G[off + 3 * i], n0, fma(G[off + 3 * i + 1], n1, G[off + 3 * i + 2] * n2));
  };
  double qoe[3], qeo[3], qoo[3];
  blk3(36, N10, N30, N12, qoe);
  blk3(45, N01, N03, N21, qeo);
  blk3(54, N11, N31, N13, qoo);
  // R = omega rho P + (1 - omega) q
  const double wr = a.omega * N00;
  const double R00 = fma(wr, P00, q[0]), R20 = fma(wr, P20, q[1]), R02 = fma(wr, P02, q[2]);
  const double R40 = fma(wr, P40, q[3]), R22 = fma(wr, P22, q[4]), R04 = fma(wr, P04, q[5]);
  const double R10 = fma(wr, P10, qoe[0]), R30 = fma(wr, P30, qoe[1]), R12 = fma(wr, P12, qoe[2]);
  const double R01 = fma(wr, P01, qeo[0]), R03 = fma(wr, P03, qeo[1]), R21 = fma(wr, P21, qeo[2]);
  const double R11 = fma(wr + wr, P11, qoo[0]), R31 = fma(wr, P31, qoo[1]), R13 = fma(wr, P13, qoo[2]);
  Rv[0] = R00; Rv[1] = R20; Rv[2] = R02; Rv[3] = R40; Rv[4] = R22; Rv[5] = R04;
  Rv[6] = R10; Rv[7] = R30; Rv[8] = R12; Rv[9] = R01; Rv[10] = R03; Rv[11] = R21;
  Rv[12] = R11; Rv[13] = R31; Rv[14] = R13;
}

// f_l = w_l R(xi_l) for the coefficient vector R (same order as N).
__device__ __forceinline__ void reg_reconstruct_f64(const double (&Rv)[15], const LatticeArgs& a, double (&f)[NPOP]) {
  const double R00 = Rv[0], R20 = Rv[1], R02 = Rv[2], R40 = Rv[3], R22 = Rv[4], R04 = Rv[5];
  const double R10 = Rv[6], R30 = Rv[7], R12 = Rv[8], R01 = Rv[9], R03 = Rv[10], R21 = Rv[11];
  const double R11 = Rv[12], R31 = Rv[13], R13 = Rv[14];
  f[0] = a.w_shell[0] * R00;
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const int x = rep_x(k), y = rep_y(k);
    double ev = R00;
    if (x) ev = fma((double)(x * x), R20, ev);
    if (y) ev = fma((double)(y * y), R02, ev);
    if (x) ev = fma((double)cpow(x, 4), R40, ev);
    if (x && y) ev = fma((double)(x * x * y * y), R22, ev);
    if (y) ev = fma((double)cpow(y, 4), R04, ev);
    if (x && y) ev = fma((double)(x * y), R11, ev);
    if (x && y) ev = fma((double)(cpow(x, 3) * y), R31, ev);
    if (x && y) ev = fma((double)(x * cpow(y, 3)), R13, ev);
    double od = -0.0;
    if (x) od = fma((double)x, R10, od);
    if (y) od = fma((double)y, R01, od);
    if (x) od = fma((double)cpow(x, 3), R30, od);
    if (x && y) od = fma((double)(x * y * y), R12, od);
    if (y) od = fma((double)cpow(y, 3), R03, od);
    if (x && y) od = fma((double)(x * x * y), R21, od);
    const double w = a.w_shell[pair_shell(k)];
    const double wod = w * od;
    f[2 * k + 1] = fma(w, ev, wod);
    f[2 * k + 2] = fma(w, ev, -wod);
  }
}

// Regularised BGK collide in float64 (the Hermite projection of Sect. 2):
//   f <- f^eq + (1 - omega) Pi(f - f^eq) = omega f^eq + (1 - omega) Pi f,
// Pi the w-weighted projection onto the polynomials of degree <= 4 in the
// velocity, which contain the equilibrium.  In integer-velocity monomials,
// Pi f = w (sum_cd q_cd xi_x^c xi_y^d) with q = G^-1 N, N_cd = sum_l f_l
// xi_x^c xi_y^d and G the (block-diagonal) Gram matrix of the monomials; the
// new populations are w_l R(xi_l) with R = omega rho P + (1 - omega) q, P the
// equilibrium polynomial expanded in the same monomials.
// This is the float64 evaluation; collide_fp64_reg_grouped below forms the
// integer-weighted sums in fixed point.
__device__ __forceinline__ void collide_fp64_reg(double (&f)[NPOP], const LatticeArgs& a) {
  double N[15], Rv[15];
  reg_moments_f64(f, N);
  reg_coefficients(N, a, Rv);
  reg_reconstruct_f64(Rv, a, f);
}

// The regularised collide with its integer-weighted sums grouped.  The 18
// +- pairs fall into x-axis pairs (a, 0), y-axis pairs (0, b) and six groups
// {(a, b), (-a, b)}.  A monomial xi_x^c xi_y^e takes the same value on both
// members of a +- pair up to the sign (-1)^(c+e), and on the two pairs of a
// group up to the sign (-1)^c, so every moment N_ce is a short integer
// combination of the pair sums s and differences d and of the group sums and
// differences of those; in the reconstruction, likewise, the even and odd
// parts of R(xi) for the four populations of a group come from four partial
// sums.  Every sum is exact in fixed point (rounded once to float64), so the
// grouping changes the operation count (about half that of summing monomial
// by monomial), not the result.
struct RegAcc {
  Fix96 S[4], T[4], U[4], V[4], Y, N22, N11, N31, N13, N21, N12;
};

// k x for a small positive integer k (a constant after inlining).
__device__ __forceinline__ Fix96 fix_scale(Fix96 x, int k) {
  return k == 1 ? x : fix_mad(Fix96{0u, 0u, 0u}, x, (unsigned)k);
}

// acc + k x, or k x alone where acc has not been set yet (FIRST).
template <bool FIRST>
__device__ __forceinline__ Fix96 fix_acc(Fix96 acc, Fix96 x, int k) {
  return FIRST ? fix_scale(x, k) : fix_axpy(acc, x, k);
}

// Group {(A, B), (-A, B)}: pairs kp (A, B) and km (-A, B).  The axis pairs
// (A, 0) and (0, B) come first, so S, T, U, V are already set; FIRST marks
// the group (1, 1) that opens the six mixed moments.
template <int A, int B, bool FIRST, typename FX>
__device__ __forceinline__ void reg_acc_diag(RegAcc& m, const FX& fx, int kp, int km) {
  const Fix96 pp = fx(2 * kp + 1), pm = fx(2 * kp + 2);
  const Fix96 mp = fx(2 * km + 1), mm = fx(2 * km + 2);
  const Fix96 sp = fix_add(pp, pm), sm = fix_add(mp, mm), dp = fix_sub(pp, pm), dm = fix_sub(mp, mm);
  const Fix96 Gs = fix_add(sp, sm), Hs = fix_sub(sp, sm), Gd = fix_add(dp, dm), Hd = fix_sub(dp, dm);
  m.S[A] = fix_add(m.S[A], Gs);
  m.T[B] = fix_add(m.T[B], Gs);
  m.N22 = fix_acc<FIRST>(m.N22, Gs, A * A * B * B);
  m.N11 = fix_acc<FIRST>(m.N11, Hs, A * B);
  m.N31 = fix_acc<FIRST>(m.N31, Hs, A * A * A * B);
  m.N13 = fix_acc<FIRST>(m.N13, Hs, A * B * B * B);
  m.V[B] = fix_add(m.V[B], Gd);
  m.N21 = fix_acc<FIRST>(m.N21, Gd, A * A * B);
  m.U[A] = fix_add(m.U[A], Hd);
  m.N12 = fix_acc<FIRST>(m.N12, Hd, A * B * B);
}

// Pair (A, 0): opens S[A] and U[A].
template <int A, typename FX>
__device__ __forceinline__ void reg_acc_axis_x(RegAcc& m, const FX& fx, int k) {
  const Fix96 p = fx(2 * k + 1), q = fx(2 * k + 2);
  m.S[A] = fix_add(p, q);
  m.U[A] = fix_sub(p, q);
}

// Pair (0, B): opens T[B] and V[B] (and Y with B = 1).
template <int B, typename FX>
__device__ __forceinline__ void reg_acc_axis_y(RegAcc& m, const FX& fx, int k) {
  const Fix96 p = fx(2 * k + 1), q = fx(2 * k + 2);
  const Fix96 s = fix_add(p, q);
  m.T[B] = s;
  m.Y = B == 1 ? s : fix_add(m.Y, s);
  m.V[B] = fix_sub(p, q);
}

// The 15 monomial moments n_i = sum_l v_l xi_l^(c_i, e_i) (order of N) of
// the fixed-point values fx(l), l = 0..36, as exact integer sums grouped per
// axis pair and per group {(a, b), (-a, b)}.
template <typename FX>
__device__ __forceinline__ void grouped_moments(const FX& fx, Fix96 (&n)[15]) {
  RegAcc m;
  reg_acc_axis_x<1>(m, fx, 0);
  reg_acc_axis_y<1>(m, fx, 1);
  reg_acc_diag<1, 1, true>(m, fx, 2, 3);
  reg_acc_axis_x<2>(m, fx, 4);
  reg_acc_axis_y<2>(m, fx, 5);
  reg_acc_diag<2, 1, false>(m, fx, 6, 9);
  reg_acc_diag<1, 2, false>(m, fx, 7, 8);
  reg_acc_diag<2, 2, false>(m, fx, 10, 11);
  reg_acc_axis_x<3>(m, fx, 12);
  reg_acc_axis_y<3>(m, fx, 13);
  reg_acc_diag<3, 1, false>(m, fx, 14, 17);
  reg_acc_diag<1, 3, false>(m, fx, 15, 16);
  const Fix96 f0 = fx(0);
  n[0] = fix_add(fix_add(f0, fix_add(m.S[1], m.S[2])), fix_add(m.S[3], m.Y));
  n[1] = fix_mad(fix_mad(m.S[1], m.S[2], 4u), m.S[3], 9u);
  n[2] = fix_mad(fix_mad(m.T[1], m.T[2], 4u), m.T[3], 9u);
  n[3] = fix_mad(fix_mad(m.S[1], m.S[2], 16u), m.S[3], 81u);
  n[4] = m.N22;
  n[5] = fix_mad(fix_mad(m.T[1], m.T[2], 16u), m.T[3], 81u);
  n[6] = fix_mad(fix_mad(m.U[1], m.U[2], 2u), m.U[3], 3u);
  n[7] = fix_mad(fix_mad(m.U[1], m.U[2], 8u), m.U[3], 27u);
  n[8] = m.N12;
  n[9] = fix_mad(fix_mad(m.V[1], m.V[2], 2u), m.V[3], 3u);
  n[10] = fix_mad(fix_mad(m.V[1], m.V[2], 8u), m.V[3], 27u);
  n[11] = m.N21;
  n[12] = m.N11;
  n[13] = m.N31;
  n[14] = m.N13;
}

// Fixed-point coefficients X of a polynomial in the monomials (order of N:
// 00 20 02 40 22 04 10 30 12 01 03 21 11 31 13).  A monomial of degree n is at
// most 3^n in magnitude at the 37 velocities, so with |X| below 2^10, 2^8,
// 2^6, 2^4 and 2^2 for degrees 0 to 4 every value of the polynomial, and so
// every sum poly_eval_grouped rounds, stays below 2^13 (7636 at most), inside
// the format; `ok` is cleared otherwise.  HALF12: c[12] holds half the
// coefficient of xi_x xi_y, doubled here exactly on the integer pipe.
template <bool HALF12 = false>
__device__ __forceinline__ void poly_to_fix(const double (&c)[15], Fix96 (&X)[15], bool& ok) {
  constexpr int E0 = kFixE0 + 39, E1 = kFixE0 + 37, E2 = kFixE0 + 35, E3 = kFixE0 + 33, E4 = kFixE0 + 31;
  X[0] = to_fix_upto<E0>(c[0], ok);
  X[1] = to_fix_upto<E2>(c[1], ok);
  X[2] = to_fix_upto<E2>(c[2], ok);
  X[3] = to_fix_upto<E4>(c[3], ok);
  X[4] = to_fix_upto<E4>(c[4], ok);
  X[5] = to_fix_upto<E4>(c[5], ok);
  X[6] = to_fix_upto<E1>(c[6], ok);
  X[7] = to_fix_upto<E3>(c[7], ok);
  X[8] = to_fix_upto<E3>(c[8], ok);
  X[9] = to_fix_upto<E1>(c[9], ok);
  X[10] = to_fix_upto<E3>(c[10], ok);
  X[11] = to_fix_upto<E3>(c[11], ok);
  if constexpr (HALF12) {
    const Fix96 h = to_fix_upto<E2 - 1>(c[12], ok);
    X[12] = fix_add(h, h);
  } else {
    X[12] = to_fix_upto<E2>(c[12], ok);
  }
  X[13] = to_fix_upto<E4>(c[13], ok);
  X[14] = to_fix_upto<E4>(c[14], ok);
}

// The polynomial with coefficients X at the 36 moving velocities, grouped
// like the moments: for pair k, emit(k, ev, od) receives the even part ev and
// the odd part od of the polynomial at +R_k (at -R_k it is ev - od).
template <typename Emit>
__device__ __forceinline__ void poly_eval_grouped(const Fix96 (&X)[15], Emit&& emit) {
  auto axis_x = [&](int k, int c) {  // pair (c, 0)
    const Fix96 ev = fix_axpy(fix_axpy(X[0], X[1], c * c), X[3], c * c * c * c);
    const Fix96 od = fix_axpy(fix_scale(X[6], c), X[7], c * c * c);
    emit(k, ev, od);
  };
  auto axis_y = [&](int k, int c) {  // pair (0, c)
    const Fix96 ev = fix_axpy(fix_axpy(X[0], X[2], c * c), X[5], c * c * c * c);
    const Fix96 od = fix_axpy(fix_scale(X[9], c), X[10], c * c * c);
    emit(k, ev, od);
  };
  auto diag = [&](int kp, int km, int A, int B) {  // pairs (A, B) and (-A, B)
    const Fix96 Ae = fix_axpy(fix_axpy(fix_axpy(fix_axpy(fix_axpy(X[0], X[1], A * A), X[2], B * B), X[3], A * A * A * A),
                                       X[4], A * A * B * B),
                              X[5], B * B * B * B);
    const Fix96 Bo = fix_axpy(fix_axpy(fix_scale(X[12], A * B), X[13], A * A * A * B), X[14], A * B * B * B);
    const Fix96 Co = fix_axpy(fix_axpy(fix_scale(X[6], A), X[7], A * A * A), X[8], A * B * B);
    const Fix96 Do = fix_axpy(fix_axpy(fix_scale(X[9], B), X[10], B * B * B), X[11], A * A * B);
    emit(kp, fix_add(Ae, Bo), fix_add(Co, Do));
    emit(km, fix_sub(Ae, Bo), fix_sub(Do, Co));
  };
  axis_x(0, 1);
  axis_y(1, 1);
  diag(2, 3, 1, 1);
  axis_x(4, 2);
  axis_y(5, 2);
  diag(6, 9, 2, 1);
  diag(7, 8, 1, 2);
  diag(10, 11, 2, 2);
  axis_x(12, 3);
  axis_y(13, 3);
  diag(14, 17, 3, 1);
  diag(15, 16, 1, 3);
}

// Populations of pair k from the even part ev and odd part od of R(xi).
__device__ __forceinline__ void reg_store_pair(double* __restrict__ dst, const LatticeArgs& a, int k, Fix96 ev,
                                               Fix96 od, int x, int y) {
  const double w = a.w_shell[pair_shell(k)];
  dst[sidx(a, 2 * k + 1, y, x)] = w * fix_to_double(fix_add(ev, od));
  dst[sidx(a, 2 * k + 2, y, x)] = w * fix_to_double(fix_sub(ev, od));
}

// The populations are staged in shared memory (s_f[l][tid]) so that the
// accumulators, not 37 float64 values, hold the registers; sites with a
// population or a coefficient outside the fixed-point range take
// collide_fp64_reg.
template <int NT>
__device__ __forceinline__ void collide_fp64_reg_grouped(const double (&f_in)[NPOP], const LatticeArgs& a,
                                                         double (*s_f)[NT], int tid, double* __restrict__ dst,
                                                         int x, int y) {
#pragma unroll
  for (int l = 0; l < NPOP; ++l) s_f[l][tid] = f_in[l];
  const auto f = [&](int l) { return s_f[l][tid]; };
  bool ok = true;
  double N[15];
  {
    Fix96 n[15];
    grouped_moments([&](int l) { return to_fix(f(l), ok); }, n);
#pragma unroll
    for (int i = 0; i < 15; ++i) N[i] = fix_to_double(n[i]);
  }
  double Rv[15];
  if (ok) reg_coefficients(N, a, Rv);
  Fix96 X[15];
  if (ok) poly_to_fix(Rv, X, ok);
  if (!ok) {  // float64 path for this site
    double g[NPOP];
#pragma unroll
    for (int l = 0; l < NPOP; ++l) g[l] = f(l);
    collide_fp64_reg(g, a);
#pragma unroll
    for (int l = 0; l < NPOP; ++l) dst[sidx(a, l, y, x)] = g[l];
    return;
  }
  dst[sidx(a, 0, y, x)] = a.w_shell[0] * Rv[0];
  poly_eval_grouped(X, [&](int k, Fix96 ev, Fix96 od) { reg_store_pair(dst, a, k, ev, od, x, y); });
}

// BGK collide (eq. 1) with the equilibrium evaluated on the integer pipe:
//   f_l <- (1 - omega) f_l + (omega rho w_l) P(xi_l),
// P the equilibrium polynomial of eq_monomials (the one collide_fp64
// evaluates population by population in float64).  The moments are the exact
// fixed-point sums of site_moments; P(xi_l) is an exact fixed-point sum of its
// 15 coefficients with integer weights, rounded once; float64 does the site
// fields, the coefficients, the eight shell factors rho (omega w_j) and one
// multiply and one fused multiply-add per population.  The populations wait in
// shared memory (s_f[l][tid]) for the relaxation.  Sites with a coefficient
// outside poly_to_fix's range take collide_fp64.
template <int NT>
__device__ __forceinline__ ObsFields collide_fp64_fix(const double (&f)[NPOP], const LatticeArgs& a,
                                                      double (*s_f)[NT], int tid, double* __restrict__ dst, int x,
                                                      int y) {
  const Moments mh = site_moments<-1>([&](int l) { return f[l]; });  // E / 2
#pragma unroll
  for (int l = 0; l < NPOP; ++l) s_f[l][tid] = f[l];
  double P[15];
  const EqSite q = eq_monomials_moments(mh, a, P);
  bool ok = true;
  Fix96 X[15];
  poly_to_fix<true>(P, X, ok);
  if (!ok) {  // float64 path for this site
    double g[NPOP];
#pragma unroll
    for (int l = 0; l < NPOP; ++l) g[l] = s_f[l][tid];
    const SiteFields sf = collide_fp64(g, a);
#pragma unroll
    for (int l = 0; l < NPOP; ++l) dst[sidx(a, l, y, x)] = g[l];
    return ObsFields{sf.rho, a.r * sf.ux, a.r * sf.uy - 0.5 * a.g, sf.T};
  }
  double sw[NSHELL];  // omega rho w_j
#pragma unroll
  for (int j = 0; j < NSHELL; ++j) sw[j] = mh.rho * a.ow_shell[j];
  dst[sidx(a, 0, y, x)] = fma(a.omc, s_f[0][tid], sw[0] * P[0]);
  poly_eval_grouped(X, [&](int k, Fix96 ev, Fix96 od) {
    const double w = sw[pair_shell(k)];
    dst[sidx(a, 2 * k + 1, y, x)] = fma(a.omc, s_f[2 * k + 1][tid], w * fix_to_double(fix_add(ev, od)));
    dst[sidx(a, 2 * k + 2, y, x)] = fma(a.omc, s_f[2 * k + 2][tid], w * fix_to_double(fix_sub(ev, od)));
  });
  // the fields for the measurement routines (dropped by the plain step):
  // r u_x = v_x / r, r u_y - g / 2 = v_y / r + tau g - g / 2, T = theta - tshift
  return ObsFields{mh.rho, q.vx * a.inv_r, fma(q.vy, a.inv_r, a.uy_obs_shift), q.theta - a.tshift};
}

// Equilibrium f^eq(rho, u, T) (physical u) into 37 float64 values.
__device__ __forceinline__ void equilibrium(double rho, double ux, double uy, double T,
                                            const LatticeArgs& a, double (&f)[NPOP]) {
  const double theta = T - 1.0;
  const double U2 = fma(ux, ux, uy * uy);
  const double v_x = a.r * ux, v_y = a.r * uy;
  const EqCoef B = eq_coef(U2, theta);
  f[0] = (rho * a.w_shell[0]) * B.B00;
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const int j = pair_shell(k);
    const double c2 = a.c2_shell[j];
    const double A0 = fma(c2, fma(c2, B.B02, B.B01), B.B00);
    const double A1 = fma(B.B11, c2, B.B10);
    const double A2 = fma(B.B21, c2, B.B20);
    const double sc = rho * a.w_shell[j];
    const double cu = pair_cu<double>(k, v_x, v_y);
    const double cu2 = cu * cu;
    const double E = fma(cu2, fma(cu2, 1.0 / 24.0, A2), A0);
    const double O = cu * fma(cu2, 1.0 / 6.0, A1);
    f[2 * k + 1] = sc * (E + O);
    f[2 * k + 2] = sc * (E - O);
  }
}

}  // namespace lbm
