// Cotangent sums of the Hermite equilibrium, shared by the adjoint kernels.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Cotangent sums of the equilibrium at one site, for cotangents lam_l on
// f^eq_l = w_l rho P(cu_l, U2, theta):
//   SP = sum lam w P,  Scu = sum lam w P_cu xi,  SU = sum lam w dP/dU2,
//   Sth = sum lam w dP/dtheta.
struct EqCot {
  double SP, Scx, Scy, SU, Sth;
};

template <typename GetLam>
__device__ __forceinline__ EqCot eq_cotangent(GetLam lam, double v_x, double v_y, double U2, double theta,
                                              const LatticeArgs& a) {
  const EqCoef B = eq_coef(U2, theta);
  // d/dU2 and d/dtheta of the shell coefficients A0, A1, A2
  const double dU0 = fma(0.25, U2, theta - 0.5);               // dB00/dU2
  const double dU1 = -0.25 * theta;                             // dB01/dU2
  const double dT0 = fma(2.0, theta, U2 - 1.0);                 // dB00/dtheta
  const double dT1 = fma(-2.0, theta, fma(-0.25, U2, 0.5));     // dB01/dtheta
  const double dT2 = 0.25 * theta;                              // dB02/dtheta
  EqCot s;
  {
    const double l0 = a.w_shell[0] * lam(0);
    s.SP = l0 * B.B00;
    s.SU = l0 * dU0;
    s.Sth = l0 * dT0;
    s.Scx = 0.0;
    s.Scy = 0.0;
  }
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const int j = pair_shell(k);
    const double c2 = a.c2_shell[j];
    const double w = a.w_shell[j];
    const double A0 = fma(c2, fma(c2, B.B02, B.B01), B.B00);
    const double A1 = fma(B.B11, c2, B.B10);
    const double A2 = fma(B.B21, c2, B.B20);
    const double aU = fma(dU1, c2, dU0);                  // dA0/dU2
    const double aT = fma(c2, fma(c2, dT2, dT1), dT0);    // dA0/dtheta
    const double hT = fma(0.5, c2, -2.0);                 // dA1/dtheta
    const double bT = fma(0.25, c2, -1.5);                // dA2/dtheta
    const double lp = lam(2 * k + 1), lm = lam(2 * k + 2);
    const double Ls = w * (lp + lm), La = w * (lp - lm);
    const double cu = pair_cu<double>(k, v_x, v_y);
    const double cu2 = cu * cu;
    const double Pe = fma(cu2, fma(cu2, 1.0 / 24.0, A2), A0);
    const double Po = cu * fma(cu2, 1.0 / 6.0, A1);
    const double Pce = fma(0.5, cu2, A1);
    const double Pco = cu * fma(cu2, 1.0 / 6.0, 2.0 * A2);
    s.SP = fma(Ls, Pe, fma(La, Po, s.SP));
    const double t = fma(La, Pce, Ls * Pco);
    if (rep_x(k) != 0) s.Scx = fma((double)rep_x(k), t, s.Scx);
    if (rep_y(k) != 0) s.Scy = fma((double)rep_y(k), t, s.Scy);
    s.SU = fma(Ls, fma(-0.25, cu2, aU), fma(-0.5 * La, cu, s.SU));
    s.Sth = fma(Ls, fma(bT, cu2, aT), fma(La * hT, cu, s.Sth));
  }
  return s;
}

}  // namespace lbm

namespace lbm {

// The 15 w-weighted cotangent moments Lam_(c,e) = sum_l w_l lam_l xi_lx^c
// xi_ly^e (order N00 N20 N02 N40 N22 N04 N10 N30 N12 N01 N03 N21 N11 N31 N13)
// from group sums: the 18 +- pairs fall into the x-axis pairs (a, 0), the
// y-axis pairs (0, b) and six groups {(a, b), (-a, b)}; within a group a
// monomial sees only the sum G or the difference H of the two pairs' values
// (which one follows from the parities of c and e), and a moment of given
// c and e sums such values with the integer weights a^c b^e.  About 190 float64
// operations per site against 280 for accumulating pair by pair.
template <typename GetLam>
__device__ __forceinline__ void cotangent_moments(GetLam lam, const LatticeArgs& a, double (&L)[15]) {
  const double* w = a.w_shell;
  double S[4], T[4], U[4], V[4];  // per |xi_x| = a (S even, U odd in x), per |xi_y| = b (T even, V odd in y)
  double Y, L4, L8, L11, L12, L13, L14;
  // x-axis pairs (a, 0): k = 0, 4, 12; y-axis pairs (0, b): k = 1, 5, 13
  {
    const int kx[4] = {0, 0, 4, 12}, ky[4] = {0, 1, 5, 13}, jw[4] = {0, 1, 3, 6};
#pragma unroll
    for (int c = 1; c <= 3; ++c) {
      const double px = lam(2 * kx[c] + 1), mx = lam(2 * kx[c] + 2);
      S[c] = w[jw[c]] * (px + mx);
      U[c] = w[jw[c]] * (px - mx);
      const double py = lam(2 * ky[c] + 1), my = lam(2 * ky[c] + 2);
      T[c] = w[jw[c]] * (py + my);
      V[c] = w[jw[c]] * (py - my);
    }
    Y = (T[1] + T[2]) + T[3];
  }
  L4 = L8 = L11 = L12 = L13 = L14 = 0.0;
  // group {(A, B), (-A, B)}: pairs kp = (A, B) and km = (-A, B), shell j
  auto group = [&](int A, int B, int kp, int km, int j) {
    const double pp = lam(2 * kp + 1), pm = lam(2 * kp + 2), mp = lam(2 * km + 1), mm = lam(2 * km + 2);
    const double sp = pp + pm, sm = mp + mm, dp = pp - pm, dm = mp - mm;
    const double Gs = w[j] * (sp + sm), Hs = w[j] * (sp - sm), Gd = w[j] * (dp + dm), Hd = w[j] * (dp - dm);
    S[A] += Gs;
    T[B] += Gs;
    U[A] += Hd;
    V[B] += Gd;
    L4 = fma((double)(A * A * B * B), Gs, L4);
    L12 = fma((double)(A * B), Hs, L12);
    L13 = fma((double)(A * A * A * B), Hs, L13);
    L14 = fma((double)(A * B * B * B), Hs, L14);
    L11 = fma((double)(A * A * B), Gd, L11);
    L8 = fma((double)(A * B * B), Hd, L8);
  };
  group(1, 1, 2, 3, 2);
  group(2, 1, 6, 9, 4);
  group(1, 2, 7, 8, 4);
  group(2, 2, 10, 11, 5);
  group(3, 1, 14, 17, 7);
  group(1, 3, 15, 16, 7);
  L[0] = fma(w[0], lam(0), ((S[1] + S[2]) + S[3]) + Y);
  L[1] = fma(9.0, S[3], fma(4.0, S[2], S[1]));
  L[2] = fma(9.0, T[3], fma(4.0, T[2], T[1]));
  L[3] = fma(81.0, S[3], fma(16.0, S[2], S[1]));
  L[4] = L4;
  L[5] = fma(81.0, T[3], fma(16.0, T[2], T[1]));
  L[6] = fma(3.0, U[3], fma(2.0, U[2], U[1]));
  L[7] = fma(27.0, U[3], fma(8.0, U[2], U[1]));
  L[8] = L8;
  L[9] = fma(3.0, V[3], fma(2.0, V[2], V[1]));
  L[10] = fma(27.0, V[3], fma(8.0, V[2], V[1]));
  L[11] = L11;
  L[12] = L12;
  L[13] = L13;
  L[14] = L14;
}

// The same 15 cotangent moments as exact fixed-point sums: the products
// w_l lam_l (37 float64 multiplies) are put on the fixed-point grid with one
// exponent D for the site, summed exactly with integer weights
// (grouped_moments) and rounded once each.  D comes from a bound on the
// largest product's exponent (that of lam_l plus that of w_l, plus one), so
// the products are formed once, as the sums consume them.  Returns false,
// having written nothing, where that bound leaves the range in which the
// rounded sums are normal float64 numbers (products of 2^1010 and above,
// nonzero products all below 2^-938, infinities, NaNs); the caller then takes
// cotangent_moments.
template <typename GetLam>
__device__ __forceinline__ bool cotangent_moments_fix(GetLam lam, const LatticeArgs& a, double (&L)[15]) {
  int ew[NSHELL];
#pragma unroll
  for (int j = 0; j < NSHELL; ++j) ew[j] = exp_field(a.w_shell[j]) - 1022;
  int elam = exp_field(lam(0)), E = elam + ew[0];
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const int ep = exp_field(lam(2 * k + 1)), em = exp_field(lam(2 * k + 2));
    elam = max(elam, max(ep, em));
    E = max(E, max(ep, em) + ew[pair_shell(k)]);
  }
  if (elam != 0 && (E < 84 || E > 2034)) return false;
  const int D = elam != 0 ? E - kFixEMax : 0;  // every |w lam| 2^-D < 4
  Fix96 n[15];
  grouped_moments(
      [&](int l) { return to_fix_scaled(a.w_shell[l == 0 ? 0 : pair_shell((l - 1) >> 1)] * lam(l), D); }, n);
#pragma unroll
  for (int i = 0; i < 15; ++i) L[i] = fix_to_double_scaled(n[i], D);
  return true;
}

// Site quantities of the float64 adjoint, straight from the moment sums
// (rho, J and E / 2) as in the forward step's coefficients: with
// s = r^2 / rho, v = (J_x s, J_y s - r^2 tau g / r) is the shifted velocity
// (r^2 u' in the lattice's units), vy0 = r^2 u_y the unshifted one,
// v2 = |v|^2 (U2 = v2 / r^2 enters only through multiples), theta =
// T + tshift, h = 1/2 - U2/4 (h2 = 2 h exactly),
// and the theta multiples t2 = theta r^2 / 2 = B11 r^2 = 2 B21 r^2 and
// t4 = theta r^2 / 4 = B21 r^2.
struct AdjSite {
  double v_x, v_y, vy0, vx2, vy2, vxy, v2, theta, h, h2, t2, t4;
};

__device__ __forceinline__ AdjSite adj_site(const Moments& mh, const LatticeArgs& a) {
  AdjSite q;
  const double s = a.r2 * rcp_nr(mh.rho);
  q.v_x = mh.Jx * s;
  q.vy0 = mh.Jy * s;
  q.v_y = q.vy0 - a.r2_tau_g_xi;
  q.vx2 = q.v_x * q.v_x;
  q.vy2 = q.v_y * q.v_y;
  q.vxy = q.v_x * q.v_y;
  q.v2 = q.vx2 + q.vy2;
  q.theta = fma(mh.Exi, s, fma(-a.half_inv_r2, q.v2, fma(-a.tau_g_xi, q.v_y, a.tshift_v)));
  q.h = fma(-a.quarter_inv_r2, q.v2, 0.5);
  q.h2 = fma(-a.half_inv_r2, q.v2, 1.0);
  q.t2 = q.theta * a.r2_2;
  q.t4 = q.theta * a.r2_4;
  return q;
}

// The cotangent sums of eq_cotangent in monomial form: with the w-weighted
// cotangent moments L_i = sum_l w_l lam_l xi_l^(c_i, e_i), every sum is a
// contraction of L with the monomial coefficients of the polynomial it sums
// (P, dP/dU2, dP/dtheta, and P_cu times xi_x or xi_y, whose monomials are
// those of P_cu shifted by one degree in x or y).  The Hermite coefficients
// are folded as in the forward step (B10 = 2 (h - theta), B01 r^2 = t2 B10,
// B02 r^4 = t2 t4); the coefficients of P_cu xi of degree 3 equal those of
// P (C7 = P30, C8 = P12, C10 = P03, C11 = P21, because 2 B21 r^2 = B11 r^2).
__device__ __forceinline__ EqCot eq_cotangent_site(const double (&L)[15], const AdjSite& q, const LatticeArgs& a) {
  const double theta = q.theta, v_x = q.v_x, v_y = q.v_y;
  const double vx2 = q.vx2, vy2 = q.vy2, vxy = q.vxy, t2 = q.t2, t4 = q.t4;
  const double B20 = fma(-1.5, theta, q.h);
  const double B10 = fma(-2.0, theta, q.h2);
  const double B00 = fma(theta, fma(a.inv_r2, q.v2, -1.0) + theta, fma(q.h2, q.h, 0.5));
  const double B01r2 = t2 * B10, q8 = t2 * t4;  // B01 r^2, B02 r^4
  const double I = fma(vx2, 1.0 / 6.0, t2), J = fma(vy2, 1.0 / 6.0, t2);
  const double Hx = fma(0.5, vx2, t2), Hy = fma(0.5, vy2, t2);
  // monomial coefficients of P (P30 P12 P03 P21 double as C7 C8 C10 C11)
  const double P30 = v_x * I, P12 = v_x * Hy, P03 = v_y * J, P21 = v_y * Hx;
  const double B20x2 = B20 + B20;
  EqCot s;
  {  // P = A0 + A1 cu + A2 cu^2 + cu^3 / 6 + cu^4 / 24
    const double P20 = fma(B20, vx2, B01r2), P02 = fma(B20, vy2, B01r2);
    const double P40 = fma(vx2, fma(vx2, 1.0 / 24.0, t4), q8);
    const double P22 = fma(t4, q.v2, fma(0.25 * vxy, vxy, q8 + q8));
    const double P04 = fma(vy2, fma(vy2, 1.0 / 24.0, t4), q8);
    s.SP = fma(B00, L[0], fma(P20, L[1], fma(P02, L[2], fma(P40, L[3], fma(P22, L[4], P04 * L[5])))));
    s.SP = fma(B10, fma(v_x, L[6], v_y * L[9]), s.SP);
    s.SP = fma(P30, L[7], fma(P12, L[8], fma(P03, L[10], fma(P21, L[11], s.SP))));
    s.SP = fma(B20x2 * vxy, L[12], fma(vxy * I, L[13], fma(vxy * J, L[14], s.SP)));
  }
  {  // dP/dU2 = (U2 / 4 + theta - 1/2) - (theta / 4) c2 - cu / 2 - cu^2 / 4
    s.SU = fma(theta - q.h, L[0], fma(fma(-0.25, vx2, -t4), L[1], fma(-0.25, vy2, -t4) * L[2]));
    s.SU = fma(-0.5, fma(v_x, L[6], fma(v_y, L[9], vxy * L[12])), s.SU);
  }
  {  // dP/dtheta = (2 theta + U2 - 1) + (1/2 - 2 theta - U2/4) c2 + (theta / 4) c2^2
     //             + (c2 / 2 - 2) cu + (c2 / 4 - 3/2) cu^2
     // (2 theta + U2 - 1 = U2 / 2 - B10, 1/2 - 2 theta - U2/4 = B10 - h)
    const double a1r2 = (B10 - q.h) * a.r2, a2r4 = theta * a.r4_4;
    s.Sth = fma(fma(a.half_inv_r2, q.v2, -B10), L[0], fma(fma(-1.5, vx2, a1r2), L[1], fma(-1.5, vy2, a1r2) * L[2]));
    s.Sth = fma(fma(a.r2_4, vx2, a2r4), L[3],
                fma(fma(a.r2_4, q.v2, a2r4 + a2r4), L[4], fma(fma(a.r2_4, vy2, a2r4), L[5], s.Sth)));
    s.Sth = fma(-2.0, fma(v_x, L[6], v_y * L[9]), s.Sth);
    s.Sth = fma(a.r2_2, fma(v_x, L[7] + L[8], fma(v_y, L[10] + L[11], vxy * (L[13] + L[14]))),
                fma(-3.0 * vxy, L[12], s.Sth));
  }
  {  // P_cu = A1 + 2 A2 cu + cu^2 / 2 + cu^3 / 6, times xi_x or xi_y
    const double C6 = B20x2 * v_x, C9 = B20x2 * v_y;
    s.Scx = fma(B10, L[6], fma(Hx, L[7], fma(Hy, L[8], fma(vxy, L[11], fma(C6, L[1], fma(C9, L[12],
            fma(P30, L[3], fma(P03, L[14], fma(P21, L[13], P12 * L[4])))))))));
    s.Scy = fma(B10, L[9], fma(Hx, L[11], fma(Hy, L[10], fma(vxy, L[8], fma(C6, L[12], fma(C9, L[2],
            fma(P30, L[13], fma(P03, L[5], fma(P21, L[4], P12 * L[14])))))))));
  }
  return s;
}

}  // namespace lbm
