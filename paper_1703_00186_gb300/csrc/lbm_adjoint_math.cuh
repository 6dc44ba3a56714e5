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

// Coefficients of Q(xi) = a(c2) + b(c2) cu + c(c2) cu^2 + d cu^3 + e cu^4 in the
// integer-velocity monomials of degree <= 4 (order N00 N20 N02 N40 N22 N04
// N10 N30 N12 N01 N03 N21 N11 N31 N13), with cu = vx xi_x + vy xi_y,
// c2 = r2 |xi|^2, a = a0 + a1 c2 + a2 c2^2, b = b0 + b1 c2, c = c0 + c1 c2.
__device__ __forceinline__ void poly_monomials(double a0, double a1, double a2, double b0, double b1, double c0,
                                               double c1, double d, double e, double vx, double vy, double r2,
                                               double (&Q)[15]) {
  const double vx2 = vx * vx, vy2 = vy * vy, vxy = vx * vy, r4 = r2 * r2;
  Q[0] = a0;
  Q[1] = fma(a1, r2, c0 * vx2);
  Q[2] = fma(a1, r2, c0 * vy2);
  Q[3] = fma(a2, r4, fma(c1 * r2, vx2, e * vx2 * vx2));
  Q[4] = fma(2.0 * a2, r4, fma(c1 * r2, vx2 + vy2, 6.0 * e * vx2 * vy2));
  Q[5] = fma(a2, r4, fma(c1 * r2, vy2, e * vy2 * vy2));
  Q[6] = b0 * vx;
  Q[7] = vx * fma(b1, r2, d * vx2);
  Q[8] = vx * fma(b1, r2, 3.0 * d * vy2);
  Q[9] = b0 * vy;
  Q[10] = vy * fma(b1, r2, d * vy2);
  Q[11] = vy * fma(b1, r2, 3.0 * d * vx2);
  Q[12] = 2.0 * c0 * vxy;
  Q[13] = vxy * fma(2.0 * c1, r2, 4.0 * e * vx2);
  Q[14] = vxy * fma(2.0 * c1, r2, 4.0 * e * vy2);
}

// The cotangent sums of eq_cotangent in monomial form: with the w-weighted
// cotangent moments Lam_i = sum_l w_l lam_l xi_l^(c_i, e_i), every sum is a
// contraction of Lam with the monomial coefficients of the polynomial it sums
// (P, dP/dU2, dP/dtheta, and P_cu times xi_x or xi_y, whose monomials are
// those of P_cu shifted by one degree in x or y).
template <typename GetLam>
__device__ __forceinline__ EqCot eq_cotangent_mono(GetLam lam, double v_x, double v_y, double U2, double theta,
                                                   const LatticeArgs& a) {
  double L[15];
  L[0] = a.w_shell[0] * lam(0);
#pragma unroll
  for (int i = 1; i < 15; ++i) L[i] = 0.0;
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const double lp = lam(2 * k + 1), lm = lam(2 * k + 2);
    const double w = a.w_shell[pair_shell(k)];
    const double ws = w * (lp + lm), wd = w * (lp - lm);
    const int x = rep_x(k), y = rep_y(k);
    // even monomials take the pair sum, odd ones the difference
    L[0] += ws;
    if (x) L[1] = fma((double)(x * x), ws, L[1]);
    if (y) L[2] = fma((double)(y * y), ws, L[2]);
    if (x) L[3] = fma((double)(x * x * x * x), ws, L[3]);
    if (x && y) L[4] = fma((double)(x * x * y * y), ws, L[4]);
    if (y) L[5] = fma((double)(y * y * y * y), ws, L[5]);
    if (x) L[6] = fma((double)x, wd, L[6]);
    if (x) L[7] = fma((double)(x * x * x), wd, L[7]);
    if (x && y) L[8] = fma((double)(x * y * y), wd, L[8]);
    if (y) L[9] = fma((double)y, wd, L[9]);
    if (y) L[10] = fma((double)(y * y * y), wd, L[10]);
    if (x && y) L[11] = fma((double)(x * x * y), wd, L[11]);
    if (x && y) L[12] = fma((double)(x * y), ws, L[12]);
    if (x && y) L[13] = fma((double)(x * x * x * y), ws, L[13]);
    if (x && y) L[14] = fma((double)(x * y * y * y), ws, L[14]);
  }
  const EqCoef B = eq_coef(U2, theta);
  const double r2 = a.r2;
  double P[15], U[15], T[15], C[15];
  poly_monomials(B.B00, B.B01, B.B02, B.B10, B.B11, B.B20, B.B21, 1.0 / 6.0, 1.0 / 24.0, v_x, v_y, r2, P);
  poly_monomials(fma(0.25, U2, theta - 0.5), -0.25 * theta, 0.0, -0.5, 0.0, -0.25, 0.0, 0.0, 0.0, v_x, v_y, r2, U);
  poly_monomials(fma(2.0, theta, U2 - 1.0), fma(-2.0, theta, fma(-0.25, U2, 0.5)), 0.25 * theta, -2.0, 0.5, -1.5,
                 0.25, 0.0, 0.0, v_x, v_y, r2, T);
  // P_cu = A1 + 2 A2 cu + cu^2 / 2 + cu^3 / 6 (degree <= 3)
  poly_monomials(B.B10, B.B11, 0.0, 2.0 * B.B20, 2.0 * B.B21, 0.5, 0.0, 1.0 / 6.0, 0.0, v_x, v_y, r2, C);
  EqCot s;
  s.SP = 0.0;
  s.SU = 0.0;
  s.Sth = 0.0;
#pragma unroll
  for (int i = 0; i < 15; ++i) {
    s.SP = fma(P[i], L[i], s.SP);
    s.SU = fma(U[i], L[i], s.SU);
    s.Sth = fma(T[i], L[i], s.Sth);
  }
  // P_cu xi_x: monomial (c, e) of P_cu lands on (c + 1, e); xi_y: on (c, e + 1)
  s.Scx = fma(C[0], L[6], fma(C[1], L[7], fma(C[2], L[8], fma(C[12], L[11], fma(C[6], L[1],
          fma(C[9], L[12], fma(C[7], L[3], fma(C[10], L[14], fma(C[11], L[13], C[8] * L[4])))))))));
  s.Scy = fma(C[0], L[9], fma(C[1], L[11], fma(C[2], L[10], fma(C[12], L[8], fma(C[6], L[12],
          fma(C[9], L[2], fma(C[7], L[13], fma(C[10], L[5], fma(C[11], L[4], C[8] * L[14])))))))));
  return s;
}

}  // namespace lbm
