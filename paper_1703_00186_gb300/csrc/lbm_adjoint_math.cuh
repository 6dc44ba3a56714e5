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

// The cotangent sums of eq_cotangent in monomial form: with the w-weighted
// cotangent moments L_i = sum_l w_l lam_l xi_l^(c_i, e_i), every sum is a
// contraction of Lam with the monomial coefficients of the polynomial it sums
// (P, dP/dU2, dP/dtheta, and P_cu times xi_x or xi_y, whose monomials are
// those of P_cu shifted by one degree in x or y).
__device__ __forceinline__ EqCot eq_cotangent_mono(const double (&L)[15], double v_x, double v_y, double U2,
                                                   double theta, const LatticeArgs& a) {
  const EqCoef B = eq_coef(U2, theta);
  const double r2 = a.r2, r4 = r2 * r2;
  const double vx2 = v_x * v_x, vy2 = v_y * v_y, vxy = v_x * v_y;
  const double B01r2 = B.B01 * r2, B02r4 = B.B02 * r4, B21r2 = B.B21 * r2, B11r2 = B.B11 * r2;
  const double vx2_6 = vx2 * (1.0 / 6.0), vy2_6 = vy2 * (1.0 / 6.0);
  // The monomial coefficients of the four polynomials (P, dP/dU2, dP/dtheta
  // and P_cu expanded from cu = xi . v and c2 = r^2 |xi|^2), written out so
  // that their zero coefficients cost nothing.
  EqCot s;
  {  // P = A0 + A1 cu + A2 cu^2 + cu^3 / 6 + cu^4 / 24
    const double P1 = fma(B.B20, vx2, B01r2), P2 = fma(B.B20, vy2, B01r2);
    const double P3 = fma(B21r2, vx2, fma(vx2 * vx2, 1.0 / 24.0, B02r4));
    const double P4 = fma(B21r2, vx2 + vy2, fma(0.25 * vx2, vy2, 2.0 * B02r4));
    const double P5 = fma(B21r2, vy2, fma(vy2 * vy2, 1.0 / 24.0, B02r4));
    const double P7 = v_x * (B11r2 + vx2_6), P8 = v_x * fma(0.5, vy2, B11r2);
    const double P10 = v_y * (B11r2 + vy2_6), P11 = v_y * fma(0.5, vx2, B11r2);
    const double B21r2x2 = 2.0 * B21r2;
    const double P13 = vxy * (B21r2x2 + vx2_6), P14 = vxy * (B21r2x2 + vy2_6);
    s.SP = fma(B.B00, L[0], fma(P1, L[1], fma(P2, L[2], fma(P3, L[3], fma(P4, L[4], P5 * L[5])))));
    s.SP = fma(B.B10, fma(v_x, L[6], v_y * L[9]), s.SP);
    s.SP = fma(P7, L[7], fma(P8, L[8], fma(P10, L[10], fma(P11, L[11], s.SP))));
    s.SP = fma(2.0 * B.B20 * vxy, L[12], fma(P13, L[13], fma(P14, L[14], s.SP)));
  }
  {  // dP/dU2 = (U2 / 4 + theta - 1/2) - (theta / 4) c2 - cu / 2 - cu^2 / 4
    const double a1r2 = -0.25 * theta * r2;
    s.SU = fma(fma(0.25, U2, theta - 0.5), L[0], fma(fma(-0.25, vx2, a1r2), L[1], fma(-0.25, vy2, a1r2) * L[2]));
    s.SU = fma(-0.5, fma(v_x, L[6], fma(v_y, L[9], vxy * L[12])), s.SU);
  }
  {  // dP/dtheta = (2 theta + U2 - 1) + (1/2 - 2 theta - U2/4) c2 + (theta / 4) c2^2
     //             + (c2 / 2 - 2) cu + (c2 / 4 - 3/2) cu^2
    const double a1r2 = fma(-2.0, theta, fma(-0.25, U2, 0.5)) * r2, a2r4 = 0.25 * theta * r4;
    const double r2q = 0.25 * r2, r2h = 0.5 * r2;
    s.Sth = fma(fma(2.0, theta, U2 - 1.0), L[0], fma(fma(-1.5, vx2, a1r2), L[1], fma(-1.5, vy2, a1r2) * L[2]));
    s.Sth = fma(fma(r2q, vx2, a2r4), L[3], fma(fma(r2q, vx2 + vy2, 2.0 * a2r4), L[4], fma(fma(r2q, vy2, a2r4), L[5], s.Sth)));
    s.Sth = fma(-2.0, fma(v_x, L[6], v_y * L[9]), s.Sth);
    s.Sth = fma(r2h, fma(v_x, L[7] + L[8], fma(v_y, L[10] + L[11], vxy * (L[13] + L[14]))), fma(-3.0 * vxy, L[12], s.Sth));
  }
  {  // P_cu = A1 + 2 A2 cu + cu^2 / 2 + cu^3 / 6, times xi_x or xi_y
    const double C1 = fma(0.5, vx2, B11r2), C2 = fma(0.5, vy2, B11r2);
    const double B20x2 = 2.0 * B.B20, B21r2x2 = 2.0 * B21r2;
    const double C6 = B20x2 * v_x, C9 = B20x2 * v_y;
    const double C7 = v_x * (B21r2x2 + vx2_6), C8 = v_x * fma(0.5, vy2, B21r2x2);
    const double C10 = v_y * (B21r2x2 + vy2_6), C11 = v_y * fma(0.5, vx2, B21r2x2);
    s.Scx = fma(B.B10, L[6], fma(C1, L[7], fma(C2, L[8], fma(vxy, L[11], fma(C6, L[1], fma(C9, L[12],
            fma(C7, L[3], fma(C10, L[14], fma(C11, L[13], C8 * L[4])))))))));
    s.Scy = fma(B.B10, L[9], fma(C1, L[11], fma(C2, L[10], fma(vxy, L[8], fma(C6, L[12], fma(C9, L[2],
            fma(C7, L[13], fma(C10, L[5], fma(C11, L[4], C8 * L[14])))))))));
  }
  return s;
}

}  // namespace lbm
