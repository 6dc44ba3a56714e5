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
