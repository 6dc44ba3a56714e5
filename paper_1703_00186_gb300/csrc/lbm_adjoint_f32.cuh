// Float32 cotangent arithmetic for the adjoint of FP32-store contexts
// (lbm_adjoint_step_f32): the transposed collide Jacobian of lbm_adjoint.cu
// with the cotangents stored as float32 and every cotangent sum in float32 on
// the FP32 pipe.  The forward site fields (rho, u, T of eq. 2) still come from
// exact fixed-point moment sums and float64 site fields, rounded to float32
// once.  The formulas are those of cotangent_moments and eq_cotangent_mono in
// lbm_adjoint_math.cuh; every constant is a float32, so no operation is
// promoted to float64.
#pragma once

#include "lbm_adjoint_math.cuh"

namespace lbm {

struct EqCotF {
  float SP, Scx, Scy, SU, Sth;
};

// The 15 w-weighted cotangent moments L_(c,e) = sum_l w_l lam_l xi_lx^c
// xi_ly^e (order N00 N20 N02 N40 N22 N04 N10 N30 N12 N01 N03 N21 N11 N31 N13)
// from the axis-pair and group {(a, b), (-a, b)} sums, in float32.
__device__ __forceinline__ void cotangent_moments_f(const float (&lam)[NPOP], const LatticeArgs& a,
                                                    float (&L)[15]) {
  const float* w = a.w_shell_f;
  float S[4], T[4], U[4], V[4];
  {
    const int kx[4] = {0, 0, 4, 12}, ky[4] = {0, 1, 5, 13}, jw[4] = {0, 1, 3, 6};
#pragma unroll
    for (int c = 1; c <= 3; ++c) {
      const float px = lam[2 * kx[c] + 1], mx = lam[2 * kx[c] + 2];
      S[c] = w[jw[c]] * (px + mx);
      U[c] = w[jw[c]] * (px - mx);
      const float py = lam[2 * ky[c] + 1], my = lam[2 * ky[c] + 2];
      T[c] = w[jw[c]] * (py + my);
      V[c] = w[jw[c]] * (py - my);
    }
  }
  const float Y = (T[1] + T[2]) + T[3];
  float L4 = 0.f, L8 = 0.f, L11 = 0.f, L12 = 0.f, L13 = 0.f, L14 = 0.f;
  auto group = [&](int A, int B, int kp, int km, int j) {
    const float pp = lam[2 * kp + 1], pm = lam[2 * kp + 2], mp = lam[2 * km + 1], mm = lam[2 * km + 2];
    const float sp = pp + pm, sm = mp + mm, dp = pp - pm, dm = mp - mm;
    const float Gs = w[j] * (sp + sm), Hs = w[j] * (sp - sm), Gd = w[j] * (dp + dm), Hd = w[j] * (dp - dm);
    S[A] += Gs;
    T[B] += Gs;
    U[A] += Hd;
    V[B] += Gd;
    L4 = fmaf((float)(A * A * B * B), Gs, L4);
    L12 = fmaf((float)(A * B), Hs, L12);
    L13 = fmaf((float)(A * A * A * B), Hs, L13);
    L14 = fmaf((float)(A * B * B * B), Hs, L14);
    L11 = fmaf((float)(A * A * B), Gd, L11);
    L8 = fmaf((float)(A * B * B), Hd, L8);
  };
  group(1, 1, 2, 3, 2);
  group(2, 1, 6, 9, 4);
  group(1, 2, 7, 8, 4);
  group(2, 2, 10, 11, 5);
  group(3, 1, 14, 17, 7);
  group(1, 3, 15, 16, 7);
  L[0] = fmaf(w[0], lam[0], ((S[1] + S[2]) + S[3]) + Y);
  L[1] = fmaf(9.f, S[3], fmaf(4.f, S[2], S[1]));
  L[2] = fmaf(9.f, T[3], fmaf(4.f, T[2], T[1]));
  L[3] = fmaf(81.f, S[3], fmaf(16.f, S[2], S[1]));
  L[4] = L4;
  L[5] = fmaf(81.f, T[3], fmaf(16.f, T[2], T[1]));
  L[6] = fmaf(3.f, U[3], fmaf(2.f, U[2], U[1]));
  L[7] = fmaf(27.f, U[3], fmaf(8.f, U[2], U[1]));
  L[8] = L8;
  L[9] = fmaf(3.f, V[3], fmaf(2.f, V[2], V[1]));
  L[10] = fmaf(27.f, V[3], fmaf(8.f, V[2], V[1]));
  L[11] = L11;
  L[12] = L12;
  L[13] = L13;
  L[14] = L14;
}

// eq_cotangent_mono in float32: the cotangent sums of the equilibrium as
// contractions of the moments L with the monomial coefficients of P, dP/dU2,
// dP/dtheta and P_cu (times xi_x or xi_y).
__device__ __forceinline__ EqCotF eq_cotangent_mono_f(const float (&L)[15], float v_x, float v_y, float U2,
                                                      float theta, const LatticeArgs& a) {
  const float B20 = fmaf(-1.5f, theta, fmaf(-0.25f, U2, 0.5f));
  const float B21 = 0.25f * theta;
  const float B10 = fmaf(-2.0f, theta, fmaf(-0.5f, U2, 1.0f));
  const float B11 = 0.5f * theta;
  const float B00 = fmaf(theta, (U2 - 1.0f) + theta, fmaf(U2, fmaf(0.125f, U2, -0.5f), 1.0f));
  const float B01 = theta * (fmaf(-0.25f, U2, 0.5f) - theta);
  const float B02 = 0.125f * (theta * theta);
  const float r2 = a.df_r2[0], r4 = r2 * r2;
  const float vx2 = v_x * v_x, vy2 = v_y * v_y, vxy = v_x * v_y;
  const float B01r2 = B01 * r2, B02r4 = B02 * r4, B21r2 = B21 * r2, B11r2 = B11 * r2;
  const float vx2_6 = vx2 * (1.0f / 6.0f), vy2_6 = vy2 * (1.0f / 6.0f);
  EqCotF s;
  {  // P = A0 + A1 cu + A2 cu^2 + cu^3 / 6 + cu^4 / 24
    const float P1 = fmaf(B20, vx2, B01r2), P2 = fmaf(B20, vy2, B01r2);
    const float P3 = fmaf(B21r2, vx2, fmaf(vx2 * vx2, 1.0f / 24.0f, B02r4));
    const float P4 = fmaf(B21r2, vx2 + vy2, fmaf(0.25f * vx2, vy2, 2.0f * B02r4));
    const float P5 = fmaf(B21r2, vy2, fmaf(vy2 * vy2, 1.0f / 24.0f, B02r4));
    const float P7 = v_x * (B11r2 + vx2_6), P8 = v_x * fmaf(0.5f, vy2, B11r2);
    const float P10 = v_y * (B11r2 + vy2_6), P11 = v_y * fmaf(0.5f, vx2, B11r2);
    const float B21r2x2 = 2.0f * B21r2;
    const float P13 = vxy * (B21r2x2 + vx2_6), P14 = vxy * (B21r2x2 + vy2_6);
    float sp = fmaf(B00, L[0], fmaf(P1, L[1], fmaf(P2, L[2], fmaf(P3, L[3], fmaf(P4, L[4], P5 * L[5])))));
    sp = fmaf(B10, fmaf(v_x, L[6], v_y * L[9]), sp);
    sp = fmaf(P7, L[7], fmaf(P8, L[8], fmaf(P10, L[10], fmaf(P11, L[11], sp))));
    s.SP = fmaf(2.0f * B20 * vxy, L[12], fmaf(P13, L[13], fmaf(P14, L[14], sp)));
  }
  {  // dP/dU2 = (U2 / 4 + theta - 1/2) - (theta / 4) c2 - cu / 2 - cu^2 / 4
    const float a1r2 = -0.25f * theta * r2;
    const float su =
        fmaf(fmaf(0.25f, U2, theta - 0.5f), L[0], fmaf(fmaf(-0.25f, vx2, a1r2), L[1], fmaf(-0.25f, vy2, a1r2) * L[2]));
    s.SU = fmaf(-0.5f, fmaf(v_x, L[6], fmaf(v_y, L[9], vxy * L[12])), su);
  }
  {  // dP/dtheta
    const float a1r2 = fmaf(-2.0f, theta, fmaf(-0.25f, U2, 0.5f)) * r2, a2r4 = 0.25f * theta * r4;
    const float r2q = 0.25f * r2, r2h = 0.5f * r2;
    float st = fmaf(fmaf(2.0f, theta, U2 - 1.0f), L[0], fmaf(fmaf(-1.5f, vx2, a1r2), L[1], fmaf(-1.5f, vy2, a1r2) * L[2]));
    st = fmaf(fmaf(r2q, vx2, a2r4), L[3], fmaf(fmaf(r2q, vx2 + vy2, 2.0f * a2r4), L[4], fmaf(fmaf(r2q, vy2, a2r4), L[5], st)));
    st = fmaf(-2.0f, fmaf(v_x, L[6], v_y * L[9]), st);
    s.Sth = fmaf(r2h, fmaf(v_x, L[7] + L[8], fmaf(v_y, L[10] + L[11], vxy * (L[13] + L[14]))),
                 fmaf(-3.0f * vxy, L[12], st));
  }
  {  // P_cu = A1 + 2 A2 cu + cu^2 / 2 + cu^3 / 6, times xi_x or xi_y
    const float C1 = fmaf(0.5f, vx2, B11r2), C2 = fmaf(0.5f, vy2, B11r2);
    const float B20x2 = 2.0f * B20, B21r2x2 = 2.0f * B21r2;
    const float C6 = B20x2 * v_x, C9 = B20x2 * v_y;
    const float C7 = v_x * (B21r2x2 + vx2_6), C8 = v_x * fmaf(0.5f, vy2, B21r2x2);
    const float C10 = v_y * (B21r2x2 + vy2_6), C11 = v_y * fmaf(0.5f, vx2, B21r2x2);
    s.Scx = fmaf(B10, L[6], fmaf(C1, L[7], fmaf(C2, L[8], fmaf(vxy, L[11], fmaf(C6, L[1], fmaf(C9, L[12],
            fmaf(C7, L[3], fmaf(C10, L[14], fmaf(C11, L[13], C8 * L[4])))))))));
    s.Scy = fmaf(B10, L[9], fmaf(C1, L[11], fmaf(C2, L[10], fmaf(vxy, L[8], fmaf(C6, L[12], fmaf(C9, L[2],
            fmaf(C7, L[13], fmaf(C10, L[5], fmaf(C11, L[4], C8 * L[14])))))))));
  }
  return s;
}

}  // namespace lbm
