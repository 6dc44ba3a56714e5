// Discrete adjoint of the D2Q37 step and the vector-Jacobian products of the
// initial state and of the macroscopic fields (eq. 2).
//
// One step is f' = C(B(P f)) (collide after bc after propagate, Sect. 2), so
// the adjoint of a cotangent lam' is  lam = P^T B^T C^T lam'.  It runs as two
// kernels:
//   adjoint_kernel : per site, recompute the post-bc populations from f_t,
//                    apply C^T (the transposed Jacobian of the BGK collide,
//                    eq. 1, through rho, u and T of eq. 2), then push every
//                    cotangent back to the site it was pulled from (P^T);
//                    cotangents of wall slots, which bc filled with M(x) q_l,
//                    are reduced per wall row into the halo rows of lam_out;
//   walls_adjoint  : each population that left through a wall receives the
//                    column sum of those wall cotangents (B^T).
#include <cuda_runtime.h>

#include "lbm_adjoint_math.cuh"
#include "lbm_adjoint_f32.cuh"
#include "lbm_device.cuh"

namespace lbm {

constexpr int ABX = 32;
constexpr int ABY = 4;

template <int PREC>
struct Dec;
template <>
struct Dec<LBM_FP64> {
  using T = double;
  const LatticeArgs* a;
  __device__ double operator()(int, double v) const { return v; }
};
template <>
struct Dec<LBM_FP32_SHIFTED> {
  using T = float;
  const LatticeArgs* a;
  __device__ double operator()(int l, float v) const { return a->w_rho0[l] + (double)v; }
};

// Halo-row scratch of lam_out: partial wall sums of row d (0..2) from the
// bottom / top wall, stored in population plane 0.
__device__ __forceinline__ long long scratch_idx(const LatticeArgs& a, bool top, int d, int x) {
  const int yh = top ? a.ly + d : -1 - d;
  return (long long)(yh + HALO) * a.lx + x;
}

// P^T: push each cotangent back to its pull source; the cotangents of wall
// slots (filled by bc with M(x) q_l) reduce into lam_out's halo-row scratch.
// R is the cotangents' storage type (double, or float for
// lbm_adjoint_step_f32).
template <typename R>
__device__ __forceinline__ void push_cotangents(const R (&mu)[NPOP], int x, int y, const LatticeArgs& a,
                                                R* __restrict__ lam_out) {
  const bool bottom = !a.periodic_y && y < 3;
  const bool top = !a.periodic_y && y >= a.ly - 3;
  R wall_sum = R(0);
#pragma unroll
  for (int l = 0; l < NPOP; ++l) {
    int ys = y - vy(l);
    bool known = true;
    if (a.periodic_y) {
      ys = ys < 0 ? ys + a.ly : (ys >= a.ly ? ys - a.ly : ys);
    } else if (ys < 0 || ys >= a.ly) {
      known = false;
    }
    if (known) {
      lam_out[sidx(a, l, ys, wrap_x(x - vx(l), a.lx))] = mu[l];
    } else {
      wall_sum = fma(R(ys < 0 ? a.q_bot[l] : a.q_top[l]), mu[l], wall_sum);
    }
  }
  if (bottom) lam_out[scratch_idx(a, false, y, x)] = wall_sum;
  if (top) lam_out[scratch_idx(a, true, a.ly - 1 - y, x)] = wall_sum;
}

#ifndef LBM_ADJ_MINB
#define LBM_ADJ_MINB 3  // minimum resident blocks per SM of the float64 adjoint step
#endif
template <int PREC>
__global__ void __launch_bounds__(ABX * ABY, LBM_ADJ_MINB) adjoint_kernel(const void* __restrict__ f_, const double* __restrict__ lam_in,
                                                            double* __restrict__ lam_out, LatticeArgs a) {
  using S = typename Dec<PREC>::T;
  const int x = blockIdx.x * ABX + threadIdx.x;
  const int y = blockIdx.y * ABY + threadIdx.y;
  if (x >= a.lx || y >= a.ly) return;
  const S* __restrict__ src = static_cast<const S*>(f_);
  Dec<PREC> dec{&a};
  // post-bc populations at this site, float64
  double f[NPOP];
  {
    S g[NPOP];
    pull(src, x, y, a, g);
#pragma unroll
    for (int l = 0; l < NPOP; ++l) f[l] = dec(l, g[l]);
  }
  walls(src, x, y, a, f, dec, [](int, double v) { return v; });
  const AdjSite q = adj_site(site_moments<-1>([&](int l) { return f[l]; }), a);  // from rho, J, E / 2
  // the cotangents wait in shared memory: the fixed-point sums and the
  // relaxation read them twice, and registers hold the accumulators
  __shared__ double s_lam[NPOP][ABX * ABY];
  const int tid = threadIdx.y * ABX + threadIdx.x;
#pragma unroll
  for (int l = 0; l < NPOP; ++l) s_lam[l][tid] = __ldg(lam_in + sidx(a, l, y, x));
  const auto lam = [&](int l) { return s_lam[l][tid]; };
  double L[15];
  if (!cotangent_moments_fix(lam, a, L)) cotangent_moments(lam, a, L);
  const EqCot s = eq_cotangent_site(L, q, a);
  // gamma_q = sum_m lam_m d f^eq_m / d q for q = rho, Jx, Jy, Exi (xi units),
  // with r^2 u = (v_x, vy0): G = r^2 (S_cu + 2 S_U v / r^2), gamma_J =
  // G - S_theta r^2 u, gamma_rho = S_P - u . G + S_theta ((r^2/2) |u|^2 - T)
  const double SU2 = s.SU + s.SU;
  const double Gx = fma(q.v_x, SU2, a.r2 * s.Scx), Gy = fma(q.v_y, SU2, a.r2 * s.Scy);
  const double gJx = fma(-s.Sth, q.v_x, Gx);
  const double gJy = fma(-s.Sth, q.vy0, Gy);
  const double gE = a.r2_2 * s.Sth;
  const double Q = fma(fma(q.vy0, q.vy0, q.vx2), a.half_inv_r2, a.tshift - q.theta);  // (r^2/2) |u|^2 - T
  const double gR = fma(s.Sth, Q, fma(-a.inv_r2, fma(q.v_x, Gx, q.vy0 * Gy), s.SP));
  const double wR = a.omega * gR, wJx = a.omega * gJx, wJy = a.omega * gJy, wE = a.omega * gE;
  // mu_l = (1 - omega) lam_l + omega (gR + gJ . xi_l + gE |xi_l|^2)
  double mu[NPOP];
  mu[0] = fma(a.omc, lam(0), wR);
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const double base = fma(wE, (double)shell_sq(pair_shell(k)), wR);
    const double lin = pair_cu<double>(k, wJx, wJy);
    mu[2 * k + 1] = fma(a.omc, lam(2 * k + 1), base + lin);
    mu[2 * k + 2] = fma(a.omc, lam(2 * k + 2), base - lin);
  }
  push_cotangents(mu, x, y, a, lam_out);
}

// The pair representatives R_k of c_pair_rep as float64: x, y and |R_k|^2.
static __constant__ double c_pair_rep_d[NPAIR][3] = {
    {1, 0, 1}, {0, 1, 1}, {1, 1, 2}, {-1, 1, 2}, {2, 0, 4}, {0, 2, 4}, {2, 1, 5}, {1, 2, 5}, {-1, 2, 5},
    {-2, 1, 5}, {2, 2, 8}, {-2, 2, 8}, {3, 0, 9}, {0, 3, 9}, {3, 1, 10}, {1, 3, 10}, {-1, 3, 10}, {-3, 1, 10}};

// Adjoint step of LBM_FP64_DF and LBM_FP32_SHIFTED contexts (the latter on
// the decoded float64 state): the same transposed Jacobian with
// the cotangent sums of the equilibrium in double-float arithmetic on the
// FP32 pipe (as the forward collide of that mode), the pair loop rolled over
// cotangents staged in shared memory; the site fields, the final cotangent
// combination and the push stay float64.
//   SP = sum lam w P,  Scu = sum lam w P_cu xi,  SU = sum lam w dP/dU2,
//   Sth = sum lam w dP/dtheta (see eq_cotangent).
template <int PREC>
__global__ void __launch_bounds__(ABX * ABY) adjoint_df_kernel(const void* __restrict__ f_,
                                                               const double* __restrict__ lam_in,
                                                               double* __restrict__ lam_out, LatticeArgs a) {
  using S = typename Dec<PREC>::T;
  __shared__ double s_lam[NPOP][ABX * ABY];
  const int x = blockIdx.x * ABX + threadIdx.x;
  const int y = blockIdx.y * ABY + threadIdx.y;
  if (x >= a.lx || y >= a.ly) return;
  const int tid = threadIdx.y * ABX + threadIdx.x;
  const S* __restrict__ src = static_cast<const S*>(f_);
  Dec<PREC> dec{&a};
  SiteFields sf;
  {
    S g[NPOP];
    pull(src, x, y, a, g);
    Moments mo;
    bool exact = false;
    if constexpr (PREC == LBM_FP32_SHIFTED) {
      // away from the walls the moment sums come straight from the float32
      // bit patterns (exact, integer pipe): no float64 decode of the 37
      // populations, which would take 74 FP64 issue slots
      if (a.periodic_y || (y >= 3 && y < a.ly - 3)) exact = moment_sums_f32_exact(g, a, mo);
    }
    if (!exact) {
      double f[NPOP];
#pragma unroll
      for (int l = 0; l < NPOP; ++l) f[l] = dec(l, g[l]);
      walls(src, x, y, a, f, dec, [](int, double v) { return v; });
      mo = site_moments([&](int l) { return f[l]; });
    }
    sf = site_fields(mo, a);
  }
#pragma unroll
  for (int l = 0; l < NPOP; ++l) s_lam[l][tid] = __ldg(lam_in + sidx(a, l, y, x));
  // site terms and equilibrium coefficients (as collide_fp64_df)
  const DF ux = df_from_double_bits(sf.ux), uy = df_from_double_bits(sf.uy);
  const DF theta = df_add(df_from_double_bits(sf.T), dfc(a.df_tshift));
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
  // d/dU2 and d/dtheta of the shell coefficients
  const DF dU0 = df_add(df_add(df_scale2(U2, 0.25f), theta), -0.5f);                   // dB00/dU2
  const DF dU1 = df_scale2(theta, -0.25f);                                              // dB01/dU2
  const DF dT0 = df_add(df_add(df_scale2(theta, 2.0f), U2), -1.0f);                    // dB00/dtheta
  const DF dT1 = df_add(df_add(df_scale2(theta, -2.0f), df_scale2(U2, -0.25f)), 0.5f);  // dB01/dtheta
  const DF dT2 = df_scale2(theta, 0.25f);                                               // dB02/dtheta
  DF SP, Scx{0.f, 0.f}, Scy{0.f, 0.f}, SU, Sth;
  {
    const DF l0 = df_mul(df_from_double_bits(s_lam[0][tid]), dfc(a.df_w_shell[0]));
    SP = df_mul(l0, B00);
    SU = df_mul(l0, dU0);
    Sth = df_mul(l0, dT0);
  }
  // Every accumulated term is a cotangent times an O(1) polynomial value, so
  // the 11-operation double-word additions keep the error at a few u^2 of the
  // sum of the terms' magnitudes, as float64 accumulation does at n u.
  // Both loops are rolled: the unrolled body overflows the instruction cache.
#pragma unroll 1
  for (int j = 1; j < NSHELL; ++j) {
    const DF c2 = dfc(a.df_c2_shell[j]);
    const DF w = dfc(a.df_w_shell[j]);
    const DF A0 = df_add_fast(df_mul(df_add_fast(df_mul(B02, c2), B01), c2), B00);
    const DF A1 = df_add_fast(df_mul(B11, c2), B10);
    const DF A2 = df_add_fast(df_mul(B21, c2), B20);
    const DF aU = df_add_fast(df_mul(dU1, c2), dU0);                                 // dA0/dU2
    const DF aT = df_add_fast(df_mul(df_add_fast(df_mul(dT2, c2), dT1), c2), dT0);  // dA0/dtheta
    const DF hT = df_add(df_scale2(c2, 0.5f), -2.0f);                                // dA1/dtheta
    const DF bT = df_add(df_scale2(c2, 0.25f), -1.5f);                               // dA2/dtheta
    const DF A2x2 = df_scale2(A2, 2.0f);
#pragma unroll 1
    for (int k = shell_first_pair(j); k < shell_first_pair(j + 1); ++k) {
      const float rx = (float)c_pair_rep[k][0], ry = (float)c_pair_rep[k][1];
      const DF lp = df_from_double_bits(s_lam[2 * k + 1][tid]), lm = df_from_double_bits(s_lam[2 * k + 2][tid]);
      const DF Ls = df_mul(df_add_fast(lp, lm), w), La = df_mul(df_add_fast(lp, df_neg(lm)), w);
      const DF cu = df_add_fast(df_mul(v_x, rx), df_mul(v_y, ry));
      const DF cu2 = df_mul(cu, cu);
      const DF Pe = df_add_fast(df_mul(df_add_fast(df_mul(cu2, DF{0x1.555556p-5f, -0x1.555556p-30f}), A2), cu2), A0);
      const DF P6 = df_mul(cu2, DF{0x1.555556p-3f, -0x1.555556p-28f});  // cu^2 / 6
      const DF Po = df_mul(df_add_fast(P6, A1), cu);
      const DF Pce = df_add_fast(df_scale2(cu2, 0.5f), A1);
      const DF Pco = df_mul(df_add_fast(P6, A2x2), cu);
      SP = df_add_fast(SP, df_add_fast(df_mul(Ls, Pe), df_mul(La, Po)));
      const DF t = df_add_fast(df_mul(La, Pce), df_mul(Ls, Pco));
      Scx = df_add_fast(Scx, df_mul(t, rx));
      Scy = df_add_fast(Scy, df_mul(t, ry));
      SU = df_add_fast(SU, df_add_fast(df_mul(Ls, df_add_fast(df_scale2(cu2, -0.25f), aU)),
                                       df_mul(df_scale2(La, -0.5f), cu)));
      Sth = df_add_fast(Sth, df_add_fast(df_mul(Ls, df_add_fast(df_mul(bT, cu2), aT)),
                                         df_mul(df_mul(La, hT), cu)));
    }
  }
  EqCot s;
  s.SP = df_to_double_bits(SP);
  s.Scx = df_to_double_bits(Scx);
  s.Scy = df_to_double_bits(Scy);
  s.SU = df_to_double_bits(SU);
  s.Sth = df_to_double_bits(Sth);
  // the rest as adjoint_kernel, float64
  const double vxd = a.r2 * sf.ux, vyd = a.r2 * (sf.uy - a.tau_g_xi);
  const double usq = fma(sf.ux, sf.ux, sf.uy * sf.uy);
  const double gJx = a.r2 * fma(-s.Sth, sf.ux, fma(2.0 * a.inv_r2 * vxd, s.SU, s.Scx));
  const double gJy = a.r2 * fma(-s.Sth, sf.uy, fma(2.0 * a.inv_r2 * vyd, s.SU, s.Scy));
  const double gE = a.r2_2 * s.Sth;
  const double gR = s.SP - a.r2 * (sf.ux * (s.Scx + 2.0 * a.inv_r2 * vxd * s.SU) +
                                   sf.uy * (s.Scy + 2.0 * a.inv_r2 * vyd * s.SU)) +
                    s.Sth * fma(a.r2_2, usq, -sf.T);
  const double wR = a.omega * gR, wJx = a.omega * gJx, wJy = a.omega * gJy, wE = a.omega * gE;
  // mu_l = (1 - omega) lam_l + omega (gR + gJ . xi_l + gE |xi_l|^2), pushed
  // back to its pull source as it is formed (P^T; wall slots reduce), in a
  // loop rolled over the pairs: the same operations as adjoint_kernel
  double wall_sum = 0.0;
  auto push = [&](int l, int ex, int ey, double m) {
    int ys = y - ey;
    bool known = true;
    if (a.periodic_y) {
      ys = ys < 0 ? ys + a.ly : (ys >= a.ly ? ys - a.ly : ys);
    } else if (ys < 0 || ys >= a.ly) {
      known = false;
    }
    if (known) lam_out[sidx(a, l, ys, wrap_x(x - ex, a.lx))] = m;
    else wall_sum = fma(ys < 0 ? a.q_bot[l] : a.q_top[l], m, wall_sum);
  };
  push(0, 0, 0, fma(a.omc, s_lam[0][tid], wR));
#pragma unroll 1
  for (int k = 0; k < NPAIR; ++k) {
    const int rx = c_pair_rep[k][0], ry = c_pair_rep[k][1];
    // float64 copies from a table: an int-to-double conversion would take an
    // FP64 issue slot
    const double base = fma(wE, c_pair_rep_d[k][2], wR);
    const double lin = fma(c_pair_rep_d[k][0], wJx, c_pair_rep_d[k][1] * wJy);  // = pair_cu(k, wJx, wJy)
    push(2 * k + 1, rx, ry, fma(a.omc, s_lam[2 * k + 1][tid], base + lin));
    push(2 * k + 2, -rx, -ry, fma(a.omc, s_lam[2 * k + 2][tid], base - lin));
  }
  if (!a.periodic_y && y < 3) lam_out[scratch_idx(a, false, y, x)] = wall_sum;
  if (!a.periodic_y && y >= a.ly - 3) lam_out[scratch_idx(a, true, a.ly - 1 - y, x)] = wall_sum;
}

// B^T for the populations that left through a wall: lam_out(l, y0, x) =
// Lambda(x + xi_lx), Lambda(x) = sum over the three wall rows of the partial
// sums written by adjoint_kernel.
template <typename R>
__global__ void walls_adjoint_kernel(R* __restrict__ lam_out, LatticeArgs a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const bool top = blockIdx.y == 1;
  if (x >= a.lx) return;
#pragma unroll
  for (int l = 0; l < NPOP; ++l) {
    const int xl = wrap_x(x + vx(l), a.lx);
    const R Lam = (lam_out[scratch_idx(a, top, 0, xl)] + lam_out[scratch_idx(a, top, 1, xl)]) +
                  lam_out[scratch_idx(a, top, 2, xl)];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      if (!top && e + vy(l) < 0) lam_out[sidx(a, l, e, x)] = Lam;
      if (top && e + vy(l) >= 3) lam_out[sidx(a, l, a.ly - 3 + e, x)] = Lam;
    }
  }
}

// lam_l = g_rho d rho/d f_l + g_u . d u/d f_l + g_T d T/d f_l  (eq. 2):
//   d rho/d f_l = 1, d u/d f_l = (c_l - u) / rho,
//   d T/d f_l = (|c_l - u|^2 - D T) / (D rho).
template <int PREC, typename R>
__global__ void __launch_bounds__(ABX * ABY) moments_vjp_kernel(const void* __restrict__ f_, const double* __restrict__ g_rho,
                                                                const double* __restrict__ g_ux,
                                                                const double* __restrict__ g_uy,
                                                                const double* __restrict__ g_T,
                                                                R* __restrict__ lam_out, LatticeArgs a) {
  using S = typename Dec<PREC>::T;
  const int x = blockIdx.x * ABX + threadIdx.x;
  const int y = blockIdx.y * ABY + threadIdx.y;
  if (x >= a.lx || y >= a.ly) return;
  const S* src = static_cast<const S*>(f_);
  Dec<PREC> dec{&a};
  const Moments mo = site_moments([&](int l) { return dec(l, src[sidx(a, l, y, x)]); });
  const SiteFields sf = site_fields(mo, a);
  const long long i = (long long)y * a.lx + x;
  const double gr = g_rho ? g_rho[i] : 0.0;
  const double gx = g_ux ? g_ux[i] : 0.0;
  const double gy = g_uy ? g_uy[i] : 0.0;
  const double gt = g_T ? g_T[i] : 0.0;
  const double ku = a.r * sf.inv;                 // d u / d f = r (xi - u_xi) / rho
  const double kt = a.r2_2 * sf.inv * gt;     // (r^2 / (2 rho)) g_T
  const double base = gr - gt * sf.T * sf.inv;
#pragma unroll
  for (int l = 0; l < NPOP; ++l) {
    const double dx = vx(l) - sf.ux, dy = vy(l) - sf.uy;
    lam_out[sidx(a, l, y, x)] = R(fma(kt, fma(dx, dx, dy * dy), fma(ku, fma(gx, dx, gy * dy), base)));
  }
}

// g_q = sum_l lam_l d f^eq_l(rho, u, T) / d q for q = rho, ux, uy, T.
template <typename R>
__global__ void __launch_bounds__(ABX * ABY) init_vjp_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                                                             const double* __restrict__ uy, const double* __restrict__ T,
                                                             const R* __restrict__ lam, double* __restrict__ g_rho,
                                                             double* __restrict__ g_ux, double* __restrict__ g_uy,
                                                             double* __restrict__ g_T, LatticeArgs a) {
  const int x = blockIdx.x * ABX + threadIdx.x;
  const int y = blockIdx.y * ABY + threadIdx.y;
  if (x >= a.lx || y >= a.ly) return;
  const long long i = (long long)y * a.lx + x;
  const double r0 = rho[i], u0 = ux[i], u1 = uy[i];
  const double U2 = fma(u0, u0, u1 * u1);
  const EqCot s = eq_cotangent([&](int l) { return (double)__ldg(lam + sidx(a, l, y, x)); }, a.r * u0, a.r * u1, U2,
                               T[i] - 1.0, a);
  if (g_rho) g_rho[i] = s.SP;
  if (g_ux) g_ux[i] = r0 * fma(a.r, s.Scx, 2.0 * u0 * s.SU);
  if (g_uy) g_uy[i] = r0 * fma(a.r, s.Scy, 2.0 * u1 * s.SU);
  if (g_T) g_T[i] = r0 * s.Sth;
}

// Adjoint step of FP32-store contexts with float32 cotangents
// (lbm_adjoint_step_f32): the transposed Jacobian of adjoint_kernel with the
// cotangents read, summed, relaxed and pushed in float32 (FP32 pipe).  The
// site fields of the forward state are exact fixed-point moment sums of the
// float32 deviations (away from the walls) and float64 fields, rounded once
// to float32.  Per site it moves 148 B of state and 2 x 148 B of cotangents.
__global__ void __launch_bounds__(ABX * ABY) adjoint_f32_kernel(const float* __restrict__ src,
                                                                const float* __restrict__ lam_in,
                                                                float* __restrict__ lam_out, LatticeArgs a) {
  const int x = blockIdx.x * ABX + threadIdx.x;
  const int y = blockIdx.y * ABY + threadIdx.y;
  if (x >= a.lx || y >= a.ly) return;
  Dec<LBM_FP32_SHIFTED> dec{&a};
  SiteFields sf;
  {
    float g[NPOP];
    pull(src, x, y, a, g);
    Moments mo;
    bool exact = false;
    if (a.periodic_y || (y >= 3 && y < a.ly - 3)) exact = moment_sums_f32_exact(g, a, mo);
    if (!exact) {
      double f[NPOP];
#pragma unroll
      for (int l = 0; l < NPOP; ++l) f[l] = dec(l, g[l]);
      walls(src, x, y, a, f, dec, [](int, double v) { return v; });
      mo = site_moments([&](int l) { return f[l]; });
    }
    sf = site_fields(mo, a);
  }
  float lam[NPOP];
#pragma unroll
  for (int l = 0; l < NPOP; ++l) lam[l] = __ldg(lam_in + sidx(a, l, y, x));
  float L[15];
  cotangent_moments_f(lam, a, L);
  const float ux = (float)sf.ux, uy = (float)sf.uy, T = (float)sf.T;
  const float theta = (float)(sf.T + a.tshift), uys = (float)(sf.uy - a.tau_g_xi);
  const float r2 = a.df_r2[0], ir2 = a.df_inv_r2[0];
  const float v_x = r2 * ux, v_y = r2 * uys;
  const float U2 = r2 * fmaf(ux, ux, uys * uys);
  const EqCotF s = eq_cotangent_mono_f(L, v_x, v_y, U2, theta, a);
  // gamma_q = sum_m lam_m d f^eq_m / d q for q = rho, Jx, Jy, Exi (xi units)
  const float usq = fmaf(ux, ux, uy * uy);
  const float kx = 2.0f * ir2 * v_x, ky = 2.0f * ir2 * v_y;
  const float gJx = r2 * fmaf(-s.Sth, ux, fmaf(kx, s.SU, s.Scx));
  const float gJy = r2 * fmaf(-s.Sth, uy, fmaf(ky, s.SU, s.Scy));
  const float gE = 0.5f * r2 * s.Sth;
  const float gR = s.SP - r2 * (ux * fmaf(kx, s.SU, s.Scx) + uy * fmaf(ky, s.SU, s.Scy)) +
                   s.Sth * fmaf(0.5f * r2, usq, -T);
  const float om = a.omega_f, omc = a.omc_f;
  const float wR = om * gR, wJx = om * gJx, wJy = om * gJy, wE = om * gE;
  // mu_l = (1 - omega) lam_l + omega (gR + gJ . xi_l + gE |xi_l|^2)
  float mu[NPOP];
  mu[0] = fmaf(omc, lam[0], wR);
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const float base = fmaf(wE, (float)shell_sq(pair_shell(k)), wR);
    const float lin = pair_cu<float>(k, wJx, wJy);
    mu[2 * k + 1] = fmaf(omc, lam[2 * k + 1], base + lin);
    mu[2 * k + 2] = fmaf(omc, lam[2 * k + 2], base - lin);
  }
  push_cotangents(mu, x, y, a, lam_out);
}

static dim3 site_grid(const LatticeArgs& a) {
  return dim3((unsigned)((a.lx + ABX - 1) / ABX), (unsigned)((a.ly + ABY - 1) / ABY));
}

cudaError_t launch_adjoint(int prec, const void* f_t, const double* lam_in, double* lam_out, const LatticeArgs& a,
                           cudaStream_t s) {
  const dim3 grid = site_grid(a), block(ABX, ABY);
  if (prec == LBM_FP64_DF)
    adjoint_df_kernel<LBM_FP64><<<grid, block, 0, s>>>(f_t, lam_in, lam_out, a);
  else if (prec == LBM_FP64)
    adjoint_kernel<LBM_FP64><<<grid, block, 0, s>>>(f_t, lam_in, lam_out, a);
  else
    adjoint_df_kernel<LBM_FP32_SHIFTED><<<grid, block, 0, s>>>(f_t, lam_in, lam_out, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.periodic_y) return e;
  walls_adjoint_kernel<<<dim3((unsigned)((a.lx + 127) / 128), 2), 128, 0, s>>>(lam_out, a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_f32(const void* f_t, const float* lam_in, float* lam_out, const LatticeArgs& a,
                               cudaStream_t s) {
  adjoint_f32_kernel<<<site_grid(a), dim3(ABX, ABY), 0, s>>>(static_cast<const float*>(f_t), lam_in, lam_out, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.periodic_y) return e;
  walls_adjoint_kernel<<<dim3((unsigned)((a.lx + 127) / 128), 2), 128, 0, s>>>(lam_out, a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_moments_vjp_t(int prec, const void* f, const double* g_rho, const double* g_ux, const double* g_uy,
                                 const double* g_T, R* lam_out, const LatticeArgs& a, cudaStream_t s) {
  const dim3 grid = site_grid(a), block(ABX, ABY);
  if (prec == LBM_FP64)
    moments_vjp_kernel<LBM_FP64, R><<<grid, block, 0, s>>>(f, g_rho, g_ux, g_uy, g_T, lam_out, a);
  else
    moments_vjp_kernel<LBM_FP32_SHIFTED, R><<<grid, block, 0, s>>>(f, g_rho, g_ux, g_uy, g_T, lam_out, a);
  return cudaGetLastError();
}

cudaError_t launch_moments_vjp(int prec, const void* f, const double* g_rho, const double* g_ux, const double* g_uy,
                               const double* g_T, double* lam_out, const LatticeArgs& a, cudaStream_t s) {
  return launch_moments_vjp_t(prec, f, g_rho, g_ux, g_uy, g_T, lam_out, a, s);
}

cudaError_t launch_moments_vjp_f32(int prec, const void* f, const double* g_rho, const double* g_ux,
                                   const double* g_uy, const double* g_T, float* lam_out, const LatticeArgs& a,
                                   cudaStream_t s) {
  return launch_moments_vjp_t(prec, f, g_rho, g_ux, g_uy, g_T, lam_out, a, s);
}

cudaError_t launch_init_vjp(const double* rho, const double* ux, const double* uy, const double* T,
                            const double* lam, double* g_rho, double* g_ux, double* g_uy, double* g_T,
                            const LatticeArgs& a, cudaStream_t s) {
  init_vjp_kernel<<<site_grid(a), dim3(ABX, ABY), 0, s>>>(rho, ux, uy, T, lam, g_rho, g_ux, g_uy, g_T, a);
  return cudaGetLastError();
}

cudaError_t launch_init_vjp_f32(const double* rho, const double* ux, const double* uy, const double* T,
                                const float* lam, double* g_rho, double* g_ux, double* g_uy, double* g_T,
                                const LatticeArgs& a, cudaStream_t s) {
  init_vjp_kernel<<<site_grid(a), dim3(ABX, ABY), 0, s>>>(rho, ux, uy, T, lam, g_rho, g_ux, g_uy, g_T, a);
  return cudaGetLastError();
}

}  // namespace lbm
