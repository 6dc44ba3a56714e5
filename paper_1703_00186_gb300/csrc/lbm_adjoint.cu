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

template <int PREC>
__global__ void __launch_bounds__(ABX * ABY) adjoint_kernel(const void* __restrict__ f_, const double* __restrict__ lam_in,
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
  const Moments mo = site_moments([&](int l) { return f[l]; });
  const SiteFields sf = site_fields(mo, a);
  const double theta = sf.T + a.tshift;
  const double uys = sf.uy - a.tau_g_xi;
  const double v_x = a.r2 * sf.ux, v_y = a.r2 * uys;
  const double U2 = a.r2 * fma(sf.ux, sf.ux, uys * uys);
  double lam[NPOP];
#pragma unroll
  for (int l = 0; l < NPOP; ++l) lam[l] = __ldg(lam_in + sidx(a, l, y, x));
  const EqCot s = eq_cotangent([&](int l) { return lam[l]; }, v_x, v_y, U2, theta, a);
  // gamma_q = sum_m lam_m d f^eq_m / d q for q = rho, Jx, Jy, Exi (xi units)
  const double usq = fma(sf.ux, sf.ux, sf.uy * sf.uy);
  const double gJx = a.r2 * fma(-s.Sth, sf.ux, fma(2.0 * a.inv_r2 * v_x, s.SU, s.Scx));
  const double gJy = a.r2 * fma(-s.Sth, sf.uy, fma(2.0 * a.inv_r2 * v_y, s.SU, s.Scy));
  const double gE = 0.5 * a.r2 * s.Sth;
  const double gR = s.SP - a.r2 * (sf.ux * (s.Scx + 2.0 * a.inv_r2 * v_x * s.SU) +
                                   sf.uy * (s.Scy + 2.0 * a.inv_r2 * v_y * s.SU)) +
                    s.Sth * fma(0.5 * a.r2, usq, -sf.T);
  const double wR = a.omega * gR, wJx = a.omega * gJx, wJy = a.omega * gJy, wE = a.omega * gE;
  // mu_l = (1 - omega) lam_l + omega (gR + gJ . xi_l + gE |xi_l|^2)
  double mu[NPOP];
  mu[0] = fma(a.omc, lam[0], wR);
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const double base = fma(wE, (double)shell_sq(pair_shell(k)), wR);
    const double lin = pair_cu<double>(k, wJx, wJy);
    mu[2 * k + 1] = fma(a.omc, lam[2 * k + 1], base + lin);
    mu[2 * k + 2] = fma(a.omc, lam[2 * k + 2], base - lin);
  }
  // P^T: push each cotangent back to its pull source; wall slots reduce.
  const bool bottom = !a.periodic_y && y < 3;
  const bool top = !a.periodic_y && y >= a.ly - 3;
  double wall_sum = 0.0;
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
      wall_sum = fma(ys < 0 ? a.q_bot[l] : a.q_top[l], mu[l], wall_sum);
    }
  }
  if (bottom) lam_out[scratch_idx(a, false, y, x)] = wall_sum;
  if (top) lam_out[scratch_idx(a, true, a.ly - 1 - y, x)] = wall_sum;
}

// B^T for the populations that left through a wall: lam_out(l, y0, x) =
// Lambda(x + xi_lx), Lambda(x) = sum over the three wall rows of the partial
// sums written by adjoint_kernel.
__global__ void walls_adjoint_kernel(double* __restrict__ lam_out, LatticeArgs a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const bool top = blockIdx.y == 1;
  if (x >= a.lx) return;
#pragma unroll
  for (int l = 0; l < NPOP; ++l) {
    const int xl = wrap_x(x + vx(l), a.lx);
    const double Lam = (lam_out[scratch_idx(a, top, 0, xl)] + lam_out[scratch_idx(a, top, 1, xl)]) +
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
template <int PREC>
__global__ void __launch_bounds__(ABX * ABY) moments_vjp_kernel(const void* __restrict__ f_, const double* __restrict__ g_rho,
                                                                const double* __restrict__ g_ux,
                                                                const double* __restrict__ g_uy,
                                                                const double* __restrict__ g_T,
                                                                double* __restrict__ lam_out, LatticeArgs a) {
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
  const double kt = 0.5 * a.r2 * sf.inv * gt;     // (r^2 / (2 rho)) g_T
  const double base = gr - gt * sf.T * sf.inv;
#pragma unroll
  for (int l = 0; l < NPOP; ++l) {
    const double dx = vx(l) - sf.ux, dy = vy(l) - sf.uy;
    lam_out[sidx(a, l, y, x)] = fma(kt, fma(dx, dx, dy * dy), fma(ku, fma(gx, dx, gy * dy), base));
  }
}

// g_q = sum_l lam_l d f^eq_l(rho, u, T) / d q for q = rho, ux, uy, T.
__global__ void __launch_bounds__(ABX * ABY) init_vjp_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                                                             const double* __restrict__ uy, const double* __restrict__ T,
                                                             const double* __restrict__ lam, double* __restrict__ g_rho,
                                                             double* __restrict__ g_ux, double* __restrict__ g_uy,
                                                             double* __restrict__ g_T, LatticeArgs a) {
  const int x = blockIdx.x * ABX + threadIdx.x;
  const int y = blockIdx.y * ABY + threadIdx.y;
  if (x >= a.lx || y >= a.ly) return;
  const long long i = (long long)y * a.lx + x;
  const double r0 = rho[i], u0 = ux[i], u1 = uy[i];
  const double U2 = fma(u0, u0, u1 * u1);
  const EqCot s = eq_cotangent([&](int l) { return __ldg(lam + sidx(a, l, y, x)); }, a.r * u0, a.r * u1, U2,
                               T[i] - 1.0, a);
  if (g_rho) g_rho[i] = s.SP;
  if (g_ux) g_ux[i] = r0 * fma(a.r, s.Scx, 2.0 * u0 * s.SU);
  if (g_uy) g_uy[i] = r0 * fma(a.r, s.Scy, 2.0 * u1 * s.SU);
  if (g_T) g_T[i] = r0 * s.Sth;
}

static dim3 site_grid(const LatticeArgs& a) {
  return dim3((unsigned)((a.lx + ABX - 1) / ABX), (unsigned)((a.ly + ABY - 1) / ABY));
}

cudaError_t launch_adjoint(int prec, const void* f_t, const double* lam_in, double* lam_out, const LatticeArgs& a,
                           cudaStream_t s) {
  const dim3 grid = site_grid(a), block(ABX, ABY);
  if (prec == LBM_FP64)
    adjoint_kernel<LBM_FP64><<<grid, block, 0, s>>>(f_t, lam_in, lam_out, a);
  else
    adjoint_kernel<LBM_FP32_SHIFTED><<<grid, block, 0, s>>>(f_t, lam_in, lam_out, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.periodic_y) return e;
  walls_adjoint_kernel<<<dim3((unsigned)((a.lx + 127) / 128), 2), 128, 0, s>>>(lam_out, a);
  return cudaGetLastError();
}

cudaError_t launch_moments_vjp(int prec, const void* f, const double* g_rho, const double* g_ux, const double* g_uy,
                               const double* g_T, double* lam_out, const LatticeArgs& a, cudaStream_t s) {
  const dim3 grid = site_grid(a), block(ABX, ABY);
  if (prec == LBM_FP64)
    moments_vjp_kernel<LBM_FP64><<<grid, block, 0, s>>>(f, g_rho, g_ux, g_uy, g_T, lam_out, a);
  else
    moments_vjp_kernel<LBM_FP32_SHIFTED><<<grid, block, 0, s>>>(f, g_rho, g_ux, g_uy, g_T, lam_out, a);
  return cudaGetLastError();
}

cudaError_t launch_init_vjp(const double* rho, const double* ux, const double* uy, const double* T,
                            const double* lam, double* g_rho, double* g_ux, double* g_uy, double* g_T,
                            const LatticeArgs& a, cudaStream_t s) {
  init_vjp_kernel<<<site_grid(a), dim3(ABX, ABY), 0, s>>>(rho, ux, uy, T, lam, g_rho, g_ux, g_uy, g_T, a);
  return cudaGetLastError();
}

}  // namespace lbm
