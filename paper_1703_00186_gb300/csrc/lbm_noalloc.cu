// lbm_adjoint_step_noalloc: the adjoint step for callers that cannot allocate
// device memory (declared and documented in include/lbm.h).
//
// A context (lbm_create) allocates a small device block, and the context
// adjoint keeps its per-wall-row partial sums in the halo rows of lam_out.
// This entry point needs neither: the lattice constants are derived on the
// host for every call, and the partial sums live in one fixed array defined
// below, which every GPU that loads the library holds until the process ends.
#include <cuda_runtime.h>

#include "lbm_adjoint_math.cuh"
#include "lbm_device.cuh"

namespace lbm {

int make_lattice_args(const lbm_params& p, LatticeArgs* a, char* err, size_t errlen);
size_t element_size(int precision);

namespace {

// Partial wall sums [wall (0 bottom, 1 top)][row offset from the wall 0..2][x].
// Every call writes each slot it later reads, so nothing needs clearing.
static __device__ __align__(256) double g_wall_partials[2 * 3 * LBM_NOALLOC_MAX_LX];

// Device address of g_wall_partials on the current device.  Host code cannot
// take the array's address directly (its name there is a host-side stand-in),
// so every call looks it up: a host-side lookup once the library's device
// code is loaded on the device.  Not caching it keeps the address right after
// a device reset, which reloads the device code, possibly elsewhere.
cudaError_t wall_partials_ptr(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_wall_partials);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

template <int PREC>
struct NDec;
template <>
struct NDec<LBM_FP64> {
  using T = double;
  const LatticeArgs* a;
  __device__ double operator()(int, double v) const { return v; }
};
template <>
struct NDec<LBM_FP32_SHIFTED> {
  using T = float;
  const LatticeArgs* a;
  __device__ double operator()(int l, float v) const { return a->w_rho0[l] + (double)v; }
};

__device__ __forceinline__ long long partial_idx(const LatticeArgs& a, int top, int d, int x) {
  return ((long long)top * 3 + d) * a.lx + x;
}

// Same arithmetic as the context adjoint: recompute the post-bc populations,
// apply the transposed collide Jacobian, push each cotangent back to its pull
// source; wall slots reduce into `partials` instead of lam_out's halo rows.
template <int PREC>
__global__ void __launch_bounds__(128) noalloc_adjoint_kernel(const void* __restrict__ f_,
                                                              const double* __restrict__ lam_in,
                                                              double* __restrict__ lam_out,
                                                              double* __restrict__ partials, LatticeArgs a) {
  using S = typename NDec<PREC>::T;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 4 + threadIdx.y;
  if (x >= a.lx || y >= a.ly) return;
  const S* __restrict__ src = static_cast<const S*>(f_);
  NDec<PREC> dec{&a};
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
  const double usq = fma(sf.ux, sf.ux, sf.uy * sf.uy);
  const double gJx = a.r2 * fma(-s.Sth, sf.ux, fma(2.0 * a.inv_r2 * v_x, s.SU, s.Scx));
  const double gJy = a.r2 * fma(-s.Sth, sf.uy, fma(2.0 * a.inv_r2 * v_y, s.SU, s.Scy));
  const double gE = a.r2_2 * s.Sth;
  const double gR = s.SP - a.r2 * (sf.ux * (s.Scx + 2.0 * a.inv_r2 * v_x * s.SU) +
                                   sf.uy * (s.Scy + 2.0 * a.inv_r2 * v_y * s.SU)) +
                    s.Sth * fma(a.r2_2, usq, -sf.T);
  const double wR = a.omega * gR, wJx = a.omega * gJx, wJy = a.omega * gJy, wE = a.omega * gE;
  double mu[NPOP];
  mu[0] = fma(a.omc, lam[0], wR);
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) {
    const double base = fma(wE, (double)shell_sq(pair_shell(k)), wR);
    const double lin = pair_cu<double>(k, wJx, wJy);
    mu[2 * k + 1] = fma(a.omc, lam[2 * k + 1], base + lin);
    mu[2 * k + 2] = fma(a.omc, lam[2 * k + 2], base - lin);
  }
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
    if (known)
      lam_out[sidx(a, l, ys, wrap_x(x - vx(l), a.lx))] = mu[l];
    else
      wall_sum = fma(ys < 0 ? a.q_bot[l] : a.q_top[l], mu[l], wall_sum);
  }
  if (!a.periodic_y && y < 3) partials[partial_idx(a, 0, y, x)] = wall_sum;
  if (!a.periodic_y && y >= a.ly - 3) partials[partial_idx(a, 1, a.ly - 1 - y, x)] = wall_sum;
}

__global__ void noalloc_walls_kernel(double* __restrict__ lam_out, const double* __restrict__ partials,
                                     LatticeArgs a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int top = blockIdx.y == 1 ? 1 : 0;
  if (x >= a.lx) return;
#pragma unroll
  for (int l = 0; l < NPOP; ++l) {
    const int xl = wrap_x(x + vx(l), a.lx);
    const double Lam = (partials[partial_idx(a, top, 0, xl)] + partials[partial_idx(a, top, 1, xl)]) +
                       partials[partial_idx(a, top, 2, xl)];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      if (!top && e + vy(l) < 0) lam_out[sidx(a, l, e, x)] = Lam;
      if (top && e + vy(l) >= 3) lam_out[sidx(a, l, a.ly - 3 + e, x)] = Lam;
    }
  }
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_adjoint_step_noalloc(const lbm_params* p, const void* f_t, const double* lam_in,
                                        double* lam_out, void* stream) {
  using namespace lbm;
  if (!p || !f_t || !lam_in || !lam_out || (const void*)lam_in == (const void*)lam_out) return LBM_ERR_INVALID;
  if (p->lx > LBM_NOALLOC_MAX_LX) return LBM_ERR_SIZE;
  LatticeArgs a;
  char err[256];
  const int rc = make_lattice_args(*p, &a, err, sizeof err);
  if (rc != LBM_OK) return rc;
  if (a.regularized) return LBM_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(f_t) % element_size(p->precision) ||
      reinterpret_cast<uintptr_t>(lam_in) % sizeof(double) || reinterpret_cast<uintptr_t>(lam_out) % sizeof(double))
    return LBM_ERR_INVALID;
  double* partials = nullptr;
  if (wall_partials_ptr(&partials) != cudaSuccess) return LBM_ERR_CUDA;
  // clear an error that earlier, unrelated calls left in the runtime's
  // last-error state, so that the checks below see this call's launches only
  (void)cudaGetLastError();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const dim3 grid((unsigned)((a.lx + 31) / 32), (unsigned)((a.ly + 3) / 4)), block(32, 4);
  if (p->precision != LBM_FP32_SHIFTED)
    noalloc_adjoint_kernel<LBM_FP64><<<grid, block, 0, s>>>(f_t, lam_in, lam_out, partials, a);
  else
    noalloc_adjoint_kernel<LBM_FP32_SHIFTED><<<grid, block, 0, s>>>(f_t, lam_in, lam_out, partials, a);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  if (!a.periodic_y) {
    noalloc_walls_kernel<<<dim3((unsigned)((a.lx + 127) / 128), 2), 128, 0, s>>>(lam_out, partials, a);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  }
  return LBM_OK;
}
