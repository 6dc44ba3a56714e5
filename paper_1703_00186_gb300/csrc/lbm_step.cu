// Forward kernels of the D2Q37 step for sm_103a.
//
// step_kernel fuses the three kernels of the paper's time step (Sect. 2:
// propagate, bc, collide; eq. 1) into one pass: every thread owns one lattice
// site, pulls its 37 populations from the neighbours up to three sites away
// (coalesced along x, the contiguous dimension of the SoA layout of Sect. 4),
// applies the thermal walls if it sits in one of the three rows next to a wall,
// relaxes in registers and writes the site of the other buffer.  The paper
// keeps propagate and collide apart because bc sits between them (Sect. 4);
// here the walls only need the three rows next to them, which the wall threads
// read directly, so the fusion removes one full read and write of the lattice.
#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

constexpr int BX = 32;  // threads along x (one warp per row segment)
constexpr int BY = 4;   // rows per block

template <int PREC>
struct Codec;

template <>
struct Codec<LBM_FP64> {
  using T = double;
  const LatticeArgs* a;
  __device__ double operator()(int, double v) const { return v; }
  __device__ double enc(int, double v) const { return v; }
};

template <>
struct Codec<LBM_FP32_SHIFTED> {
  using T = float;
  const LatticeArgs* a;
  __device__ double operator()(int l, float v) const { return a->w_rho0[l] + (double)v; }
  __device__ float enc(int l, double v) const { return (float)(v - a->w_rho0[l]); }
};

template <int PREC, bool COLLIDE, bool DFARITH = false, bool REG = false, bool OBS = false>
__global__ void __launch_bounds__(BX * BY) step_kernel(const void* __restrict__ src_,
                                                       void* __restrict__ dst_, LatticeArgs a,
                                                       double* __restrict__ obs = nullptr) {
  using T = typename Codec<PREC>::T;
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y = blockIdx.y * BY + threadIdx.y;
  if (x >= a.lx || y >= a.ly) return;
  const T* __restrict__ src = static_cast<const T*>(src_);
  T* __restrict__ dst = static_cast<T*>(dst_);
  Codec<PREC> codec{&a};
  T f[NPOP];
  if (fast_site(a, x)) pull_fast(src, site_off(a, y, x), a, f);
  else pull(src, x, y, a, f);
  walls(src, x, y, a, f, codec, [&](int l, double v) { return codec.enc(l, v); });
  if constexpr (PREC == LBM_FP64 && DFARITH) {
    if (COLLIDE) {
      __shared__ double s_f[NPOP][BX * BY];
      collide_fp64_df<BX * BY>(f, a, s_f, threadIdx.y * BX + threadIdx.x, dst, x, y);
      return;
    }
  }
  if (COLLIDE) {
    if constexpr (PREC == LBM_FP64 && REG) {
      collide_fp64_reg(f, a);
    } else if constexpr (PREC == LBM_FP64 && OBS) {
      // measurement epilogue: the collide leaves rho and T unchanged and adds
      // the impulse g_vec to u, so the new state's mid-step velocity is the
      // pre-collide u + g_vec / 2; warp sums (one row segment) go to the row
      // totals with one atomic add per quantity.
      const SiteFields sf = collide_fp64(f, a);
      double o[NOBS];
      site_observables(sf.rho, a.r * sf.ux, a.r * sf.uy - 0.5 * a.g, sf.T, o);
      const unsigned mask = __activemask();
#pragma unroll
      for (int i = 0; i < NOBS; ++i) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) o[i] += __shfl_down_sync(mask, o[i], off);
      }
      if ((threadIdx.x & 31) == __ffs(mask) - 1) {
#pragma unroll
        for (int i = 0; i < NOBS; ++i) atomicAdd(obs + (long long)i * a.ly + y, o[i]);
      }
    } else if constexpr (PREC == LBM_FP64) {
      collide_fp64(f, a);
    } else {
      collide_fp32(f, a);
    }
  }
  store_site(dst, x, y, a, f);
}

template <int PREC>
__global__ void __launch_bounds__(BX * BY) init_kernel(void* __restrict__ dst_, const double* __restrict__ rho,
                                                       const double* __restrict__ ux,
                                                       const double* __restrict__ uy,
                                                       const double* __restrict__ T, LatticeArgs a) {
  using S = typename Codec<PREC>::T;
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y = blockIdx.y * BY + threadIdx.y;
  if (x >= a.lx || y >= a.ly) return;
  const long long i = (long long)y * a.lx + x;
  double f[NPOP];
  equilibrium(rho[i], ux[i], uy[i], T[i], a, f);
  S* dst = static_cast<S*>(dst_);
  Codec<PREC> codec{&a};
#pragma unroll
  for (int l = 0; l < NPOP; ++l) dst[sidx(a, l, y, x)] = codec.enc(l, f[l]);
}

// eq. (2): rho, u = j / rho, T = (E / rho - |u|^2) / D of a stored state.
template <int PREC>
__global__ void __launch_bounds__(BX * BY) moments_kernel(const void* __restrict__ src_, double* __restrict__ rho,
                                                          double* __restrict__ ux, double* __restrict__ uy,
                                                          double* __restrict__ T, LatticeArgs a) {
  using S = typename Codec<PREC>::T;
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y = blockIdx.y * BY + threadIdx.y;
  if (x >= a.lx || y >= a.ly) return;
  const S* src = static_cast<const S*>(src_);
  Codec<PREC> codec{&a};
  Moments mo = moment_sums([&](int l) { return codec(l, src[sidx(a, l, y, x)]); });
  const SiteFields sf = site_fields(mo, a);
  const long long i = (long long)y * a.lx + x;
  if (rho) rho[i] = sf.rho;
  if (ux) ux[i] = a.r * sf.ux;
  if (uy) uy[i] = a.r * sf.uy;
  if (T) T[i] = sf.T;
}

template <int PREC>
__global__ void finite_kernel(const void* __restrict__ src_, LatticeArgs a, unsigned int* flag) {
  using S = typename Codec<PREC>::T;
  const S* src = static_cast<const S*>(src_);
  const long long per_plane = (long long)a.ly * a.lx;
  const long long n = per_plane * NPOP;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long l = i / per_plane, r = i - l * per_plane;
    const double v = (double)src[l * a.plane + HALO * (long long)a.lx + r];
    bad |= !isfinite(v);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// Row averages of the observables of a stored state (deterministic: fixed
// per-thread strides and a fixed-order tree reduction).  One block per row.
template <int PREC>
__global__ void __launch_bounds__(256) profiles_kernel(const void* __restrict__ src_, double* __restrict__ out,
                                                       LatticeArgs a) {
  using S = typename Codec<PREC>::T;
  const int y = blockIdx.x;
  const S* src = static_cast<const S*>(src_);
  Codec<PREC> codec{&a};
  double acc[NOBS];
#pragma unroll
  for (int i = 0; i < NOBS; ++i) acc[i] = 0.0;
  for (int x = threadIdx.x; x < a.lx; x += blockDim.x) {
    const Moments mo = moment_sums([&](int l) { return codec(l, src[sidx(a, l, y, x)]); });
    const SiteFields sf = site_fields(mo, a);
    double o[NOBS];
    site_observables(sf.rho, a.r * sf.ux, a.r * sf.uy + 0.5 * a.g, sf.T, o);
#pragma unroll
    for (int i = 0; i < NOBS; ++i) acc[i] += o[i];
  }
  __shared__ double red[NOBS][256];
#pragma unroll
  for (int i = 0; i < NOBS; ++i) red[i][threadIdx.x] = acc[i];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
#pragma unroll
      for (int i = 0; i < NOBS; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x < NOBS) out[(long long)threadIdx.x * a.ly + y] = red[threadIdx.x][0] / a.lx;
}

// Divide observed row totals by lx.
__global__ void scale_rows_kernel(double* __restrict__ obs, long long n, double s) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) obs[i] *= s;
}

static dim3 site_grid(const LatticeArgs& a) {
  return dim3((unsigned)((a.lx + BX - 1) / BX), (unsigned)((a.ly + BY - 1) / BY));
}

cudaError_t launch_step(int prec, bool collide, const void* src, void* dst, const LatticeArgs& a,
                        cudaStream_t s) {
  const dim3 grid = site_grid(a), block(BX, BY);
  if (prec == LBM_FP64_DF) {
    if (collide)
      step_kernel<LBM_FP64, true, true><<<grid, block, 0, s>>>(src, dst, a);
    else
      step_kernel<LBM_FP64, false><<<grid, block, 0, s>>>(src, dst, a);
  } else if (prec == LBM_FP64) {
    if (collide && a.regularized)
      step_kernel<LBM_FP64, true, false, true><<<grid, block, 0, s>>>(src, dst, a);
    else if (collide)
      step_kernel<LBM_FP64, true><<<grid, block, 0, s>>>(src, dst, a);
    else
      step_kernel<LBM_FP64, false><<<grid, block, 0, s>>>(src, dst, a);
  } else {
    if (collide)
      step_kernel<LBM_FP32_SHIFTED, true><<<grid, block, 0, s>>>(src, dst, a);
    else
      step_kernel<LBM_FP32_SHIFTED, false><<<grid, block, 0, s>>>(src, dst, a);
  }
  return cudaGetLastError();
}

cudaError_t launch_profiles(int prec, const void* src, double* out, const LatticeArgs& a, cudaStream_t s) {
  if (prec == LBM_FP64)
    profiles_kernel<LBM_FP64><<<a.ly, 256, 0, s>>>(src, out, a);
  else
    profiles_kernel<LBM_FP32_SHIFTED><<<a.ly, 256, 0, s>>>(src, out, a);
  return cudaGetLastError();
}

// One float64 step that also adds the row totals of the new state's
// observables into obs[NOBS][ly] (zeroed here) and scales them to averages.
cudaError_t launch_step_observe(const void* src, void* dst, const LatticeArgs& a, double* obs, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(obs, 0, sizeof(double) * NOBS * (size_t)a.ly, s);
  if (e != cudaSuccess) return e;
  step_kernel<LBM_FP64, true, false, false, true><<<site_grid(a), dim3(BX, BY), 0, s>>>(src, dst, a, obs);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = (long long)NOBS * a.ly;
  scale_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(obs, n, 1.0 / a.lx);
  return cudaGetLastError();
}

cudaError_t launch_init(int prec, void* dst, const double* rho, const double* ux, const double* uy,
                        const double* T, const LatticeArgs& a, cudaStream_t s) {
  const dim3 grid = site_grid(a), block(BX, BY);
  if (prec == LBM_FP64)
    init_kernel<LBM_FP64><<<grid, block, 0, s>>>(dst, rho, ux, uy, T, a);
  else
    init_kernel<LBM_FP32_SHIFTED><<<grid, block, 0, s>>>(dst, rho, ux, uy, T, a);
  return cudaGetLastError();
}

cudaError_t launch_moments(int prec, const void* src, double* rho, double* ux, double* uy, double* T,
                           const LatticeArgs& a, cudaStream_t s) {
  const dim3 grid = site_grid(a), block(BX, BY);
  if (prec == LBM_FP64)
    moments_kernel<LBM_FP64><<<grid, block, 0, s>>>(src, rho, ux, uy, T, a);
  else
    moments_kernel<LBM_FP32_SHIFTED><<<grid, block, 0, s>>>(src, rho, ux, uy, T, a);
  return cudaGetLastError();
}

cudaError_t launch_finite(int prec, const void* src, const LatticeArgs& a, unsigned int* flag,
                          cudaStream_t s) {
  const int blocks = 152 * 8;
  if (prec == LBM_FP64)
    finite_kernel<LBM_FP64><<<blocks, 256, 0, s>>>(src, a, flag);
  else
    finite_kernel<LBM_FP32_SHIFTED><<<blocks, 256, 0, s>>>(src, a, flag);
  return cudaGetLastError();
}

}  // namespace lbm
