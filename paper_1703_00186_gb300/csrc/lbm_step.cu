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
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "lbm_device.cuh"
#include "tma.cuh"

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

// Occupancy caps, as measured: the double-float step with its pair groups
// unrolled runs best at 128 registers (4 blocks per SM, no spills; a
// 96-register cap spills and is 1.5 % slower), the regularised step at 128
// (4 blocks; 96 spills, 163 unconstrained is slower).
#ifndef LBM_DF_MINB
#define LBM_DF_MINB 4  // minimum resident blocks per SM of the double-float step
#endif
#ifndef LBM_FP64_FIX
#define LBM_FP64_FIX 1  // float64 BGK step: equilibrium polynomial on the integer pipe
#endif
#ifndef LBM_FP64_MINB
#define LBM_FP64_MINB 0  // minimum resident blocks per SM of the float64 BGK step (0: no cap)
#endif
#ifndef LBM_REG_MINB
#define LBM_REG_MINB 4  // minimum resident blocks per SM of the regularised step
#endif
template <int PREC, bool COLLIDE, bool DFARITH = false, bool REG = false, int F32M = FP32_ARITH_SPLIT>
__global__ void __launch_bounds__(BX * BY, REG ? LBM_REG_MINB : DFARITH ? LBM_DF_MINB : (PREC == LBM_FP64 && COLLIDE) ? LBM_FP64_MINB : 0) step_kernel(const void* __restrict__ src_,
                                                       void* __restrict__ dst_, LatticeArgs a, int xb, int xe) {
  using T = typename Codec<PREC>::T;
  const int x = xb + (int)blockIdx.x * BX + (int)threadIdx.x;  // columns xb <= x < xe
  const int y = blockIdx.y * BY + threadIdx.y;
  if (x >= xe || y >= a.ly) return;
  const T* __restrict__ src = static_cast<const T*>(src_);
  T* __restrict__ dst = static_cast<T*>(dst_);
  Codec<PREC> codec{&a};
  T f[NPOP];
  if (fast_warp(a, x)) pull_fast(src, site_off(a, y, x), a, f);
  else pull(src, x, y, a, f);
  if constexpr (PREC == LBM_FP32_SHIFTED && F32M == FP32_ARITH_F64_COLLIDE) {
    if (COLLIDE) {
      // the float64 step on the decoded populations, walls included, stored
      // back once: the error of the float32 storage alone
      double g[NPOP];
#pragma unroll
      for (int l = 0; l < NPOP; ++l) g[l] = codec(l, f[l]);
      walls(src, x, y, a, g, codec, [](int, double v) { return v; });
      collide_fp64(g, a);
#pragma unroll
      for (int l = 0; l < NPOP; ++l) f[l] = codec.enc(l, g[l]);
      store_site(dst, x, y, a, f);
      return;
    }
  }
  walls(src, x, y, a, f, codec, [&](int l, double v) { return codec.enc(l, v); });
  if constexpr (PREC == LBM_FP64 && DFARITH) {
    if (COLLIDE) {
      __shared__ double s_f[NPOP][BX * BY];
      collide_fp64_df<BX * BY>(f, a, s_f, threadIdx.y * BX + threadIdx.x, dst, x, y);
      return;
    }
  }
  if constexpr (PREC == LBM_FP64 && REG) {
    if (COLLIDE) {
      __shared__ double s_f[NPOP][BX * BY];
      collide_fp64_reg_grouped<BX * BY>(f, a, s_f, threadIdx.y * BX + threadIdx.x, dst, x, y);
      return;
    }
  }
  if constexpr (PREC == LBM_FP64 && LBM_FP64_FIX) {
    if (COLLIDE) {
      __shared__ double s_f[NPOP][BX * BY];
      collide_fp64_fix<BX * BY>(f, a, s_f, threadIdx.y * BX + threadIdx.x, dst, x, y);
      return;
    }
  }
  if (COLLIDE) {
    if constexpr (PREC == LBM_FP64) {
      collide_fp64(f, a);
    } else if constexpr (F32M == FP32_ARITH_F64_TERMS) {
      collide_fp32_f64terms(f, a);
    } else {
      collide_fp32(f, a);
    }
  }
  store_site(dst, x, y, a, f);
}

// float64 step with a measurement epilogue: the collide leaves rho and T
// unchanged and adds the impulse g_vec to u, so the new state's mid-step
// velocity is the pre-collide u + g_vec / 2.  A warp is one 32-site row
// segment (BX = 32): every lane takes part in the warp sums, lanes beyond the
// right edge with zeros.  The sums are exact in fixed point on the integer
// pipe (float64 shuffles and adds only if a value is outside the fixed-point
// range) and go to the row totals with one atomic add per quantity.
__global__ void __launch_bounds__(BX * BY, 4) step_observe_kernel(const double* __restrict__ src,
                                                               double* __restrict__ dst, LatticeArgs a,
                                                               double* __restrict__ obs) {
  static_assert(BX == 32, "one warp per row segment");
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y = blockIdx.y * BY + threadIdx.y;
  if (y >= a.ly) return;  // whole warps
  double o[NOBS];
#pragma unroll
  for (int i = 0; i < NOBS; ++i) o[i] = 0.0;
  if (x < a.lx) {
    Codec<LBM_FP64> codec{&a};
    double f[NPOP];
    if (fast_site(a, x)) pull_fast(src, site_off(a, y, x), a, f);
    else pull(src, x, y, a, f);
    walls(src, x, y, a, f, codec, [&](int l, double v) { return codec.enc(l, v); });
    __shared__ double s_f[NPOP][BX * BY];
    const ObsFields of = collide_fp64_fix<BX * BY>(f, a, s_f, threadIdx.y * BX + threadIdx.x, dst, x, y);
    site_observables(of.rho, of.ux, of.uy, of.T, o);
  }
  constexpr unsigned kAll = 0xffffffffu;
  bool ok = true;
  Fix96 q[NOBS];
#pragma unroll
  for (int i = 0; i < NOBS; ++i) q[i] = to_fix(o[i], ok);
  if (__all_sync(kAll, ok)) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int i = 0; i < NOBS; ++i) {
        const Fix96 other{__shfl_down_sync(kAll, q[i].w0, off), __shfl_down_sync(kAll, q[i].w1, off),
                          __shfl_down_sync(kAll, q[i].w2, off)};
        q[i] = fix_add(q[i], other);
      }
    }
    if ((threadIdx.x & 31) == 0) {  // only the lane that adds to the totals rounds
#pragma unroll
      for (int i = 0; i < NOBS; ++i) o[i] = fix_to_double(q[i]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < NOBS; ++i) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) o[i] += __shfl_down_sync(kAll, o[i], off);
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int i = 0; i < NOBS; ++i) atomicAdd(obs + (long long)i * a.ly + y, o[i]);
  }
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
  Moments mo = site_moments([&](int l) { return codec(l, src[sidx(a, l, y, x)]); });
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
    const Moments mo = site_moments([&](int l) { return codec(l, src[sidx(a, l, y, x)]); });
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

// ---------------------------------------------------------------------------
// FP32-store step with TMA-staged pull sources (LBM_FLAG_TMA_LOADS).
//
// A persistent grid walks tiles of 32 x TY sites.  For every tile one thread
// issues 37 three-dimensional TMA loads, one per population plane, of the box
// of columns x0 - 4 .. x0 + 35 (the start is 16-byte aligned, as TMA requires)
// and of the TY rows y0 - xi_ly .. that hold the pull sources of population l
// (Sect. 2, propagate); the box of population l therefore holds
// src_l(x - xi_lx, y - xi_ly) at column tx + 4 - xi_lx, row ty.  The registers
// are the second buffer: every thread copies its 37 sources out of the stage,
// the block synchronises, and the loads of the block's next tile are issued
// at once, in flight while this tile computes.  Columns within 3 of the
// periodic seam read their sources with plain loads (the box does not wrap);
// wall rows read the halo rows like the plain kernel and are then overwritten
// by the walls.  Same arithmetic as step_kernel, so the results are
// bit-identical.  On GB300 it hides the load latency (long-scoreboard stalls
// fall from 1.4 to 0.5 per issue) but the per-tile block barrier costs more
// (1.3 per issue), and it runs about 10% slower than step_kernel.
constexpr int TMA_TX = 32;
constexpr int TMA_BOXW = TMA_TX + 8;
constexpr int TMA_STAGES = 1;  // shared-memory stages (the registers add one)
constexpr int TMA_MINB = 5;  // minimum resident blocks per SM (register cap)
constexpr unsigned long long TMA_WAIT_NS = 2000000000ull;  // 2 s
constexpr unsigned kStatusTmaTimeout = 2u;

template <int TY>
struct TmaTile {
  static constexpr int box_floats = TMA_BOXW * TY;                  // one population box
  static constexpr int box_stride = (box_floats + 31) / 32 * 32;    // 128-byte aligned
  static constexpr int stage_floats = NPOP * box_stride;
  static constexpr unsigned stage_tx = NPOP * box_floats * 4u;       // bytes landed per stage
  static constexpr size_t smem_bytes = TMA_STAGES * stage_floats * 4u + 128 + TMA_STAGES * 8;
};

template <int TY>
__global__ void __launch_bounds__(TMA_TX * TY, TMA_MINB) step_tma_kernel(const __grid_constant__ CUtensorMap map,
                                                               const float* __restrict__ src,
                                                               float* __restrict__ dst, LatticeArgs a,
                                                               int tiles_x, int n_tiles) {
  using Tile = TmaTile<TY>;
  extern __shared__ unsigned char smem_raw[];
  float* stages = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint64_t* bar = reinterpret_cast<uint64_t*>(stages + TMA_STAGES * Tile::stage_floats);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool leader = (tx | ty) == 0;
  Codec<LBM_FP32_SHIFTED> codec{&a};

  auto issue = [&](int s, int t) {
    const int x0 = (t % tiles_x) * TMA_TX, y0 = (t / tiles_x) * TY;
    mbar_arrive_expect_tx(&bar[s], Tile::stage_tx);
    float* base = stages + s * Tile::stage_floats;
#pragma unroll
    for (int l = 0; l < NPOP; ++l)
      tma_load_3d(base + l * Tile::box_stride, &map, x0 - 4, y0 + HALO - vy(l), l, &bar[s]);
  };

  if (leader) {
    for (int s = 0; s < TMA_STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
    for (int s = 0; s < TMA_STAGES; ++s) {
      const int t = blockIdx.x + s * gridDim.x;
      if (t < n_tiles) issue(s, t);
    }
  }
  __syncthreads();

  int it = 0;
  bool timed_out = false;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
    const int s = it % TMA_STAGES;
    const bool arrived = mbar_wait_bounded(&bar[s], (unsigned)(it / TMA_STAGES) & 1u, TMA_WAIT_NS);
    const int x = (t % tiles_x) * TMA_TX + tx, y = (t / tiles_x) * TY + ty;
    const bool active = x < a.lx && y < a.ly;
    float f[NPOP];
    if (active) {
      if (x >= 3 && x < a.lx - 3) {
        const float* b = stages + s * Tile::stage_floats + ty * TMA_BOXW + tx + 4;
#pragma unroll
        for (int l = 0; l < NPOP; ++l) f[l] = b[l * Tile::box_stride - vx(l)];
      } else {
        pull(src, x, y, a, f);
      }
    }
    // every thread has read stage s (or the wait gave up somewhere)
    if (__syncthreads_or(!arrived)) {
      timed_out = true;
      break;
    }
    const int next = t + TMA_STAGES * gridDim.x;
    if (leader && next < n_tiles) {
      fence_proxy_async_smem();
      issue(s, next);
    }
    if (active) {
      walls(src, x, y, a, f, codec, [&](int l, double v) { return codec.enc(l, v); });
      collide_fp32(f, a);
      store_site(dst, x, y, a, f);
    }
  }
  if (timed_out && leader) {
    if (a.status) atomicOr(a.status, kStatusTmaTimeout);
    // let loads still in flight land before the block's shared memory goes away
    for (int k = 0; k < TMA_STAGES; ++k) {
      const int j = it + k;
      if (blockIdx.x + j * gridDim.x < (unsigned)n_tiles)
        mbar_wait_bounded(&bar[j % TMA_STAGES], (unsigned)(j / TMA_STAGES) & 1u, TMA_WAIT_NS);
    }
  }
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

constexpr int TMA_TY = 4;

// Per-device launch shape of the TMA kernel (set up once per device).
struct TmaLaunch {
  int grid_per_sm = 0;
  bool ready = false;
};

static bool tma_launch_shape(int dev, int* ctas) {
  static std::mutex mu;
  static TmaLaunch shapes[64];
  if (dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lock(mu);
  TmaLaunch& sh = shapes[dev];
  if (!sh.ready) {
    const size_t smem = TmaTile<TMA_TY>::smem_bytes;
    if (cudaFuncSetAttribute(step_tma_kernel<TMA_TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return false;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_tma_kernel<TMA_TY>, TMA_TX * TMA_TY, smem) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
      return false;
    sh.grid_per_sm = per_sm * sms;
    sh.ready = true;
  }
  *ctas = sh.grid_per_sm;
  return true;
}

// Whether an FP32-store collide step from `src` runs the TMA-staged kernel.
bool step_uses_tma(const LatticeArgs& a, const void* src) {
  int dev = 0, ctas = 0;
  return a.tma_loads && a.fp32_arith == FP32_ARITH_SPLIT && !a.periodic_y && a.idx32 && a.lx % 4 == 0 &&
         (reinterpret_cast<uintptr_t>(src) & 15u) == 0 && tensor_map_encoder() != nullptr &&
         cudaGetDevice(&dev) == cudaSuccess && tma_launch_shape(dev, &ctas);
}

// The TMA-staged FP32 step, or cudaErrorNotSupported when its conditions do
// not hold (the caller then uses step_kernel).
static cudaError_t launch_step_tma(const void* src, void* dst, const LatticeArgs& a, cudaStream_t s) {
  if (!step_uses_tma(a, src)) return cudaErrorNotSupported;
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  int dev = 0, ctas = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || !tma_launch_shape(dev, &ctas)) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[3] = {(cuuint64_t)a.lx, (cuuint64_t)(a.ly + 2 * HALO), (cuuint64_t)NPOP};
  const cuuint64_t strides[2] = {(cuuint64_t)a.lx * sizeof(float), (cuuint64_t)a.plane * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)TMA_BOXW, (cuuint32_t)TMA_TY, 1u};
  const cuuint32_t elem[3] = {1u, 1u, 1u};
  if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(src), dims, strides, box, elem,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorNotSupported;
  const int tiles_x = (a.lx + TMA_TX - 1) / TMA_TX;
  const long long n_tiles = (long long)tiles_x * ((a.ly + TMA_TY - 1) / TMA_TY);
  if (n_tiles > 0x7fffffffLL) return cudaErrorNotSupported;
  const int grid = (int)std::min<long long>(n_tiles, ctas);
  step_tma_kernel<TMA_TY><<<grid, dim3(TMA_TX, TMA_TY), TmaTile<TMA_TY>::smem_bytes, s>>>(
      map, static_cast<const float*>(src), static_cast<float*>(dst), a, tiles_x, (int)n_tiles);
  return cudaGetLastError();
}

static dim3 site_grid(const LatticeArgs& a) {
  return dim3((unsigned)((a.lx + BX - 1) / BX), (unsigned)((a.ly + BY - 1) / BY));
}

// One step (collide = false: propagate and bc only) from src to dst for the
// sites of columns x0 <= x < x1 (every physical row); other columns of dst
// are not written.
cudaError_t launch_step_columns(int prec, bool collide, const void* src, void* dst, const LatticeArgs& a, int x0,
                                int x1, cudaStream_t s) {
  if (x1 <= x0) return cudaSuccess;
  const dim3 grid((unsigned)((x1 - x0 + BX - 1) / BX), (unsigned)((a.ly + BY - 1) / BY)), block(BX, BY);
  if (prec == LBM_FP64_DF) {
    if (collide)
      step_kernel<LBM_FP64, true, true><<<grid, block, 0, s>>>(src, dst, a, x0, x1);
    else
      step_kernel<LBM_FP64, false><<<grid, block, 0, s>>>(src, dst, a, x0, x1);
  } else if (prec == LBM_FP64) {
    if (collide && a.regularized)
      step_kernel<LBM_FP64, true, false, true><<<grid, block, 0, s>>>(src, dst, a, x0, x1);
    else if (collide)
      step_kernel<LBM_FP64, true><<<grid, block, 0, s>>>(src, dst, a, x0, x1);
    else
      step_kernel<LBM_FP64, false><<<grid, block, 0, s>>>(src, dst, a, x0, x1);
  } else {
    if (collide && a.fp32_arith == FP32_ARITH_F64_TERMS)
      step_kernel<LBM_FP32_SHIFTED, true, false, false, FP32_ARITH_F64_TERMS><<<grid, block, 0, s>>>(src, dst, a, x0,
                                                                                                    x1);
    else if (collide && a.fp32_arith == FP32_ARITH_F64_COLLIDE)
      step_kernel<LBM_FP32_SHIFTED, true, false, false, FP32_ARITH_F64_COLLIDE><<<grid, block, 0, s>>>(src, dst, a,
                                                                                                      x0, x1);
    else if (collide)
      step_kernel<LBM_FP32_SHIFTED, true><<<grid, block, 0, s>>>(src, dst, a, x0, x1);
    else
      step_kernel<LBM_FP32_SHIFTED, false><<<grid, block, 0, s>>>(src, dst, a, x0, x1);
  }
  return cudaGetLastError();
}

cudaError_t launch_step(int prec, bool collide, const void* src, void* dst, const LatticeArgs& a,
                        cudaStream_t s) {
  if (prec == LBM_FP32_SHIFTED && collide && a.fp32_arith == FP32_ARITH_SPLIT) {
    const cudaError_t e = launch_step_tma(src, dst, a, s);
    if (e != cudaErrorNotSupported) return e;
    (void)cudaGetLastError();  // a refused set-up call leaves no error behind
  }
  return launch_step_columns(prec, collide, src, dst, a, 0, a.lx, s);
}

// Columns [x0, x0 + n) of every population's physical rows to / from a
// contiguous buffer [37][ly][n] (the halo exchange of an x-slab, Sect. 4).
template <typename T>
__global__ void pack_columns_kernel(const T* __restrict__ f, T* __restrict__ buf, LatticeArgs a, int x0, int n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)NPOP * a.ly * n;
  if (i >= total) return;
  const int c = (int)(i % n);
  const long long r = i / n;  // l * ly + y
  const int l = (int)(r / a.ly), y = (int)(r - (long long)l * a.ly);
  buf[i] = f[sidx(a, l, y, x0 + c)];
}

template <typename T>
__global__ void unpack_columns_kernel(const T* __restrict__ buf, T* __restrict__ f, LatticeArgs a, int x0, int n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)NPOP * a.ly * n;
  if (i >= total) return;
  const int c = (int)(i % n);
  const long long r = i / n;
  const int l = (int)(r / a.ly), y = (int)(r - (long long)l * a.ly);
  f[sidx(a, l, y, x0 + c)] = buf[i];
}

cudaError_t launch_columns_copy(int prec, bool pack, const void* from, void* to, const LatticeArgs& a, int x0, int n,
                                cudaStream_t s) {
  const long long total = (long long)NPOP * a.ly * n;
  if (total == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (prec == LBM_FP32_SHIFTED) {
    if (pack)
      pack_columns_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(from), static_cast<float*>(to), a,
                                                         x0, n);
    else
      unpack_columns_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(from), static_cast<float*>(to),
                                                           a, x0, n);
  } else {
    if (pack)
      pack_columns_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(from), static_cast<double*>(to),
                                                          a, x0, n);
    else
      unpack_columns_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(from),
                                                            static_cast<double*>(to), a, x0, n);
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
  step_observe_kernel<<<site_grid(a), dim3(BX, BY), 0, s>>>(static_cast<const double*>(src), static_cast<double*>(dst),
                                                         a, obs);
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
