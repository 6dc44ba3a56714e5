// Batched stepping of many independent D2Q37 lattices (include/lbm_batch.h).
//
// One launch advances every lattice of the batch by one step: block b reads
// its lattice from a per-tile table (one load), copies that lattice's
// constants into shared memory and runs the fused propagate + bc + collide
// on its tile (the same device code as the single-lattice kernel).  n steps
// are captured into a CUDA graph on a private stream and replayed on the
// caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/lbm_batch.h"
#include "lbm_device.cuh"

namespace lbm {

int make_lattice_args(const lbm_params& p, LatticeArgs* a, char* err, size_t errlen);
cudaError_t launch_step(int prec, bool collide, const void* src, void* dst, const LatticeArgs& a, cudaStream_t s);
size_t element_size(int precision);
int storage_prec(int precision);
cudaError_t launch_init(int prec, void* dst, const double* rho, const double* ux, const double* uy,
                        const double* T, const LatticeArgs& a, cudaStream_t s);
cudaError_t launch_moments(int prec, const void* src, double* rho, double* ux, double* uy, double* T,
                           const LatticeArgs& a, cudaStream_t s);

struct BatchEntry {
  LatticeArgs a;
  void* f[2];
};

namespace {

constexpr int kTiles = 9;
constexpr int kTileBX[kTiles] = {32, 32, 64, 128, 32, 64, 32, 32, 32};
constexpr int kTileBY[kTiles] = {4, 8, 2, 1, 2, 4, 4, 4, 4};
// sites per thread along y: a tile covers kTileBY * kTileRows rows, so the
// per-tile work (lattice lookup, constants, barriers) is shared by more sites
constexpr int kTileRows[kTiles] = {1, 1, 1, 1, 1, 1, 2, 4, 8};
// Launch candidate kTiles is not a tile shape: every lattice is stepped by the
// single-lattice kernel (its constants in the kernel parameters, 32 x 4
// blocks), the lattices spread over kAux streams, all captured in one graph.
constexpr int kPerLattice = kTiles;
// Candidates kTiles + 1 .. : FP32-store tiles with the per-lattice constants
// in the kernel parameters (batch_param_kernel), 32 x 4 threads, these rows
// per thread.
constexpr int kParamTiles = 3;
constexpr int kParamRows[kParamTiles] = {1, 4, 8};
constexpr int kParamFirst = kTiles + 1;
constexpr int kCandidates = kParamFirst + kParamTiles;
constexpr int kAux = 8;

template <int PREC>
struct BCodec;
template <>
struct BCodec<LBM_FP64> {
  using T = double;
  const LatticeArgs* a;
  __device__ double operator()(int, double v) const { return v; }
  __device__ double enc(int, double v) const { return v; }
};
template <>
struct BCodec<LBM_FP32_SHIFTED> {
  using T = float;
  const LatticeArgs* a;
  __device__ double operator()(int l, float v) const { return a->w_rho0[l] + (double)v; }
  __device__ float enc(int l, double v) const { return (float)(v - a->w_rho0[l]); }
};

using Codec32 = BCodec<LBM_FP32_SHIFTED>;

// One tile of the batch work list; block-wide: every thread of the block
// calls it (threads outside the lattice skip the work but reach the barriers).
template <int PREC, int TBX, int TBY, bool DFARITH, bool COHERENT, int ROWS = 1>
__device__ __forceinline__ void batch_tile(const BatchEntry* __restrict__ ent, const long long* __restrict__ tile_start,
                                           const int* __restrict__ tile_lattice, int parity, long long b,
                                           LatticeArgs& sa, const void*& s_src, void*& s_dst) {
  using T = typename BCodec<PREC>::T;
  const int lo = __ldg(tile_lattice + b);  // the lattice that owns tile b
  const int tid = threadIdx.y * TBX + threadIdx.x;
  {
    static_assert(sizeof(LatticeArgs) % 8 == 0, "LatticeArgs must be a multiple of 8 bytes");
    const unsigned long long* g = reinterpret_cast<const unsigned long long*>(&ent[lo].a);
    unsigned long long* sm = reinterpret_cast<unsigned long long*>(&sa);
    for (int k = tid; k < (int)(sizeof(LatticeArgs) / 8); k += TBX * TBY) sm[k] = __ldg(g + k);
    if (tid == 0) {
      s_src = ent[lo].f[parity];
      s_dst = ent[lo].f[parity ^ 1];
    }
  }
  __syncthreads();
  const LatticeArgs& a = sa;
  const long long t = b - __ldg(tile_start + lo);
  const int tiles_x = (a.lx + TBX - 1) / TBX;
  const int ty = (int)(t / tiles_x), tx = (int)(t - (long long)ty * tiles_x);
  const int x = tx * TBX + threadIdx.x;
#pragma unroll 1
  for (int r = 0; r < ROWS; ++r) {
  const int y = (ty * ROWS + r) * TBY + threadIdx.y;
  if (x < a.lx && y < a.ly) {
    const T* __restrict__ src = static_cast<const T*>(s_src);
    T* __restrict__ dst = static_cast<T*>(s_dst);
    BCodec<PREC> codec{&a};
    T f[NPOP];
    if (fast_site(a, x)) pull_fast<T, COHERENT>(src, site_off(a, y, x), a, f);
    else pull<T, COHERENT>(src, x, y, a, f);
    walls<COHERENT>(src, x, y, a, f, codec, [&](int l, double v) { return codec.enc(l, v); });
    if constexpr (PREC == LBM_FP64 && DFARITH) {
      __shared__ double s_f[NPOP][TBX * TBY];
      collide_fp64_df<TBX * TBY>(f, a, s_f, tid, dst, x, y);
    } else if constexpr (PREC == LBM_FP64 && TBX * TBY <= 128) {
      __shared__ double s_f[NPOP][TBX * TBY];  // 37.9 KB per 128-thread tile; larger tiles keep collide_fp64
      collide_fp64_fix<TBX * TBY>(f, a, s_f, tid, dst, x, y);
    } else {
      if constexpr (PREC == LBM_FP64)
        collide_fp64(f, a);
      else
        collide_fp32<!COHERENT>(f, a);  // the persistent kernel keeps the scalar relaxation
      store_site(dst, x, y, a, f);
    }
  }
  }
  __syncthreads();  // sa / s_src / s_dst are reused by the block's next tile
}

// FP32 tiles: at most 128 registers for 128-thread blocks (4 blocks per SM).
// With the packed relaxation a 96-register cap spilled 124-140 bytes and
// measured 10% slower.
template <int PREC, int TBX, int TBY, bool DFARITH = false, int ROWS = 1>
__global__ void __launch_bounds__(TBX * TBY, PREC == LBM_FP32_SHIFTED ? 4 * 128 / (TBX * TBY) : 0) batch_step_kernel(const BatchEntry* __restrict__ ent,
                                                               const long long* __restrict__ tile_start,
                                                               const int* __restrict__ tile_lattice, int parity) {
  __shared__ __align__(16) LatticeArgs sa;
  __shared__ const void* s_src;
  __shared__ void* s_dst;
  batch_tile<PREC, TBX, TBY, DFARITH, false, ROWS>(ent, tile_start, tile_lattice, parity, blockIdx.x, sa, s_src, s_dst);
}

// ---------------------------------------------------------------------------
// FP32-store tiles with the per-lattice constants in the kernel parameters.
//
// The shared-memory tile kernel above copies each tile's LatticeArgs into
// shared memory and reads every constant back from there (38 shared loads
// per site, and the registers that hold them).  This kernel takes a table of
// up to kParamLattices lattices as a __grid_constant__ parameter instead: a
// block finds its lattice by a binary search over the table's tile offsets
// (block-uniform, in the parameter bank), and every per-lattice constant it
// then reads - the pull and store offsets, the size, the density, tau and g
// terms of the collide - is a load from the parameter bank at a block-uniform
// address, as in the single-lattice kernel, where these are compile-time
// parameter offsets.  The quadrature constants, the same for every lattice,
// come from one LatticeArgs parameter.  Wall rows and the three columns next
// to the periodic seam read the full LatticeArgs of their lattice from global
// memory (the wall ratios, the shift constants and the general index path).
// Batches of more lattices run one launch per group of kParamLattices.
constexpr int kParamLattices = 64;

struct ParamLat {
  long long tile_start;     // first tile of the lattice in the group's work list
  long long edge_start;     // first edge site of the lattice in the group's edge list
  const void* f[2];         // ping-pong state buffers
  const LatticeArgs* args;  // the lattice's full constants (device copy)
  int lx, ly, tiles_x, pad;
  float omega_f, omc_f, df_rho0[2], df_e0[2], df_tshift[2], df_taug_r[2], df_g_r[2];
  int pull_off[NPOP];   // bytes, as LatticeArgs::pull_off (32-bit lattices only)
  int plane_off[NPOP];  // bytes, as LatticeArgs::plane_off
};

struct ParamTable {
  int n, pad;
  ParamLat e[kParamLattices];
};
static_assert(sizeof(ParamTable) + sizeof(LatticeArgs) + 16 <= 32764, "kernel parameters above 32 KB");

// Tile b of the group's work list (interior and seam sites; the wall rows
// are edge sites).  COHERENT: loads through L2 only, for the persistent
// kernel, whose blocks read what other blocks wrote in the previous step.
template <int TBX, int TBY, int ROWS, bool COHERENT>
__device__ __forceinline__ void param_tile(const ParamTable& t, const LatticeArgs& m, int parity, long long b) {
  int lo = 0, hi = t.n - 1;  // the last lattice whose first tile is <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.e[mid].tile_start <= b) lo = mid;
    else hi = mid - 1;
  }
  const ParamLat& e = t.e[lo];
  F32Args a;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    a.df_rho0[k] = e.df_rho0[k];
    a.df_e0[k] = e.df_e0[k];
    a.df_tshift[k] = e.df_tshift[k];
    a.df_taug_r[k] = e.df_taug_r[k];
    a.df_g_r[k] = e.df_g_r[k];
    a.df_half_r2[k] = m.df_half_r2[k];
    a.df_r2[k] = m.df_r2[k];
  }
  a.omega_f = e.omega_f;
  a.omc_f = e.omc_f;
#pragma unroll
  for (int j = 0; j < NSHELL; ++j) {
    a.w_shell_f[j] = m.w_shell_f[j];
    a.c2_shell_f[j] = m.c2_shell_f[j];
  }
  const int lx = e.lx, ly = e.ly;
  const long long tl = b - e.tile_start;
  const int ty = (int)(tl / e.tiles_x), tx = (int)(tl - (long long)ty * e.tiles_x);
  const int x = tx * TBX + threadIdx.x;
  // a tile holding a seam column takes the wrapped offsets for all its lanes
  // (block-uniform, so no warp runs both paths)
  const bool seam_tile = tx * TBX < 3 || tx * TBX + TBX > lx - 3;
  const float* __restrict__ src = static_cast<const float*>(e.f[parity]);
  float* __restrict__ dst = static_cast<float*>(const_cast<void*>(e.f[parity ^ 1]));
#pragma unroll 1
  for (int r = 0; r < ROWS; ++r) {
    const int y = (ty * ROWS + r) * TBY + threadIdx.y;
    if (x < lx && y < ly) {
      float f[NPOP];
      const int site = (y + HALO) * lx + x;
      if (y < 3 || y >= ly - 3) continue;  // wall rows: batch_edge_kernel
      if (!seam_tile) {
        const char* s = reinterpret_cast<const char*>(src + site);
#pragma unroll
        for (int l = 0; l < NPOP; ++l) f[l] = load<COHERENT>(reinterpret_cast<const float*>(s + e.pull_off[l]));
      } else {  // the three columns next to the periodic seam on each side
        const char* s = reinterpret_cast<const char*>(src + (y + HALO) * lx);
#pragma unroll
        for (int l = 0; l < NPOP; ++l)
          f[l] = load<COHERENT>(reinterpret_cast<const float*>(s + e.pull_off[l]) + (wrap_x(x - vx(l), lx) + vx(l)));
      }
      collide_fp32(f, a);
      char* d = reinterpret_cast<char*>(dst + site);
#pragma unroll
      for (int l = 0; l < NPOP; ++l) *reinterpret_cast<float*>(d + e.plane_off[l]) = f[l];
    }
  }
}

template <int TBX, int TBY, int ROWS>
__global__ void __launch_bounds__(TBX * TBY, 5 * 128 / (TBX * TBY))
    batch_param_kernel(const __grid_constant__ ParamTable t, const __grid_constant__ LatticeArgs m, int parity) {
  param_tile<TBX, TBY, ROWS, false>(t, m, parity, blockIdx.x);
}

// Number of edge sites of a lattice: the three rows next to each wall.
__host__ __device__ inline long long edge_sites(int lx, int ly) { return 6LL * lx; }

// The edge sites of every lattice of the group (those batch_param_kernel
// leaves out): the three rows next to each wall, through the general index
// path, the walls and the lattice's full LatticeArgs in global memory.  One thread per edge
// site; a thread finds its lattice by binary search over the edge offsets.
template <bool COHERENT>
__device__ __forceinline__ void param_edge(const ParamTable& t, int parity, long long j) {
  int lo = 0, hi = t.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.e[mid].edge_start <= j) lo = mid;
    else hi = mid - 1;
  }
  const ParamLat& e = t.e[lo];
  const int lx = e.lx, ly = e.ly;
  long long k = j - e.edge_start;
  int x, y;
  if (k < 3LL * lx) {  // bottom rows
    y = (int)(k / lx);
    x = (int)(k - (long long)y * lx);
  } else if ((k -= 3LL * lx) < 3LL * lx) {  // top rows
    const int r = (int)(k / lx);
    y = ly - 3 + r;
    x = (int)(k - (long long)r * lx);
  } else {
    return;  // not reached: the edge list holds the wall rows only
  }
  const LatticeArgs& ga = *e.args;
  const float* __restrict__ src = static_cast<const float*>(e.f[parity]);
  float* __restrict__ dst = static_cast<float*>(const_cast<void*>(e.f[parity ^ 1]));
  Codec32 codec{&ga};
  float f[NPOP];
  pull<float, COHERENT>(src, x, y, ga, f);
  walls<COHERENT>(src, x, y, ga, f, codec, [&](int l, double v) { return codec.enc(l, v); });
  collide_fp32(f, ga);
  store_site(dst, x, y, ga, f);
}

__global__ void __launch_bounds__(128) batch_edge_kernel(const __grid_constant__ ParamTable t,
                                                         const __grid_constant__ LatticeArgs m, int parity,
                                                         long long total) {
  const long long j = blockIdx.x * 128LL + threadIdx.x;
  if (j < total) param_edge<false>(t, parity, j);
}

// Grid barrier of the persistent kernel with a bounded wait.  State in global
// memory: arrival count, generation, abort flag, status word.  A block reads
// the generation, arrives, and (unless it is the last to arrive, which resets
// the count and advances the generation) waits for the generation to move.
// The wait gives up after budget_ns of global time or 2^24 polls: the block
// then sets LBM_STATUS_BARRIER_TIMEOUT in the status word and the abort flag,
// and every waiting block leaves; the kernel returns instead of hanging.
struct GridBarrier {
  unsigned int count, gen, abort, status;
};
constexpr unsigned int kBarrierTimeout = 1u;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool grid_barrier(GridBarrier* bar, unsigned int expected, unsigned long long budget_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int ok = 1;
    __threadfence();  // this block's writes before its arrival
    const unsigned int gen = atomicAdd(&bar->gen, 0u);
    const unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
    if (arrived == expected) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      for (unsigned int polls = 0;; ++polls) {
        if (atomicAdd(&bar->gen, 0u) != gen) break;
        if (atomicAdd(&bar->abort, 0u) != 0u) {
          ok = 0;
          break;
        }
        if (polls >= (1u << 24) || global_ns() - t0 > budget_ns) {
          atomicOr(&bar->status, kBarrierTimeout);
          atomicExch(&bar->abort, 1u);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// All `steps` batch steps in one cooperative launch: blocks stride over the
// tile list, then meet at the grid barrier before the next step reads the
// populations other blocks have just written (coherent loads).
template <int PREC, bool DFARITH>
__global__ void __launch_bounds__(128, PREC == LBM_FP32_SHIFTED ? 5 : 0) batch_persistent_kernel(const BatchEntry* __restrict__ ent,
                                                               const long long* __restrict__ tile_start,
                                                               const int* __restrict__ tile_lattice,
                                                               long long tiles, int parity0, int steps,
                                                               GridBarrier* bar, unsigned long long budget_ns) {
  __shared__ __align__(16) LatticeArgs sa;
  __shared__ const void* s_src;
  __shared__ void* s_dst;
  for (int st = 0; st < steps; ++st) {
    const int parity = (parity0 + st) & 1;
    for (long long b = blockIdx.x; b < tiles; b += gridDim.x)
      batch_tile<PREC, 32, 4, DFARITH, true, 8>(ent, tile_start, tile_lattice, parity, b, sa, s_src, s_dst);
    if (st + 1 < steps && !grid_barrier(bar, gridDim.x, budget_ns)) return;
  }
}

// The persistent form of the parameter-table kernel (FP32-store batches of
// at most kParamLattices lattices): each step, blocks stride over the tile
// list and then over the edge sites, and meet at the bounded grid barrier;
// loads go through L2 (other blocks wrote the state in the previous step).
__global__ void __launch_bounds__(128, 4) batch_param_persistent_kernel(const __grid_constant__ ParamTable t,
                                                                        const __grid_constant__ LatticeArgs m,
                                                                        long long tiles, long long edges,
                                                                        int parity0, int steps, GridBarrier* bar,
                                                                        unsigned long long budget_ns) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int st = 0; st < steps; ++st) {
    const int parity = (parity0 + st) & 1;
    for (long long b = blockIdx.x; b < tiles; b += gridDim.x) param_tile<32, 4, 8, true>(t, m, parity, b);
    for (long long j = blockIdx.x * 128LL + tid; j < edges; j += gridDim.x * 128LL) param_edge<true>(t, parity, j);
    if (st + 1 < steps && !grid_barrier(bar, gridDim.x, budget_ns)) return;
  }
}

// Self-test of the bounded wait: the barrier expects one block more than the
// grid has, so it can never fill and must time out.
__global__ void barrier_selftest_kernel(GridBarrier* bar, unsigned long long budget_ns) {
  grid_barrier(bar, gridDim.x + 1u, budget_ns);
}

template <int PREC, int I>
cudaError_t launch_tile_i(long long blocks, const BatchEntry* ent, const long long* ts, const int* tl, int parity,
                          cudaStream_t s) {
  constexpr int BX = kTileBX[I], BY = kTileBY[I], RW = kTileRows[I];
  if constexpr (PREC == LBM_FP64_DF)
    batch_step_kernel<LBM_FP64, BX, BY, true, RW><<<(unsigned)blocks, dim3(BX, BY), 0, s>>>(ent, ts, tl, parity);
  else
    batch_step_kernel<PREC, BX, BY, false, RW><<<(unsigned)blocks, dim3(BX, BY), 0, s>>>(ent, ts, tl, parity);
  return cudaGetLastError();
}

// The wall rows (batch_edge_kernel) run on the side stream `aux`, forked
// from and joined back to `s` around the interior launch: the two write
// disjoint sites of the same step and may overlap.
cudaError_t launch_param_tile(int i, const ParamTable& t, long long blocks, long long edges, const LatticeArgs& m,
                              int parity, cudaStream_t s, cudaStream_t aux, cudaEvent_t ev_fork,
                              cudaEvent_t ev_join) {
  if (edges > 0) {
    cudaError_t e = cudaEventRecord(ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev_fork, 0);
    if (e != cudaSuccess) return e;
    batch_edge_kernel<<<(unsigned)((edges + 127) / 128), 128, 0, aux>>>(t, m, parity, edges);
    e = cudaGetLastError();
    const cudaError_t r = cudaEventRecord(ev_join, aux);  // joined back below, also after an error
    if (e != cudaSuccess) {
      cudaStreamWaitEvent(s, ev_join, 0);
      return e;
    }
    if (r != cudaSuccess) return r;
  }
  const auto join = [&](cudaError_t e) {
    const cudaError_t w = edges > 0 ? cudaStreamWaitEvent(s, ev_join, 0) : cudaSuccess;
    return e != cudaSuccess ? e : w;
  };
  if (blocks <= 0) return join(cudaSuccess);
  const dim3 grid((unsigned)blocks), block(32, 4);
  if (kParamRows[i] == 1)
    batch_param_kernel<32, 4, 1><<<grid, block, 0, s>>>(t, m, parity);
  else if (kParamRows[i] == 4)
    batch_param_kernel<32, 4, 4><<<grid, block, 0, s>>>(t, m, parity);
  else
    batch_param_kernel<32, 4, 8><<<grid, block, 0, s>>>(t, m, parity);
  return join(cudaGetLastError());
}

template <int PREC>
cudaError_t launch_tile(int tile, long long blocks, const BatchEntry* ent, const long long* ts, const int* tl,
                        int parity, cudaStream_t s) {
  switch (tile) {
    case 0: return launch_tile_i<PREC, 0>(blocks, ent, ts, tl, parity, s);
    case 1: return launch_tile_i<PREC, 1>(blocks, ent, ts, tl, parity, s);
    case 2: return launch_tile_i<PREC, 2>(blocks, ent, ts, tl, parity, s);
    case 3: return launch_tile_i<PREC, 3>(blocks, ent, ts, tl, parity, s);
    case 4: return launch_tile_i<PREC, 4>(blocks, ent, ts, tl, parity, s);
    case 5: return launch_tile_i<PREC, 5>(blocks, ent, ts, tl, parity, s);
    case 6: return launch_tile_i<PREC, 6>(blocks, ent, ts, tl, parity, s);
    case 7: return launch_tile_i<PREC, 7>(blocks, ent, ts, tl, parity, s);
    default: return launch_tile_i<PREC, 8>(blocks, ent, ts, tl, parity, s);
  }
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_batch {
  int n;
  int precision;
  cudaStream_t stream;
  cudaStream_t capture;
  std::vector<LatticeArgs> args;
  std::vector<void*> fa, fb;
  BatchEntry* d_ent;
  long long* d_tiles[kTiles];  // tile offsets per shape
  int* d_tile_lat[kTiles];     // per shape: the lattice of every tile
  long long blocks[kTiles];
  int tile;
  int parity;
  long long sites;
  std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;  // (n, parity, tile)
  cudaStream_t aux[kAux];  // per-lattice launches: the lattices' streams
  cudaEvent_t ev_fork, ev_join;  // the wall-row launch of the parameter-table candidates
  std::vector<int> order;  // lattices by decreasing size
  std::vector<int> lane;   // stream of each lattice (balanced by sites)
  GridBarrier* d_bar;  // persistent-kernel barrier state
  // parameter-table candidates: usable for FP32-store batches whose lattices
  // all have 32-bit offsets; one table and block count per group of lattices
  bool param_ok;
  std::vector<ParamTable> ptab[kParamTiles];
  std::vector<long long> pblocks[kParamTiles];
  std::vector<long long> pedges[kParamTiles];
  char err[512];
};

namespace {

int bfail(lbm_batch* b, int code, const char* fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(b->err, sizeof b->err, fmt, ap);
    va_end(ap);
  }
  return code;
}

int bcuda(lbm_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LBM_OK;
  return bfail(b, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// The shared-memory tile shape with the same threads and rows as parameter
// candidate i (used where the parameter tables do not apply).
constexpr int param_fallback(int i) { return kParamRows[i] == 1 ? 0 : kParamRows[i] == 4 ? 7 : 8; }

cudaError_t launch_batch(const lbm_batch* b, int parity, cudaStream_t s) {
  int t = b->tile;
  if (t >= kParamFirst) {
    const int i = t - kParamFirst;
    if (b->param_ok) {
      for (size_t g = 0; g < b->ptab[i].size(); ++g) {
        const cudaError_t e =
            launch_param_tile(i, b->ptab[i][g], b->pblocks[i][g], b->pedges[i][g], b->args[0], parity, s,
                              b->aux[0], b->ev_fork, b->ev_join);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
    t = param_fallback(i);
  }
  if (b->precision == LBM_FP64_DF)
    return launch_tile<LBM_FP64_DF>(t, b->blocks[t], b->d_ent, b->d_tiles[t], b->d_tile_lat[t], parity, s);
  if (b->precision == LBM_FP64)
    return launch_tile<LBM_FP64>(t, b->blocks[t], b->d_ent, b->d_tiles[t], b->d_tile_lat[t], parity, s);
  return launch_tile<LBM_FP32_SHIFTED>(t, b->blocks[t], b->d_ent, b->d_tiles[t], b->d_tile_lat[t], parity, s);
}

void free_batch(lbm_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
  for (int t = 0; t < kTiles; ++t) {
    if (b->d_tiles[t]) cudaFree(b->d_tiles[t]);
    if (b->d_tile_lat[t]) cudaFree(b->d_tile_lat[t]);
  }
  if (b->d_ent) cudaFree(b->d_ent);
  if (b->d_bar) cudaFree(b->d_bar);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (int k = 0; k < kAux; ++k)
    if (b->aux[k]) cudaStreamDestroy(b->aux[k]);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  delete b;
}

// Capture n steps of every lattice, one single-lattice kernel launch per
// lattice and step, on the lattices' streams (forked from and joined back to
// the capture stream).  A lattice's steps stay in order on its stream; the
// lattices run concurrently.
cudaError_t capture_per_lattice(lbm_batch* b, int n) {
  cudaEvent_t fork = nullptr, join[kAux] = {};
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int k = 0; k < kAux && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(fork, b->capture);
  bool forked[kAux] = {};
  for (int k = 0; k < kAux && e == cudaSuccess; ++k) {
    e = cudaStreamWaitEvent(b->aux[k], fork, 0);
    forked[k] = e == cudaSuccess;
  }
  for (size_t j = 0; j < b->order.size() && e == cudaSuccess; ++j) {
    const int i = b->order[j];
    int p = b->parity;
    for (int t = 0; t < n && e == cudaSuccess; ++t) {
      e = launch_step(b->precision, true, p ? b->fb[i] : b->fa[i], p ? b->fa[i] : b->fb[i], b->args[i],
                      b->aux[b->lane[i]]);
      p ^= 1;
    }
  }
  // join every stream that was forked, also after an error, so the capture
  // can end
  for (int k = 0; k < kAux; ++k) {
    if (!forked[k]) continue;
    const cudaError_t r = cudaEventRecord(join[k], b->aux[k]);
    const cudaError_t w = r == cudaSuccess ? cudaStreamWaitEvent(b->capture, join[k], 0) : r;
    if (e == cudaSuccess) e = w;
  }
  for (int k = 0; k < kAux; ++k)
    if (join[k]) cudaEventDestroy(join[k]);
  if (fork) cudaEventDestroy(fork);
  return e;
}

// Graph of n batch steps starting at parity p with the current tile shape.
int get_graph(lbm_batch* b, int n, cudaGraphExec_t* out) {
  auto key = std::make_tuple(n, b->parity, b->tile);
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    *out = it->second;
    return LBM_OK;
  }
  cudaGraph_t g = nullptr;
  int rc = bcuda(b, cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "graph capture");
  if (rc) return rc;
  cudaError_t le = cudaSuccess;
  if (b->tile == kPerLattice) {
    le = capture_per_lattice(b, n);
  } else {
    int p = b->parity;
    for (int i = 0; i < n && le == cudaSuccess; ++i) {
      le = launch_batch(b, p, b->capture);
      p ^= 1;
    }
  }
  cudaError_t ee = cudaStreamEndCapture(b->capture, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bcuda(b, le, "batch launch during capture");
  }
  rc = bcuda(b, ee, "graph end capture");
  if (rc) return rc;
  cudaGraphExec_t exec = nullptr;
  rc = bcuda(b, cudaGraphInstantiate(&exec, g, 0), "graph instantiate");
  cudaGraphDestroy(g);
  if (rc) return rc;
  b->graphs[key] = exec;
  *out = exec;
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_tile_count(void) { return kCandidates; }

int lbm_batch_tile_shape(int i, int* bx, int* by) {
  if (i < 0 || i >= kCandidates || !bx || !by) return LBM_ERR_INVALID;
  *bx = i >= kPerLattice ? 32 : kTileBX[i];  // per-lattice and parameter candidates: 32 x 4 blocks
  *by = i >= kPerLattice ? 4 : kTileBY[i];
  return LBM_OK;
}

int lbm_batch_tile_rows(int i) {
  if (i < 0 || i >= kCandidates) return LBM_ERR_INVALID;
  return i == kPerLattice ? 1 : i >= kParamFirst ? kParamRows[i - kParamFirst] : kTileRows[i];
}

int lbm_batch_tile_kind(int i) {
  if (i < 0 || i >= kCandidates) return LBM_ERR_INVALID;
  return i == kPerLattice ? LBM_BATCH_PER_LATTICE : i >= kParamFirst ? LBM_BATCH_PARAM_TILES : LBM_BATCH_SHARED_TILES;
}

int lbm_batch_tile_per_lattice(int i) {
  if (i < 0 || i >= kCandidates) return LBM_ERR_INVALID;
  return i == kPerLattice ? 1 : 0;
}

int lbm_batch_create(lbm_batch** out, int n, const lbm_lattice_desc* descs, int precision, void* stream) {
  if (!out) return LBM_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || !descs) return LBM_ERR_INVALID;
  if (precision != LBM_FP64 && precision != LBM_FP32_SHIFTED && precision != LBM_FP64_DF) return LBM_ERR_INVALID;
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ERR_INVALID;
  b->n = n;
  b->precision = precision;
  b->stream = static_cast<cudaStream_t>(stream);
  b->args.resize(n);
  b->fa.resize(n);
  b->fb.resize(n);
  b->sites = 0;
  for (int i = 0; i < n; ++i) {
    const lbm_lattice_desc& d = descs[i];
    lbm_params p{d.lx, d.ly, precision, 0, d.tau, d.g, d.t_top, d.t_bottom, d.rho0};
    int rc = make_lattice_args(p, &b->args[i], b->err, sizeof b->err);
    if (rc != LBM_OK || !d.f_a || !d.f_b || d.f_a == d.f_b) {
      free_batch(b);
      return rc != LBM_OK ? rc : LBM_ERR_INVALID;
    }
    b->fa[i] = d.f_a;
    b->fb[i] = d.f_b;
    b->sites += (long long)d.lx * d.ly;
  }
  std::vector<BatchEntry> h(n);
  for (int i = 0; i < n; ++i) {
    h[i].a = b->args[i];
    h[i].f[0] = b->fa[i];
    h[i].f[1] = b->fb[i];
  }
  if (cudaMalloc(&b->d_ent, sizeof(BatchEntry) * n) != cudaSuccess ||
      cudaMemcpy(b->d_ent, h.data(), sizeof(BatchEntry) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return LBM_ERR_CUDA;
  }
  for (int t = 0; t < kTiles; ++t) {
    std::vector<long long> ts(n + 1, 0);
    for (int i = 0; i < n; ++i) {
      const int rows = kTileBY[t] * kTileRows[t];
      const long long tiles = (long long)((b->args[i].lx + kTileBX[t] - 1) / kTileBX[t]) *
                              ((b->args[i].ly + rows - 1) / rows);
      ts[i + 1] = ts[i] + tiles;
    }
    b->blocks[t] = ts[n];
    if (ts[n] >= (1LL << 31) || cudaMalloc(&b->d_tiles[t], sizeof(long long) * (n + 1)) != cudaSuccess ||
        cudaMemcpy(b->d_tiles[t], ts.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return LBM_ERR_CUDA;
    }
    std::vector<int> owner((size_t)ts[n]);
    for (int i = 0; i < n; ++i)
      for (long long k = ts[i]; k < ts[i + 1]; ++k) owner[(size_t)k] = i;
    if (cudaMalloc(&b->d_tile_lat[t], sizeof(int) * owner.size()) != cudaSuccess ||
        cudaMemcpy(b->d_tile_lat[t], owner.data(), sizeof(int) * owner.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return LBM_ERR_CUDA;
    }
  }
  // parameter tables (FP32-store, 32-bit offsets)
  b->param_ok = precision == LBM_FP32_SHIFTED;
  for (int i = 0; i < n; ++i) b->param_ok = b->param_ok && b->args[i].idx32;
  if (b->param_ok) {
    for (int t = 0; t < kParamTiles; ++t) {
      for (int g0 = 0; g0 < n; g0 += kParamLattices) {
        ParamTable tab;
        std::memset(&tab, 0, sizeof tab);
        tab.n = std::min(kParamLattices, n - g0);
        long long start = 0, edges = 0;
        for (int k = 0; k < tab.n; ++k) {
          const int i = g0 + k;
          const LatticeArgs& a = b->args[i];
          ParamLat& e = tab.e[k];
          const int rows = 4 * kParamRows[t];
          e.tile_start = start;
          e.edge_start = edges;
          edges += edge_sites(a.lx, a.ly);
          e.tiles_x = (a.lx + 31) / 32;
          start += (long long)e.tiles_x * ((a.ly + rows - 1) / rows);
          e.f[0] = b->fa[i];
          e.f[1] = b->fb[i];
          e.args = &b->d_ent[i].a;
          e.lx = a.lx;
          e.ly = a.ly;
          e.omega_f = a.omega_f;
          e.omc_f = a.omc_f;
          for (int c = 0; c < 2; ++c) {
            e.df_rho0[c] = a.df_rho0[c];
            e.df_e0[c] = a.df_e0[c];
            e.df_tshift[c] = a.df_tshift[c];
            e.df_taug_r[c] = a.df_taug_r[c];
            e.df_g_r[c] = a.df_g_r[c];
          }
          for (int l = 0; l < NPOP; ++l) {
            e.pull_off[l] = (int)a.pull_off[l];
            e.plane_off[l] = (int)a.plane_off[l];
          }
        }
        b->ptab[t].push_back(tab);
        b->pblocks[t].push_back(start);
        b->pedges[t].push_back(edges);
      }
    }
  }
  if (cudaMalloc(&b->d_bar, sizeof(GridBarrier)) != cudaSuccess ||
      cudaMemset(b->d_bar, 0, sizeof(GridBarrier)) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return LBM_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return LBM_ERR_CUDA;
  }
  for (int k = 0; k < kAux; ++k) {
    if (cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return LBM_ERR_CUDA;
    }
  }
  if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return LBM_ERR_CUDA;
  }
  // per-lattice launches: largest lattices first, each to the stream with the
  // fewest sites so far
  b->order.resize(n);
  b->lane.assign(n, 0);
  for (int i = 0; i < n; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int p, int q) {
    return (long long)b->args[p].lx * b->args[p].ly > (long long)b->args[q].lx * b->args[q].ly;
  });
  {
    long long load[kAux] = {};
    for (int i : b->order) {
      int k = 0;
      for (int m = 1; m < kAux; ++m)
        if (load[m] < load[k]) k = m;
      b->lane[i] = k;
      load[k] += (long long)b->args[i].lx * b->args[i].ly;
    }
  }
  b->tile = 0;
  b->parity = 0;
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : "null batch"; }

int lbm_batch_init(lbm_batch* b, int i, const double* rho, const double* ux, const double* uy, const double* T) {
  if (!b) return LBM_ERR_INVALID;
  if (i < 0 || i >= b->n || !rho || !ux || !uy || !T) return bfail(b, LBM_ERR_INVALID, "lbm_batch_init: bad args");
  void* cur = b->parity ? b->fb[i] : b->fa[i];
  return bcuda(b, launch_init(storage_prec(b->precision), cur, rho, ux, uy, T, b->args[i], b->stream), "lbm_batch_init");
}

int lbm_batch_set_tile(lbm_batch* b, int tile) {
  if (!b) return LBM_ERR_INVALID;
  if (tile < 0 || tile >= kCandidates) return bfail(b, LBM_ERR_INVALID, "tile %d out of range", tile);
  b->tile = tile;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int n) {
  if (!b) return LBM_ERR_INVALID;
  if (n < 0) return bfail(b, LBM_ERR_INVALID, "lbm_batch_step: n < 0");
  if (n == 0) return LBM_OK;
  cudaGraphExec_t exec;
  int rc = get_graph(b, n, &exec);
  if (rc) return rc;
  rc = bcuda(b, cudaGraphLaunch(exec, b->stream), "graph launch");
  if (rc) return rc;
  b->parity ^= (n & 1);
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int steps, int* best, double* times_ms) {
  if (!b) return LBM_ERR_INVALID;
  if (steps < 1 || !best) return bfail(b, LBM_ERR_INVALID, "lbm_batch_autotune: bad args");
  cudaEvent_t e0, e1;
  int rc = bcuda(b, cudaEventCreate(&e0), "event");
  if (rc) return rc;
  rc = bcuda(b, cudaEventCreate(&e1), "event");
  if (rc) {
    cudaEventDestroy(e0);
    return rc;
  }
  double best_t = 1e300;
  int best_i = 0;
  for (int t = 0; t < kCandidates && rc == LBM_OK; ++t) {
    b->tile = t;
    rc = lbm_batch_step(b, 1);  // warm-up (and graph capture of the 1-step graph)
    cudaGraphExec_t exec;
    if (!rc) rc = get_graph(b, steps, &exec);
    if (!rc) rc = bcuda(b, cudaEventRecord(e0, b->stream), "event record");
    if (!rc) rc = lbm_batch_step(b, steps);
    if (!rc) rc = bcuda(b, cudaEventRecord(e1, b->stream), "event record");
    if (!rc) rc = bcuda(b, cudaEventSynchronize(e1), "event sync");
    float ms = 0.f;
    if (!rc) rc = bcuda(b, cudaEventElapsedTime(&ms, e0, e1), "event time");
    if (!rc) {
      const double per = ms / steps;
      if (times_ms) times_ms[t] = per;
      if (per < best_t) {
        best_t = per;
        best_i = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->tile = best_i;
  *best = best_i;
  return LBM_OK;
}

void* lbm_batch_current(const lbm_batch* b, int i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->parity ? b->fb[i] : b->fa[i];
}

int lbm_batch_moments(lbm_batch* b, int i, double* rho, double* ux, double* uy, double* T) {
  if (!b) return LBM_ERR_INVALID;
  if (i < 0 || i >= b->n) return bfail(b, LBM_ERR_INVALID, "lbm_batch_moments: bad index");
  return bcuda(b, launch_moments(storage_prec(b->precision), lbm_batch_current(b, i), rho, ux, uy, T, b->args[i], b->stream),
               "lbm_batch_moments");
}

long long lbm_batch_sites(const lbm_batch* b) { return b ? b->sites : 0; }

int lbm_batch_status(lbm_batch* b) {
  if (!b) return LBM_ERR_INVALID;
  int rc = bcuda(b, cudaStreamSynchronize(b->stream), "lbm_batch_status");
  if (rc) return rc;
  GridBarrier h;
  rc = bcuda(b, cudaMemcpy(&h, b->d_bar, sizeof h, cudaMemcpyDeviceToHost), "lbm_batch_status");
  if (rc) return rc;
  if (h.status & kBarrierTimeout) return bfail(b, LBM_ERR_TIMEOUT, "persistent step: grid barrier wait timed out");
  return LBM_OK;
}

}  // extern "C"

namespace {
template <int PREC, bool DF>
int launch_persistent(lbm_batch* b, int n, unsigned long long budget_ns) {
  auto kernel = batch_persistent_kernel<PREC, DF>;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  int rc = bcuda(b, cudaGetDevice(&dev), "persistent step");
  if (!rc) rc = bcuda(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "persistent step");
  if (!rc) rc = bcuda(b, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev), "persistent step");
  if (!rc) rc = bcuda(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0), "persistent step");
  if (rc) return rc;
  if (!coop || per_sm < 1) return bfail(b, LBM_ERR_INVALID, "persistent step: cooperative launch unavailable");
  const long long tiles = b->blocks[8];  // the 32 x 4 x 8 tiling
  const unsigned int grid = (unsigned int)std::min<long long>((long long)per_sm * sms, tiles);
  rc = bcuda(b, cudaMemsetAsync(b->d_bar, 0, sizeof(GridBarrier), b->stream), "persistent step");
  if (rc) return rc;
  const BatchEntry* ent = b->d_ent;
  const long long* ts = b->d_tiles[8];
  const int* tl = b->d_tile_lat[8];
  int parity = b->parity, steps = n;
  GridBarrier* bar = b->d_bar;
  void* args[] = {(void*)&ent, (void*)&ts, (void*)&tl, (void*)&tiles, (void*)&parity, (void*)&steps, (void*)&bar,
                  (void*)&budget_ns};
  return bcuda(b, cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(32, 4), args, 0, b->stream),
               "persistent step");
}
// The parameter-table persistent kernel: one group, the 32 x 4 x 8 tiling.
int launch_param_persistent(lbm_batch* b, int n, unsigned long long budget_ns) {
  static_assert(kParamRows[kParamTiles - 1] == 8, "the persistent kernel uses the 8-row tiling");
  auto kernel = batch_param_persistent_kernel;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  int rc = bcuda(b, cudaGetDevice(&dev), "persistent step");
  if (!rc) rc = bcuda(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "persistent step");
  if (!rc) rc = bcuda(b, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev), "persistent step");
  if (!rc) rc = bcuda(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0), "persistent step");
  if (rc) return rc;
  if (!coop || per_sm < 1) return bfail(b, LBM_ERR_INVALID, "persistent step: cooperative launch unavailable");
  const ParamTable& t = b->ptab[kParamTiles - 1][0];
  long long tiles = b->pblocks[kParamTiles - 1][0], edges = b->pedges[kParamTiles - 1][0];
  const unsigned int grid = (unsigned int)std::max<long long>(
      1, std::min<long long>((long long)per_sm * sms, std::max(tiles, (edges + 127) / 128)));
  rc = bcuda(b, cudaMemsetAsync(b->d_bar, 0, sizeof(GridBarrier), b->stream), "persistent step");
  if (rc) return rc;
  const LatticeArgs& m = b->args[0];
  int parity = b->parity, steps = n;
  GridBarrier* bar = b->d_bar;
  void* args[] = {(void*)&t, (void*)&m, (void*)&tiles, (void*)&edges, (void*)&parity, (void*)&steps, (void*)&bar,
                  (void*)&budget_ns};
  return bcuda(b, cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(32, 4), args, 0, b->stream),
               "persistent step");
}
}  // namespace

extern "C" {

int lbm_batch_step_persistent(lbm_batch* b, int n) {
  if (!b) return LBM_ERR_INVALID;
  if (n < 0) return bfail(b, LBM_ERR_INVALID, "lbm_batch_step_persistent: n < 0");
  if (n == 0) return LBM_OK;
  const unsigned long long budget = 2000000000ull;  // 2 s per barrier wait
  int rc;
  if (b->param_ok && b->ptab[kParamTiles - 1].size() == 1)
    rc = launch_param_persistent(b, n, budget);
  else if (b->precision == LBM_FP64_DF)
    rc = launch_persistent<LBM_FP64, true>(b, n, budget);
  else if (b->precision == LBM_FP64)
    rc = launch_persistent<LBM_FP64, false>(b, n, budget);
  else
    rc = launch_persistent<LBM_FP32_SHIFTED, false>(b, n, budget);
  if (rc) return rc;
  b->parity ^= (n & 1);
  return LBM_OK;
}

int lbm_batch_barrier_selftest(lbm_batch* b, int budget_ms) {
  if (!b) return LBM_ERR_INVALID;
  if (budget_ms < 1 || budget_ms > 10000) return bfail(b, LBM_ERR_INVALID, "budget_ms out of range");
  int rc = bcuda(b, cudaMemsetAsync(b->d_bar, 0, sizeof(GridBarrier), b->stream), "barrier self-test");
  if (rc) return rc;
  GridBarrier* bar = b->d_bar;
  unsigned long long budget = (unsigned long long)budget_ms * 1000000ull;
  void* args[] = {(void*)&bar, (void*)&budget};
  rc = bcuda(b, cudaLaunchCooperativeKernel((const void*)barrier_selftest_kernel, dim3(2), dim3(32, 4), args, 0,
                                            b->stream), "barrier self-test");
  if (rc) return rc;
  rc = lbm_batch_status(b);  // LBM_ERR_TIMEOUT when the bounded wait gave up
  cudaMemsetAsync(b->d_bar, 0, sizeof(GridBarrier), b->stream);
  cudaStreamSynchronize(b->stream);
  return rc;
}

}  // extern "C"
