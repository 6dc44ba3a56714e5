// FMA throughput probe and the site reciprocal (include/lbm_probe.h).
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "../../include/lbm_probe.h"
#include "lbm_device.cuh"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void fma_probe_kernel(T* out, int iters, T b, T c) {
  T acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = fma(acc[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i];
  if (s == (T)12345.678) out[0] = s;  // keeps the chains alive; practically never taken
}

__global__ void rcp_probe_kernel(const double* __restrict__ x, double* __restrict__ y, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = lbm::rcp_nr(x[i]);
}

}  // namespace

extern "C" int lbm_probe_rcp(void* stream, const double* x, double* y, long long n) {
  if (n < 0 || (n > 0 && (!x || !y))) return LBM_ERR_INVALID;
  if (n == 0) return LBM_OK;
  const long long blocks = (n + 255) / 256;
  if (blocks > 0x7fffffffLL) return LBM_ERR_INVALID;
  rcp_probe_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

extern "C" int lbm_probe_fma(void* stream, int iters, int fp32, double* tflops, double* ms) {
  if (iters < 1 || !tflops || !ms) return LBM_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LBM_ERR_CUDA;
  const int threads = 256, blocks = sms * 8;
  void* out = nullptr;
  if (cudaMalloc(&out, 16) != cudaSuccess) return LBM_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // warm-up launch, then the timed one
  for (int rep = 0; rep < 2; ++rep) {
    if (rep == 1) cudaEventRecord(e0, s);
    if (fp32)
      fma_probe_kernel<float><<<blocks, threads, 0, s>>>(static_cast<float*>(out), iters, 0.999999f, 1e-7f);
    else
      fma_probe_kernel<double><<<blocks, threads, 0, s>>>(static_cast<double*>(out), iters, 0.999999, 1e-7);
  }
  cudaEventRecord(e1, s);
  cudaError_t err = cudaEventSynchronize(e1);
  float t = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return LBM_ERR_CUDA;
  *ms = t;
  *tflops = 2.0 * kChains * (double)iters * threads * blocks / (t * 1e-3) / 1e12;
  return LBM_OK;
}
