/*
 * lbm_probe.h - throughput probe used by the benchmark to measure the
 * float64 FMA rate of the GPU it runs on (the roofline denominator of the
 * float64 collide, which is bound by the FP64 pipe rather than by HBM).
 * The paper quotes its efficiency E_c against peak double-precision rates
 * (Sect. 5, Table "comparison"); this measures that peak instead of
 * assuming it.
 */
#ifndef LBM_PROBE_H
#define LBM_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Run a kernel of independent float64 FMA chains on every SM for about
 * `iters` x 8 FMAs per thread (iters >= 1), timed with CUDA events on
 * `stream` (a cudaStream_t, NULL = legacy default stream).  Writes the
 * achieved rate in TFLOP/s (2 flops per FMA) to *tflops and the kernel time
 * in ms to *ms.  Synchronises the stream.  Returns 0 or a negative LBM_ERR_*
 * code.  `fp32` = 1 runs the same probe in float32. */
int lbm_probe_fma(void* stream, int iters, int fp32, double* tflops, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* LBM_PROBE_H */
