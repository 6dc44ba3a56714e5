/*
 * lbm_probe.h - a throughput probe used by the benchmark to measure the
 * float64 FMA rate of the GPU it runs on (the roofline denominator of the
 * float64 collide, which is bound by the FP64 pipe rather than by HBM; the
 * paper quotes its efficiency E_c against peak double-precision rates,
 * Sect. 5, Table "comparison", and this measures that peak instead of
 * assuming it), and the collide's own reciprocal 1/rho on arrays, for
 * tests of its error bound.
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

/* y[i] = 1 / x[i] as the float64 collide and adjoint form the site's 1/rho
 * (eq. 2: u = J / rho): a float32 seed from x's top 23 significand bits and
 * the approximate float32 reciprocal, then one third-order Newton-Raphson
 * correction y0 (1 + e + e^2), e = 1 - x y0, in float64 (within one unit in
 * the last place of 1/x for x in [2^-125, 2^126); NaN outside).  x and y are
 * device arrays of n float64 values (n >= 0), owned by the caller; the
 * launch is queued on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and not waited for.  Returns 0, LBM_ERR_INVALID for n < 0 or a
 * NULL array with n > 0, or LBM_ERR_CUDA if the launch fails.  For tests of
 * the reciprocal's error bound. */
int lbm_probe_rcp(void* stream, const double* x, double* y, long long n);

#ifdef __cplusplus
}
#endif

#endif /* LBM_PROBE_H */
