/*
 * lbm_probe.h -- measured arithmetic rates of the current GPU, the
 * denominators of the arithmetic rooflines of the step kernels.
 *
 * The paper has no counterpart: it names no hardware. The FP64 step of
 * include/lbm.h is bound by the FP64 units of the device, not by memory, so its
 * roofline needs the rate at which the device retires FP64 fused
 * multiply-adds; the double-word step (LBM_DF64) is bound by the FP32 units.
 * These probes measure both rates in the calling process, so that a benchmark
 * reports against the device it ran on rather than a data-sheet figure.
 */
#ifndef LBM_PROBE_H
#define LBM_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Kinds of fused multiply-add timed by lbm_probe_fma_rate. */
enum lbm_probe_kind {
  LBM_PROBE_FP64 = 0,      /* fma.rn.f64 */
  LBM_PROBE_FP32 = 1,      /* fma.rn.f32 */
  LBM_PROBE_FP32X2 = 2     /* fma.rn.f32x2: two FP32 lanes per instruction */
};

/* Times a kernel of independent fused multiply-add chains (8 per thread, 8
 * warps per block, 8 blocks per multiprocessor, every multiprocessor busy)
 * for `kind`, three launches of about `millis` ms each after one warm-up
 * launch, and writes the best rate in lane operations per second (one FMA of
 * one lane = 1; a paired f32x2 instruction counts 2) to *fma_per_s. Work is
 * issued on cuda_stream (NULL: legacy default stream) and the call
 * synchronises it. Allocates and frees a small device buffer (the chains'
 * results, so that the compiler keeps the arithmetic).
 * Returns LBM_OK, LBM_ERR_INVALID (bad kind, NULL output, millis outside
 * [1, 2000]) or LBM_ERR_CUDA. */
int lbm_probe_fma_rate(int kind, double millis, double* fma_per_s, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_PROBE_H */
