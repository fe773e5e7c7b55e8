/*
 * ttprobe -- measured arithmetic peaks of the current GPU, the denominators of
 * the pricer's roofline fractions.  The paper has no counterpart: its method is
 * bound by plain FP32 (mixed path) or FP64 arithmetic on the CUDA cores, and
 * the only measured peaks at hand are a memory copy and a BF16 matrix product.
 *
 * tt_probe_fma_peak runs a kernel of independent fused multiply-adds (eight
 * chains per thread, 4 resident CTAs of 256 threads per SM, every SM) long
 * enough to time, and returns the best of `reps` timed launches in TFLOP/s
 * (2 flops per FMA).  precision: 0 = FP64, 1 = FP32.  Runs on the current CUDA
 * device and the legacy default stream, and synchronises.  Allocates one
 * small device buffer per call (the sink that keeps the chains live).
 * Returns 0, or -1 on a bad argument, -5 on a CUDA error.
 */
#ifndef TTPROBE_H
#define TTPROBE_H

#ifdef __cplusplus
extern "C" {
#endif

int tt_probe_fma_peak(int precision, int reps, double* tflops);

#ifdef __cplusplus
}
#endif

#endif /* TTPROBE_H */
