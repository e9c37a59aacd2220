/*
 * nys_peak.h -- arithmetic-peak probes of the GPU (measurement utility).
 *
 * Not part of the solver and not a passage of the paper: the roofline fractions
 * that the benchmark reports for the solver's kernels divide their achieved
 * FLOP rate by the peak of the pipe each kernel's contraction runs on, and
 * these probes measure those peaks on the device at hand instead of assuming
 * nominal figures.  Each probe keeps one pipe busy with independent work:
 *   NYS_PEAK_FFMA      FP32 fused multiply-adds on the CUDA cores
 *   NYS_PEAK_DFMA      FP64 fused multiply-adds
 *   NYS_PEAK_TF32_MMA  tcgen05.mma kind::tf32, M = 128, N = 256, K = 8,
 *                      accumulators in tensor memory, operands in shared memory
 *   NYS_PEAK_BF16_MMA  tcgen05.mma kind::f16 with bf16 operands, M = 128,
 *                      N = 256, K = 16 (to compare with a cuBLAS bf16 figure)
 * One CTA per SM for the MMA probes (one thread issues, back to back into one
 * accumulator); 4 CTAs of 256 threads per SM for the FMA probes.
 *
 * nys_peak_launch enqueues one launch of probe `kind` with `iters` loop trips
 * on `stream` (cudaStream_t as void*, NULL = legacy default stream) and
 * returns NYS_PEAK_OK (0).  *flops_out (host) receives the floating-point
 * operations that launch performs (an FMA counts 2), so that the caller, which
 * times the launch with events on the same stream, gets the rate.
 * err_word (device int32, may be NULL) is set to 1 when an MMA probe's bounded
 * wait for its own MMAs gave up (the launch then still frees its tensor
 * memory and returns).
 * Errors (returned synchronously): -1 bad kind or iters <= 0, -3 CUDA error.
 * The probes change no device setting (clocks, power limits).
 */
#ifndef NYS_PEAK_H
#define NYS_PEAK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NYS_PEAK_FFMA = 0,
  NYS_PEAK_DFMA = 1,
  NYS_PEAK_TF32_MMA = 2,
  NYS_PEAK_BF16_MMA = 3
} nys_peak_kind;

int32_t nys_peak_launch(int32_t kind, int32_t iters, void* stream, int32_t* err_word,
                        double* flops_out);

#ifdef __cplusplus
}
#endif
#endif /* NYS_PEAK_H */
