/*
 * m2l_peaks.h - FMA-throughput probe used as the roofline denominator of the CUDA-core kernels
 * of the M2L library (the FP64 and FP32 contractions and Hadamard products). The paper has no
 * counterpart; it measures the GPU the library runs on.
 *
 * GB300 lists no FP64 or FP32 CUDA-core rate that the library can read at run time, and its
 * FP64 units run far below the tensor cores, so the fraction of peak that a CUDA-core kernel
 * reaches is taken against this measured rate: independent FMA chains in every thread of a
 * grid that fills every SM, timed with CUDA events.
 */
#ifndef M2L_PEAKS_H
#define M2L_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* Measure the FMA throughput of the current device in TFLOP/s (2 flops per FMA).
 * fp64: 1 for double-precision FMAs, 0 for single precision.
 * iters: loop trips per thread (each trip issues 128 FMAs in 8 independent chains); >= 1.
 * reps: timed launches after one untimed warm-up launch; 1..64.
 * best, median: receive the fastest and the median launch's rate (TFLOP/s); either may be NULL.
 * ms_best: receives the duration of the fastest launch in milliseconds (may be NULL).
 * Synchronous on the legacy default stream. Allocates one small device buffer (freed before it
 * returns). Returns 0, or -1 on a bad argument, -3 on a CUDA error. */
int m2l_fma_peak(int fp64, long long iters, int reps, double *best, double *median, double *ms_best);

#ifdef __cplusplus
}
#endif

#endif /* M2L_PEAKS_H */
