/*
 * gmps_peaks.h -- peak-rate microbenchmarks (libgmps_peaks.so).
 *
 * Not part of the method: the paper reports no hardware rates.  These
 * launches measure the rates that bound the iterative-Grover kernels on the
 * GPU at hand -- FP64 FMA and FP32 FMA throughput over the whole chip and
 * shared-memory read bandwidth -- so that roofline fractions divide by a
 * measured peak.  The caller times the launch with CUDA events on `stream`.
 */
#ifndef GMPS_PEAKS_H
#define GMPS_PEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  GMPS_PEAK_FP64_FMA = 0,   /* work = flops (2 per FMA) */
  GMPS_PEAK_FP32_FMA = 1,   /* work = flops (2 per FMA) */
  GMPS_PEAK_SMEM_READ = 2   /* work = bytes read from shared memory; threads must be 256 */
};

/* Enqueue one measurement launch of `blocks` x `threads` threads (threads a
 * multiple of 32 in [32, 256]) running `trips` loop trips on `stream` (a
 * cudaStream_t or NULL).  sink: device memory of blocks*threads doubles,
 * written only if the computed value is impossible (it keeps the work from
 * being optimised away).  *work receives the launch's flops or bytes.
 * Returns 0 on success, 1 for invalid arguments, 2 if the launch failed. */
int gmps_peak_launch(int kind, int blocks, int threads, long long trips, void* stream, void* sink,
                     double* work);

#ifdef __cplusplus
}
#endif
#endif /* GMPS_PEAKS_H */
