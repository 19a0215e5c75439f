/*
 * Throughput probes for the roofline denominators of the IFGF kernels (a library of its own,
 * libifgf_peaks; the IFGF library does not depend on it).
 *
 * Each probe runs independent dependency chains on every SM of the current device for a few
 * milliseconds and reports operations per second measured with CUDA events: FP32 FFMA, packed
 * FP32x2 FFMA2, FP64 DFMA, the special-function unit (sine) and TF32 mma.sync (m16n8k8).
 */
#ifndef IFGF_PEAKS_H
#define IFGF_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/*
 * out: host array of 6 doubles, written as
 *   out[0] FP32 FFMA TFLOP/s, out[1] FP32x2 FFMA2 TFLOP/s, out[2] FP64 DFMA TFLOP/s,
 *   out[3] sine operations per second / 1e9, out[4] TF32 mma.sync TFLOP/s, out[5] SM count.
 * Synchronous; allocates and frees a small device buffer.  Returns 0, or the CUDA error code of
 * the first failing call (out is then partly written).
 */
int ifgf_peaks_measure(double* out);

#ifdef __cplusplus
}
#endif

#endif /* IFGF_PEAKS_H */
