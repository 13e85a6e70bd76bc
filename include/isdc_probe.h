/*
 * isdc_probe.h -- measurement of the GPU's FP64 issue rate (libisdc_probe.so).
 *
 * Not from the paper: the paper reports no timings.  The number is the peak
 * against which the FP64-bound kernels of the library (stencils, right-hand
 * side, sweep end) are reported as a fraction ("alu" roofline).
 */
#ifndef ISDC_PROBE_H
#define ISDC_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/*
 * On the current device, launches kernels of independent FP64 FMA chains on
 * a private stream (4, 8 or 16 chains per thread, 4, 8 or 16 blocks of 256
 * threads per SM, about 10 G FMAs per launch; one warm-up round and three
 * timed rounds over the nine shapes) and returns the best rate in *ops_per_s
 * (one FMA = one FP64 operation) and that launch's time in *ms_best (may be
 * NULL).  Synchronises.  Allocates nothing.
 * Returns 0, 1 for a NULL ops_per_s, 2 for a CUDA error.
 */
int isdc_probe_fp64_rate(double *ops_per_s, double *ms_best);

#ifdef __cplusplus
}
#endif

#endif
