/*
 * mcpeaks.h - microbenchmarks that measure the issue-rate peaks the photon
 * walk is bounded by (single-precision FMA, 32-bit integer multiply-add, the
 * special-function unit, shared-memory bandwidth). They complement the copy
 * bandwidth and tensor-core figures measured elsewhere; the walk itself never
 * calls them. Not part of the method: the paper has no counterpart.
 *
 * mc_peak_run launches `blocks` CTAs of `threads` threads running kernel
 * `kind` for `iters` inner iterations on `stream` (asynchronous) and writes
 * to *ops the number of operations that launch performs (thread-level FMAs,
 * integer multiply-adds, special-function ops, or shared-memory bytes).
 * d_sink: device scratch of at least blocks*threads floats (results land
 * there so nothing is optimised away). Returns 0, or -1 on bad arguments,
 * or -2 on a launch error.
 */
#ifndef MCPEAKS_H
#define MCPEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_PEAK_FFMA 0   /* fmaf, 8 independent chains per thread   */
#define MC_PEAK_IMAD 1   /* 32-bit integer multiply-add chains      */
#define MC_PEAK_MUFU 2   /* rsqrt.approx chains (special-function)  */
#define MC_PEAK_SMEM 3   /* 16-byte shared-memory loads             */
#define MC_PEAK_IMULWIDE 4 /* 32x32->64 multiplies (Philox round) */

int mc_peak_run(int kind, int blocks, int threads, int iters, float *d_sink, double *ops, void *stream);

#ifdef __cplusplus
}
#endif
#endif
