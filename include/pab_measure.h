/*
 * pab_measure.h - measurement aid shipped with libpab.
 *
 * The paper has no counterpart of this entry point: it only serves the
 * roofline of the bubble kernels by measuring how fast this GPU retires
 * fused multiply-adds in FP64 and in FP32.
 */
#ifndef PAB_MEASURE_H
#define PAB_MEASURE_H

#include <stdint.h>

#include "pab.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Throughput of dependent-free FMA streams: `blocks` CTAs of `threads`
 * threads each run 8 independent FMA chains of `iters` steps in FP64
 * (precision = PAB_FP64) or FP32 (PAB_MIXED), launched on `stream` and timed
 * with CUDA events.  Writes the kernel time in ms to *ms_out and the FMA
 * count (2 flops each) to *fma_out; the result of the chains goes to the
 * device scratch sink_dev (>= blocks*threads doubles, caller-owned) so that
 * nothing is optimised away.  Synchronises `stream`.
 * Errors: PAB_EINVAL (bad sizes or NULL pointers), PAB_ECUDA.
 */
pab_status pab_peak_fma(int32_t precision, int32_t blocks, int32_t threads, int32_t iters,
                        double *sink_dev, float *ms_out, double *fma_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PAB_MEASURE_H */
