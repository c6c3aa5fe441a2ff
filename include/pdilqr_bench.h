/*
 * pdilqr_bench.h -- measurement helpers of the pdilqr library (not part of the
 * solver path).
 *
 * The roofline fractions that the benchmark reports divide a kernel's rate
 * by the rate of the pipe that bounds it.  The paper has no counterpart: it
 * reports run times only.  These probes measure those denominators on the
 * GPU at hand instead of deriving them from unit counts and clocks.
 */
#ifndef PDILQR_BENCH_H
#define PDILQR_BENCH_H

#include "pdilqr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PDILQR_PEAK_FFMA = 0,      /* FP32 fused multiply-add pipe                    */
    PDILQR_PEAK_DFMA = 1,      /* FP64 fused multiply-add pipe                    */
    PDILQR_PEAK_TF32_MMA = 2   /* tensor cores, tcgen05.mma kind::tf32, M = 128,  */
                               /* N = 256, K = 8, FP32 accumulators in TMEM       */
} pdilqr_peak_kind;

/* Measure one peak rate on the current device: a kernel that only issues the
 * operation (8 independent FMA chains per thread on 8 CTAs of 256 threads per
 * SM; or one CTA per SM issuing back-to-back MMAs on fixed shared-memory
 * tiles) is sized to about 50 ms, launched `reps` times on the legacy default
 * stream and timed with CUDA events; *tflops receives the best rate (2 flop
 * per FMA, 2 M N K per MMA) and *ms (may be NULL) that launch's time.
 * Synchronous.  Allocates 1 MiB of device memory for the duration of the
 * call.  Errors: INVALID_ARG, NO_MEMORY, CUDA, TIMEOUT (the MMA probe's
 * bounded wait ran out). */
PDILQR_API pdilqr_status pdilqr_peak_probe(int32_t kind, int32_t reps, double *tflops, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* PDILQR_BENCH_H */
