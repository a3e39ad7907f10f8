/*
 * kitc_peak.h -- arithmetic-issue micro-benchmarks of libkitc.
 *
 * Not part of the treecode (the paper has no counterpart).  They measure the
 * rates that bound the fused evaluator (FP32 FMA, packed FP32x2 FMA, the MUFU
 * reciprocal square root) and the plain FP64 form (FP64 FMA) on the device at
 * hand, so that a roofline fraction divides by a measured peak rather than by
 * unit counts times the nominal clock.
 *
 * Each launch runs `blocks` x `threads` threads; every thread evaluates
 * 8 independent chains a <- a * b + c (or a <- rsqrt(a) * b + c) for
 * iters x 16 rounds and writes one float to sink[global thread index].
 * sink: device, blocks * threads floats, owned by the caller.  The launch is
 * queued on `stream` (a cudaStream_t, NULL = legacy default stream) and does
 * not synchronize; time it with events on the same stream.
 * KITC_ERR_INVALID_ARG for blocks outside 1..2^20, threads not a multiple of
 * 32 in 32..256, iters < 1, a NULL sink or an unknown kind.
 */
#ifndef KITC_PEAK_H
#define KITC_PEAK_H

#include "kitc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KITC_PEAK_FFMA = 0,   /* scalar FP32 FMA (fma.rn.f32), 2 flops each            */
    KITC_PEAK_FFMA2 = 1,  /* packed FP32x2 FMA (fma.rn.f32x2), 4 flops each         */
    KITC_PEAK_DFMA = 2,   /* FP64 FMA (fma.rn.f64), 2 flops each                    */
    KITC_PEAK_RSQRT = 3   /* rsqrt.approx.ftz.f32 (+ one FP32 FMA), 1 result each   */
} kitc_peak_kind;

kitc_status kitc_peak_launch(int kind, int blocks, int threads, int iters, float *sink,
                             void *stream);

/* Work of one kitc_peak_launch with these arguments: flops for the FMA kinds
 * (an FMA counts 2, a packed FMA 4), reciprocal square roots for
 * KITC_PEAK_RSQRT; -1 for an unknown kind. */
double kitc_peak_ops_per_launch(int kind, int blocks, int threads, int iters);

#ifdef __cplusplus
}
#endif
#endif /* KITC_PEAK_H */
