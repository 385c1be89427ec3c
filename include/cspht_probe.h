/*
 * cspht_probe.h -- measured arithmetic peaks of the current GPU.
 *
 * Not part of the method (the paper has no counterpart): the CSPH-TVD step's
 * kernels are bound by arithmetic and instruction issue rather than memory
 * bandwidth, so their roofline is taken against the rate at which this GPU
 * retires fused multiply-adds, measured here by the library's own kernels.
 */
#ifndef CSPHT_PROBE_H
#define CSPHT_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CSPHT_PROBE_FP32 = 0,   /* scalar FP32 fma (FFMA) */
    CSPHT_PROBE_FP32X2 = 1, /* packed two-lane FP32 fma (fma.rn.f32x2) */
    CSPHT_PROBE_FP64 = 2    /* FP64 fma (DFMA) */
};

/* Runs one multiply-add throughput kernel of the given kind on the current
 * device and stream-orders nothing else: 8 blocks of 256 threads per SM, 8
 * independent chains per thread, `trips` loop trips of 8 multiply-adds per
 * chain (a multiply-add = 2 flops, a packed one 4), after a warm-up launch of
 * trips/16.  Writes the achieved TFLOP/s (CUDA-event time of the timed
 * launch) to *tflops and that time in milliseconds to *ms (may be NULL).
 * Allocates and frees a small device buffer and a stream.  Returns 0, or -1
 * for invalid arguments, -2 when an allocation fails, -3 on a CUDA error.
 * Pick trips so that the launch takes tens of milliseconds: about 2e5 for
 * FP32, 1e5 for packed FP32, 4e3 for FP64 on a 148-SM part. */
int cspht_probe_fma(int kind, int trips, double *tflops, double *ms);

#ifdef __cplusplus
}
#endif
#endif
