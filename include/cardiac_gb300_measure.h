/*
 * cardiac_gb300_measure.h -- measurement utilities of libcardiac_gb300.so.
 *
 * The stepper is bound by the FP64 pipe on GB300, so its roofline needs the
 * FP64 throughput of the device it runs on; the paper reports its GPU's
 * FP64 peak the same way (Sect. 4: about 128 GFLOP/s on its Kepler card).
 * These calls time small kernels with CUDA events and return measured
 * rates.  They are synchronous and use their own stream.
 */
#ifndef CARDIAC_GB300_MEASURE_H
#define CARDIAC_GB300_MEASURE_H

#include <stdint.h>

#include "cardiac_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Operation timed by cg_measure_fp64_rate. */
enum {
    CG_MEASURE_DFMA = 0,   /* a = fma(a, b, c): 2 flops per op */
    CG_MEASURE_DADD = 1,   /* a = a + c */
    CG_MEASURE_DMUL = 2,   /* a = a * b */
    CG_MEASURE_TANH = 3,   /* a = tanh(a) * b + c (CUDA's double tanh, plus one FMA) */
    CG_MEASURE_EXP = 4,    /* a = exp(-a) * b + c (CUDA's double exp, plus one FMA) */
    CG_MEASURE_DIV = 5,    /* a = b / a + c (IEEE double division, plus one add) */
    CG_MEASURE_DFMA_ONE_LANE = 6   /* DFMA as op 0, on the first lane of each warp only (the other
                                      31 lanes exit at once): ops_per_s counts the active lanes, so a
                                      pipe that takes a warp instruction in the same time whatever
                                      its active lanes reads 1/32 of op 0's rate */
};

/* Launch 4 blocks of 256 threads per SM on the current device, each thread
 * running 8 independent dependency chains of `op` for `iters` iterations,
 * and write the number of operations per second to *ops_per_s and the kernel
 * time to *seconds (either may be NULL).  iters <= 0 picks a count that runs
 * for about 100 ms on GB300 (after an untimed run half as long, so that the
 * clocks have ramped).  Synchronous. */
cg_status cg_measure_fp64_rate(int32_t op, int64_t iters, double *ops_per_s, double *seconds);

/* Evaluate the library's own FP64 elementary functions on the device beside
 * CUDA's, for verification: fn 0 = reciprocal 1/x (x positive, normal, within
 * single-precision exponent range), fn 1 = e^x for x <= 0 (table-driven, after
 * Tang 1989), fn 2 = sigmoid 1/(1 + e^-x).  own[i] gets the library's value,
 * ref[i] CUDA's (1.0/x, exp(x), (1 + tanh(x/2))/2).  x, own, ref: device
 * arrays of n doubles.  Synchronous. */
cg_status cg_check_fastmath(int32_t fn, const double *x, double *own, double *ref, int64_t n);

#ifdef __cplusplus
}
#endif

#endif /* CARDIAC_GB300_MEASURE_H */
