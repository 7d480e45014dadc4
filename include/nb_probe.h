/*
 * nb_probe.h -- measurement aid of libnb (not a step of the method): the
 * FP64 / FP32 fused-multiply-add throughput of the current GPU, used as the
 * denominator of "% of FP64 / FP32 peak" for the pairwise evaluation (the
 * paper's Sec. 4 O(N^2) kernel is bound by the arithmetic pipes, not memory).
 */
#ifndef NB_PROBE_H
#define NB_PROBE_H

#include <stdint.h>

#include "nb.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * nb_probe_fma_peak -- run a kernel of independent FMA chains (8 per thread,
 * every SM filled) on the current device and time it with CUDA events.
 *   precision   : NB_FP64 (DFMA) or NB_FP32 (FFMA), or 3: an FP64 stream of
 *                 16 DFMA : 6 DMUL : 5 DADD per chain (the fused : non-fused
 *                 mix of the FP64 pair evaluation), reported as 2 x its
 *                 instruction rate so it compares with the DFMA figure;
 *                 4: the same stream with its multiplies and adds issued as
 *                 FMAs (x*b - 0, x*1 + c); 5: DADD only; 6: DMUL only;
 *                 7: packed two-lane FP32 FMA (fma.rn.f32x2), 4 flops
 *                 per instruction; others -> NB_EINVAL
 *   iters       : FMA iterations per chain (>= 1), e.g. 4096
 *   stream      : cudaStream_t (NULL = legacy default)
 *   flops_per_s : HOST out, 2 flops per FMA
 *   seconds     : HOST out, kernel time
 * Synchronises.  Allocates and frees a small device buffer.  Errors:
 * NB_EINVAL, NB_ECUDA.
 */
nb_status nb_probe_fma_peak(int32_t precision, int64_t iters, void *stream, double *flops_per_s,
                            double *seconds);

/*
 * nb_selftest_wait_timeout -- failure-detection self-test of the bounded
 * device-side waits the evaluation kernel uses on its TMA pipeline: one CTA
 * waits on an mbarrier whose byte count nothing will ever satisfy.  The wait
 * must give up after budget_seconds (0 < budget <= 2), record the timeout in
 * a device error word and let the kernel finish; the call then returns
 * NB_ETIMEOUT (the expected answer).  NB_OK would mean the wait did not give
 * up.  Synchronises `stream`; allocates a 4-byte device word.  Errors:
 * NB_EINVAL (budget), NB_ENOMEM, NB_ECUDA.
 */
nb_status nb_selftest_wait_timeout(double budget_seconds, void *stream);

/*
 * nb_probe_rsqrt -- the evaluation kernel's reciprocal square roots applied
 * elementwise, for accuracy tests against a higher-precision reference:
 *   y[k] = 1 / sqrt(x[k])
 *   which : 0 = the FP64 form the FP64 pair terms use (x scaled into
 *               [1, 4), SFU seed refined in float-float on the FP32 pipe,
 *               assembled as a double on the integer pipe, one FP64 Newton
 *               step: three DFMAs);
 *           1 = the float-float form of the EX pair terms, on x rounded to a
 *               float-float pair, result returned as hi + lo in FP64;
 *           2 = the earlier five-DFMA FP64 form (integer-built FP32 seed,
 *               SFU, one third-order step), for comparison
 *   x, y  : DEVICE double [n]; n >= 0
 *   stream: cudaStream_t (NULL = legacy default); asynchronous
 * Valid inputs: forms 1 and 2: x in [2^-126, 2^127] (the seed's FP32
 * exponent range); form 0: any positive normal double.  Outside these the
 * result is undefined.  Errors: NB_EINVAL (which, n < 0, NULL
 * pointers with n > 0), NB_ECUDA.
 */
nb_status nb_probe_rsqrt(int32_t which, const double *x, double *y, int64_t n, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NB_PROBE_H */
