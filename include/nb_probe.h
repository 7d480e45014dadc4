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
 *   precision   : NB_FP64 (DFMA) or NB_FP32 (FFMA); others -> NB_EINVAL
 *   iters       : FMA iterations per chain (>= 1), e.g. 4096
 *   stream      : cudaStream_t (NULL = legacy default)
 *   flops_per_s : HOST out, 2 flops per FMA
 *   seconds     : HOST out, kernel time
 * Synchronises.  Allocates and frees a small device buffer.  Errors:
 * NB_EINVAL, NB_ECUDA.
 */
nb_status nb_probe_fma_peak(int32_t precision, int64_t iters, void *stream, double *flops_per_s,
                            double *seconds);

#ifdef __cplusplus
}
#endif

#endif /* NB_PROBE_H */
