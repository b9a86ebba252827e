/* sc_probe.h -- peak-rate probes that the measurement harness divides by.
 *
 * The paper has no counterpart: these are measurement aids.  The assembly's
 * FP64 kernels are bound by the GPU's FP64 fused multiply-add pipe, so their
 * roofline fraction is taken against this probe's measured rate instead of a
 * nominal figure.
 */
#ifndef SC_PROBE_H
#define SC_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Launch a kernel that issues only FP64 fused multiply-adds: every thread
 * runs 8 independent chains of `iters` multiply-adds (x <- x * a + c), on a
 * grid of blocks_per_sm x (number of SMs) blocks of 256 threads, so that
 * flops = 2 * 8 * iters * 256 * blocks_per_sm * SMs (returned in *flops).
 * One double per thread is written to out_dev (device, at least
 * 256 * blocks_per_sm * SMs doubles; query with out_dev = NULL: only *flops
 * and *out_len are set and nothing is launched).  Asynchronous on `stream`;
 * the caller times it (CUDA events on that stream).
 * Returns 0, 1 (invalid argument) or 3 (CUDA error). */
int sc_probe_fp64_fma(int32_t iters, int32_t blocks_per_sm, double *out_dev, double *flops, int64_t *out_len,
                      void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SC_PROBE_H */
