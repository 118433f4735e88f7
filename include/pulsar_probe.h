/*
 * pulsar_probe.h: measurement utility of the renderer library (no
 * counterpart in the paper).
 *
 * The render passes are bound by FP32 arithmetic issue rather than by HBM
 * or tensor cores, so their roofline is stated against the device's FP32
 * FMA throughput.  This entry point measures that throughput on the current
 * device instead of assuming the nominal lanes x clock figure.
 */
#ifndef PULSAR_PROBE_H
#define PULSAR_PROBE_H

#include "pulsar.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Runs a kernel of independent FP32 FMA chains on every SM (enough resident
 * warps to hide the FMA latency), timed with CUDA events on `stream`, and
 * returns the achieved FP32 FLOP/s (2 per FMA) through *flops_per_s and the
 * kernel's duration through *ms (either may be NULL).
 *   sink   device pointer to one float the kernel may write (it never does
 *          for finite inputs; it keeps the chains from being optimised away)
 *   iters  FMA steps per chain, >= 1 (4096 takes well under a millisecond)
 * Synchronises the stream.  PULSAR_ERR_INVALID_ARG for a NULL sink or
 * iters < 1, PULSAR_ERR_CUDA when a runtime call fails. */
pulsar_status pulsar_probe_fma_throughput(float* sink, int iters, double* flops_per_s, float* ms,
                                          void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PULSAR_PROBE_H */
