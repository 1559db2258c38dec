/*
 * fockdiag_probe.h -- measurement utility shipped with libfockdiag.so.
 *
 * The paper has no counterpart: this entry point exists to measure the
 * FP64 roof that the walk kernels are compared against.  The walk's work
 * is complex multiply-accumulates, four FP64 fused multiply-adds each, so
 * the relevant ceiling is the FP64 FMA issue rate of the GPU.
 */
#ifndef FOCKDIAG_PROBE_H
#define FOCKDIAG_PROBE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * FP64 FMA throughput of the current device in TFLOP/s (2 flops per FMA):
 * every SM runs independent FMA chains for a fixed iteration count, timed
 * with CUDA events on `stream` (synchronises it).  d_ws: device scratch of
 * at least 256 bytes, 256-byte aligned, owned by the caller.  Writes *tflops.
 * Returns 0 or an fk_status (FK_EWORKSPACE, FK_ECUDA).
 */
int fk_measure_fp64_fma_rate(void *d_ws, size_t ws_bytes, double *tflops, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FOCKDIAG_PROBE_H */
