/*
 * xr_probe.h -- measurement probes exported by libxr.
 *
 * These calls compute nothing of the method (the paper has no counterpart):
 * they measure the two ceilings of the fill on the GPU they run on, so that a
 * benchmark can state its roofline against numbers taken in the same process
 * at the same clocks.  The fill writes its outputs and reads almost nothing,
 * and its per-value integer work runs on the integer ALU pipe, so:
 *   - the HBM write ceiling is the rate of a store-only kernel and of
 *     cudaMemsetAsync over the same buffer;
 *   - the integer ceiling is the rate of a kernel that issues nothing but
 *     independent 32-bit logic operations (lop3) on the ALU pipe.
 * Conventions as in xr.h: d_* is caller-owned device memory, `stream` a
 * cudaStream_t passed as void*, calls only enqueue work, status codes as in
 * xr.h (XR_EINVAL for bad arguments, XR_ECUDA for a failed launch).
 */
#ifndef XR_PROBE_H
#define XR_PROBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Write `bytes` bytes at d_buf with 16-byte vector stores from a grid of
 * ctas_per_sm CTAs of 512 threads per SM (0 = 4), each thread storing 16-byte
 * words a grid apart.  d_buf 16-byte aligned, bytes a multiple of 16.  The
 * written values are unspecified. */
int xr_probe_store(void *d_buf, size_t bytes, int ctas_per_sm, void *stream);

/* cudaMemsetAsync(d_buf, 0, bytes, stream): the runtime's own store path. */
int xr_probe_memset(void *d_buf, size_t bytes, void *stream);

/* Integer-ALU probe: `blocks` CTAs of 256 threads each run `iters`
 * iterations of 16 independent lop3.b32 operations (8 chains, two rounds);
 * the total is blocks x 256 x iters x 16 lane operations.  d_sink (one
 * uint32, device) receives a value that depends on every chain, so no work
 * is removed.  blocks >= 1; iters a positive multiple of 8. */
int xr_probe_alu(uint32_t *d_sink, int blocks, int iters, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* XR_PROBE_H */
