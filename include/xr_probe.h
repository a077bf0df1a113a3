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

/* The fill's own store pattern with nothing generated: rows x row_bytes
 * bytes at d_buf (row-major), each warp writing 32 consecutive rows as
 * 32-row x 128-byte swizzled tiles (staged with st.shared, stored by TMA),
 * column after column.  config 0: 2 warps per CTA x 6 tiles in flight per
 * warp (the fill of light outputs), 1: 1 warp x 8 tiles, 2: 1 warp x 3
 * tiles (the fill of heavy outputs).  d_buf 128-byte aligned, row_bytes a
 * multiple of 128 (at most 2^30), rows a multiple of 32 x warps per CTA,
 * below 2^31; else XR_EINVAL.  The written values are unspecified. */
int xr_probe_tile_store(void *d_buf, size_t rows, size_t row_bytes, int config, void *stream);

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
