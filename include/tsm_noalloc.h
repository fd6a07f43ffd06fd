/*
 * tsm_noalloc.h -- a TSMTTSM entry point that allocates no device memory.
 *
 * The paper has no counterpart: this is an interface addition for callers
 * that must not allocate GPU memory themselves or let a library do it --
 * for example code running inside a memory pool or arena that owns every
 * byte of the device, a real-time or capture-sensitive path where a
 * cudaMalloc would synchronize the device, or a host framework that forbids
 * hidden allocations.  tsm_tsmttsm() keeps a per-stream workspace that it
 * grows with cudaMalloc on first use; this variant instead uses one fixed
 * scratch array compiled into the library.
 *
 * Scratch.  A file-scope device array of TSM_NOALLOC_SCRATCH_BYTES bytes
 * (16 MiB), present on every GPU that loads the library until the process
 * exits.  It holds the per-CTA partial sums of the deterministic reduction
 * and the reduction ticket.  A call runs the kernel and grid that
 * tsm_tsmttsm would run (tuning table, then heuristic) and, like it, a
 * separate final reduction kernel when the partials are many.  When the
 * partials of that grid,  grid * M * N * (1 real | 2 complex) * 8  bytes,
 * do not fit the array, the grid is lowered to the largest multiple of the
 * SM count that fits; results then differ from tsm_tsmttsm's in rounding
 * only.  On a 152-SM GB300 every shape fits at one CTA per SM (at most
 * 152 * 64 * 64 * 2 * 8 = 9.5 MiB); a shape that does not fit even at one
 * CTA per SM (a larger GPU) returns TSM_ERR_NOT_SUPPORTED and launches
 * nothing.
 *
 * Set-up.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call outside any stream capture.
 *
 * Sharing.  Every call on every stream of a device uses the same array, and
 * the array keeps the contents of the last call.  Calls whose work overlaps
 * on the GPU (different streams without ordering) race on it and give wrong
 * results; order them.  The ticket is cleared at the start of every call
 * (cudaMemsetAsync on `stream`, which allocates nothing).
 *
 * Semantics, arguments, layout and errors otherwise as tsm_tsmttsm (tsm.h):
 * C = alpha * op(A)^T B + beta * C in binary64, bitwise reproducible.
 */
#ifndef TSM_NOALLOC_H
#define TSM_NOALLOC_H

#include "tsm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define TSM_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

tsm_status tsm_tsmttsm_noalloc(tsm_op opA, tsm_dtype dtype, int M, int N,
                               int64_t K, const double *alpha, const void *A,
                               int64_t lda, const void *B, int64_t ldb,
                               const double *beta, void *C, int64_t ldc,
                               tsm_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TSM_NOALLOC_H */
