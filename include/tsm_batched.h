/*
 * tsm_batched.h -- many uneven TSMTTSM / TSMM instances in one persistent,
 * CUDA-graph-captured launch.
 *
 * The paper tunes one product at a time.  Block-vector solvers issue many
 * small ones of different shapes; launching each separately leaves the GPU
 * idle in launch gaps and reduction tails (the small-K concern of Sec. 3.2).
 * Here every instance is cut into work items (row ranges); one persistent
 * kernel with one resident wave of CTAs claims items largest-first from a
 * device counter and runs each with its instance's configuration:
 *   TSMTTSM items: a T_M x T_N register tile per thread over the item's rows
 *     (Listing 5, transposed mapping of Fig. 10), lanes reduced in shared
 *     memory, the item's M x N partial written to its own slot; the last item
 *     of an instance to finish sums the instance's slots in item order and
 *     applies alpha/beta (deterministic, no floating-point atomics);
 *   TSMM items: alpha * C staged in shared memory (Sec. 4.2), TPR threads per
 *     row of B with interleaved results (Fig. 12), two rows per thread per
 *     iteration (Sec. 4.2 unrolling).
 * tsm_batched_create builds the item list and the workspace and captures
 * {reset counter, persistent kernel} in a CUDA graph; tsm_batched_run
 * replays it.  Replays give bitwise identical results.
 *
 * Descriptor fields (pointers are DEVICE pointers owned by the caller and
 * must stay valid while the batch exists; scalars are copied at creation):
 *   kind       TSM_KIND_TSMTTSM or TSM_KIND_TSMM
 *   op         TSMTTSM: TSM_OP_T or TSM_OP_C;  TSMM: TSM_OP_N
 *   dtype, M, N, K, alpha, beta   as in tsm.h (alpha/beta: re, im)
 *   A, lda     K x M block vector
 *   B, ldb     TSMTTSM: B (K x N);  TSMM: the small matrix C (M x N)
 *   out, ldo   TSMTTSM: C (M x N);  TSMM: B (K x N)
 *   config     per-instance configuration, 0 = built-in default:
 *              bits 0-7  TSMTTSM tile code (1: 1x1, 2: 2x2, 3: 4x4, 4: 4x8,
 *                        5: 8x4, 6: 3x3, 7: 2x5, 8: 5x2, 9: 3x5, 10: 5x3,
 *                        11: 2x7, 12: 7x2, 13: 8x8, 14: 5x5 -- complex data
 *                        runs 4, 5 and 13 as 4x4 and 14 as 3x3; a code whose
 *                        tile needs more than 256 threads, or 0, takes the
 *                        default) or TSMM threads per row code (1: 4,
 *                        2: 8, 3: 16, 4: any count, chosen from N so that
 *                        up to 4 results per thread cover N with the least
 *                        padding);  bits 8-15  log2 of rows per work item
 *                        (10..22; 0 = chosen from the instance's share of
 *                        the whole batch).
 * Instances must not write to memory another instance reads or writes.
 * Errors: INVALID_VALUE / NOT_SUPPORTED as for the single products (checked
 * for every descriptor before anything is allocated), ALLOC if the workspace
 * cannot be allocated, LAUNCH if capture fails.
 */
#ifndef TSM_BATCHED_H
#define TSM_BATCHED_H

#include "tsm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int kind;
    int op;
    int dtype;
    int M, N;
    int64_t K;
    double alpha[2];
    double beta[2];
    const void *A;
    int64_t lda;
    const void *B;
    int64_t ldb;
    void *out;
    int64_t ldo;
    int config;
} tsm_batch_desc;

typedef struct tsm_batch tsm_batch;

tsm_status tsm_batched_create(const tsm_batch_desc *descs, int count, tsm_batch **out);

/* Replays the captured graph on `stream` (asynchronous). */
tsm_status tsm_batched_run(tsm_batch *batch, tsm_stream_t stream);

/* Runs the same work without the graph (one launch of the persistent kernel
 * after a counter reset), for comparison. */
tsm_status tsm_batched_run_direct(tsm_batch *batch, tsm_stream_t stream);

/* Work items and CTAs of the plan. */
tsm_status tsm_batched_info(const tsm_batch *batch, int *items, int *ctas);

void tsm_batched_destroy(tsm_batch *batch);

#ifdef __cplusplus
}
#endif

#endif /* TSM_BATCHED_H */
