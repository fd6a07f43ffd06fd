/*
 * tsm_tune.h -- exhaustive autotuning of libtsm's kernel variants.
 *
 * The paper picks the best kernel configuration for each size by exhaustive
 * search over its generated variants (Sec. 5.1: best tile size and
 * configuration per size; Sec. 7: found by parameter search).  These calls
 * do that search on the caller's device buffers and keep the winners in a
 * tuning table that tsm_tsmttsm / tsm_tsmm consult before their built-in
 * heuristic.
 *
 * Operand roles: for TSM_KIND_TSMTTSM, X = A (K x M), Y = B (K x N),
 * Z = C (M x N); for TSM_KIND_TSMM, X = A (K x M), Y = C (M x N),
 * Z = B (K x N).  All three are DEVICE pointers owned by the caller, laid out
 * as in tsm.h; timing runs compute alpha = 1, beta = 0 into Z (its contents
 * are overwritten).  Timing uses CUDA events on `stream` and synchronizes
 * it.
 */
#ifndef TSM_TUNE_H
#define TSM_TUNE_H

#include "tsm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int variant;   /* index as in tsm_variant_get */
    int grid;      /* CTAs launched */
    float ms;      /* mean milliseconds per call */
} tsm_tune_sample;

/*
 * Times every variant of `kind` that supports (dtype, M, N) at a few grid
 * sizes (multiples of the SM count up to twice the resident-CTA count),
 * `reps` calls each after one warm-up call, records the fastest in the
 * tuning table under (kind, dtype, M, N, floor(log2 K)), and writes up to
 * max_samples measurements to `samples` (may be NULL; *n_samples gets the
 * total count).  NOT_SUPPORTED if no variant fits.  X, Y, Z are the
 * operands in the order of the product's call: TSMTTSM A, B, C; TSMM A, C,
 * B.  With kind TSM_KIND_TSMM_BETA the TSMM variants run with beta = 1, so
 * Z (B) is read as well and must hold finite values.
 */
tsm_status tsm_tune(tsm_kind kind, tsm_dtype dtype, int M, int N, int64_t K,
                    const void *X, int64_t ldx, const void *Y, int64_t ldy,
                    void *Z, int64_t ldz, int reps, tsm_tune_sample *samples,
                    int max_samples, int *n_samples, tsm_stream_t stream);

/* Mean milliseconds of `reps` calls of one variant at one grid size (grid
 * <= 0: the variant's default), with beta = 1 for TSM_KIND_TSMM_BETA.
 * NOT_SUPPORTED if it cannot run the shape. */
tsm_status tsm_time_variant(tsm_kind kind, tsm_dtype dtype, int M, int N,
                            int64_t K, const void *X, int64_t ldx,
                            const void *Y, int64_t ldy, void *Z, int64_t ldz,
                            int variant, int grid, int reps, float *ms,
                            tsm_stream_t stream);

/* Grid sizes tsm_tune tries for a variant and shape: writes up to `max`
 * values to `grids` and their count to *count (0 if the variant cannot run
 * the shape).  Needs the device (occupancy query). */
tsm_status tsm_tune_grids(tsm_kind kind, int variant, tsm_dtype dtype, int M,
                          int N, int *grids, int max, int *count);

/* Puts one entry into the tuning table (e.g. a model's prediction). */
tsm_status tsm_set_tuning(tsm_kind kind, tsm_dtype dtype, int M, int N,
                          int64_t K, int variant, int grid);

/* As tsm_set_tuning, also recording the measured milliseconds of the entry
 * (written to the table file; informational).  Used by the model-pruned
 * search, which times only the candidates the cost model ranks first.
 * INVALID_VALUE for a bad variant, a variant that cannot run the shape, or
 * a negative grid. */
tsm_status tsm_set_tuning_timed(tsm_kind kind, tsm_dtype dtype, int M, int N,
                                int64_t K, int variant, int grid, float ms);

/* Table persistence: text file, one entry per line
 * "kind dtype M N kbucket variant_name grid ms".  Loading merges into the
 * table; the environment variable TSM_TUNE_FILE names a file loaded before
 * the first lookup. */
tsm_status tsm_load_tuning(const char *path);
tsm_status tsm_save_tuning(const char *path);
tsm_status tsm_clear_tuning(void);

#ifdef __cplusplus
}
#endif

#endif /* TSM_TUNE_H */
