/*
 * tsm.h -- C ABI of libtsm: tall & skinny FP64 matrix products on one GB300
 * (sm_103a), after Ernst, Hager, Thies, Wellein, "Performance Engineering for
 * Real and Complex Tall & Skinny Matrix Multiplication Kernels on GPUs"
 * (arXiv:1905.03136).
 *
 * Operations (Sec. 1.1 of the paper; alpha/beta follow the BLAS convention):
 *   TSMTTSM  C = alpha * op(A)^T * B + beta * C     A: K x M, B: K x N, C: M x N
 *   TSMM     B = alpha * A * C + beta * B           A: K x M, C: M x N, B: K x N
 * with 1 <= M, N <= 64 and K >= 0 (the paper's "skinny" range is 1..64
 * columns and "tall" is more than 10^6 rows; smaller K is accepted).
 *
 * Layout (Sec. 1.2: block vectors are row-major).  Every matrix is row-major
 * with a leading dimension counted in ELEMENTS: element (r, c) of X sits at
 * X[r * ldx + c].  Real data (TSM_R64) is binary64; complex data (TSM_C64) is
 * interleaved (re, im) binary64 pairs, i.e. cuDoubleComplex / complex128, and
 * its leading dimensions count complex elements.
 *
 * Pointers and ownership.  A, B, C are DEVICE pointers owned by the caller;
 * the library never frees or retains them after the call's work completes.
 * alpha and beta are HOST pointers to one double (real) or two doubles
 * (complex: re, im), read during the call.  The library owns one workspace
 * per (device, stream) pair for the cross-CTA reduction; tsm_release() frees
 * them.
 *
 * Asynchrony.  Calls enqueue work on `stream` and return; only argument
 * errors and launch errors are reported synchronously.  Results are
 * bitwise reproducible from run to run for a fixed kernel variant, device and
 * problem (the reductions have a fixed order; no floating-point atomics).
 *
 * Error behaviour.  Every entry point validates all arguments before
 * enqueueing anything; on an error nothing is launched and the outputs are
 * untouched.  TSM_ERR_NOT_SUPPORTED marks a valid request outside what this
 * library implements (e.g. M > 64); TSM_ERR_INVALID_VALUE a malformed one.
 * There is no CPU fallback: without a usable device, calls fail.
 *
 * BLAS rules.  beta == 0 means the output is not read (NaNs in it do not
 * propagate).  alpha == 0 or K == 0 means the output is only scaled by beta.
 * Outputs must not alias inputs (undefined).  Unaligned pointers or leading
 * dimensions are never an error; they only select slower load paths.
 */
#ifndef TSM_H
#define TSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t / CUstream; NULL is the legacy default stream. */
typedef struct CUstream_st *tsm_stream_t;

typedef enum {
    TSM_OK = 0,
    TSM_ERR_INVALID_VALUE = 1, /* malformed argument (null pointer, ld < width, K < 0, ...) */
    TSM_ERR_NOT_SUPPORTED = 2, /* valid but outside the implemented range */
    TSM_ERR_ALLOC = 3,         /* workspace allocation failed */
    TSM_ERR_LAUNCH = 4,        /* a kernel launch or CUDA runtime call failed */
    TSM_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    TSM_ERR_INTERNAL = 6,      /* inconsistent internal state */
    TSM_ERR_NO_DEVICE = 7      /* no usable sm_103 device */
} tsm_status;

typedef enum { TSM_R64 = 0, TSM_C64 = 1 } tsm_dtype;

/* op(A): TSMTTSM accepts T (A^T B) and C (A^H B; identical to T for real
 * data); TSMM accepts N only. */
typedef enum { TSM_OP_N = 0, TSM_OP_T = 1, TSM_OP_C = 2 } tsm_op;

/* ------------------------------------------------------------------ core */

/*
 * TSMTTSM (Sec. 3 of the paper; Listing 1 is the definition): the K-parallel
 * product C = alpha * op(A)^T B + beta * C in binary64 arithmetic on the
 * FP64 pipe.  A: K x M (lda >= M), B: K x N (ldb >= N), C: M x N (ldc >= N).
 * Every CTA reduces a fixed contiguous K range; partials are combined in a
 * fixed order by the last CTA to finish (no floating-point atomics).
 * Errors: M or N outside [1, 64] -> NOT_SUPPORTED; op not T/C, K < 0,
 * ld too small, or a null pointer that would be dereferenced -> INVALID_VALUE.
 */
tsm_status tsm_tsmttsm(tsm_op opA, tsm_dtype dtype, int M, int N, int64_t K,
                       const double *alpha, const void *A, int64_t lda,
                       const void *B, int64_t ldb, const double *beta, void *C,
                       int64_t ldc, tsm_stream_t stream);

/*
 * TSMM (Sec. 4): B = alpha * A C + beta * B in binary64.  A: K x M (lda >= M),
 * C: M x N (ldc >= N), B: K x N (ldb >= N).  alpha * C is staged once per
 * CTA in shared memory or registers (Sec. 4.2); rows of B are independent,
 * so there is no reduction.  With beta != 0 each old B value is read with
 * the row's A values and starts its FMA chain (as it is for beta == 1).
 * opC must be TSM_OP_N.  Errors as for tsm_tsmttsm.
 */
tsm_status tsm_tsmm(tsm_op opC, tsm_dtype dtype, int M, int N, int64_t K,
                    const double *alpha, const void *A, int64_t lda,
                    const void *C, int64_t ldc, const double *beta, void *B,
                    int64_t ldb, tsm_stream_t stream);

/* Human-readable text for a status code (static storage, never NULL). */
const char *tsm_status_string(tsm_status status);

/* Library version as "major.minor.patch" (static storage). */
const char *tsm_version(void);

/* Frees every workspace this library allocated on the current device and
 * forgets cached per-stream state.  Must not overlap with queued work that
 * uses those workspaces (synchronize first). */
tsm_status tsm_release(void);

/* ------------------------------------------------------ kernel variants */

/*
 * Kernel variants.  Each product is implemented by a family of kernels that
 * differ in thread mapping (Sec. 2.2, 3, 4.1), tile shape T_M x T_N
 * (Listing 5), row unrolling (Sec. 4.2), threads per row (Sec. 6.3) and
 * specialisation to fixed M, N by the code generator (Sec. 2.1).  The
 * autotuner and tests address them by index.
 */
typedef enum {
    TSM_KIND_TSMTTSM = 0,
    TSM_KIND_TSMM = 1,
    /* TSMM with beta != 0, which also streams B in: a tuning-table key of
     * its own (the best kernel for three streams differs from the best for
     * two).  It names the same variants as TSM_KIND_TSMM; tsm_tune and
     * tsm_time_variant time them with beta = 1, and a TSMM call with
     * beta != 0 looks this key up first, then the TSM_KIND_TSMM entry. */
    TSM_KIND_TSMM_BETA = 2
} tsm_kind;

typedef struct {
    char name[64];  /* e.g. "tsmttsm_r64_direct_t4x4_u2" */
    int kind;       /* tsm_kind */
    int dtype;      /* tsm_dtype, or -1 if both */
    int fixed_m;    /* 0 = any M, else the only M this variant accepts */
    int fixed_n;    /* 0 = any N */
    int tile_m;     /* TSMTTSM: register tile rows T_M; TSMM: 0 */
    int tile_n;     /* TSMTTSM: tile columns T_N; TSMM: results per thread cap */
    int threads_per_row; /* TSMM: threads sharing one row of B; TSMTTSM: 0 */
    int unroll;     /* rows per thread per loop iteration */
    int block;      /* threads per CTA */
    int generated;  /* 1 if emitted by the code generator */
    int runtime_tile; /* 1: tile_m x tile_n (TSMTTSM) or threads_per_row x
                         tile_n (TSMM) are maxima; each launch picks the size
                         that pads M, N least (tsm_variant_shape) */
} tsm_variant_info;

/* Number of compiled variants of a product, or -1 for an unknown kind. */
int tsm_variant_count(tsm_kind kind);

/* Describes variant `index` of `kind`.  INVALID_VALUE if out of range or
 * info is NULL. */
tsm_status tsm_variant_get(tsm_kind kind, int index, tsm_variant_info *info);

/* As tsm_variant_get, with the tile fields resolved for shape (M, N): for
 * runtime-tile variants the tile (TSMTTSM) or threads per row and results
 * per thread (TSMM) a launch of that shape uses.  INVALID_VALUE for a bad
 * index or NULL info; NOT_SUPPORTED if the variant cannot run the shape. */
tsm_status tsm_variant_shape(tsm_kind kind, int index, tsm_dtype dtype, int M, int N,
                             tsm_variant_info *info);

/* 1 if variant `index` can run (op, dtype, M, N), else 0. */
int tsm_variant_supports(tsm_kind kind, int index, tsm_dtype dtype, int M, int N);

/* Kernel launches one TSMTTSM call of shape (dtype, M, N) makes with `grid`
 * CTAs: 1, or 2 when the CTA partials (grid * M * N doubles, twice that for
 * complex) are many enough that a separate final kernel sums them (Sec. 3.2
 * reduction, second pass).  -1 for a shape outside [1, 64] or grid < 1. */
int tsm_tsmttsm_kernels_per_call(tsm_dtype dtype, int M, int N, int grid);

/*
 * As tsm_tsmttsm / tsm_tsmm but with an explicit variant and grid size
 * (grid <= 0 picks the variant's default: a multiple of the SM count).
 * variant < 0 uses the library's choice (tuning table, then heuristic).
 * NOT_SUPPORTED if the variant cannot run this shape.
 */
tsm_status tsm_tsmttsm_ex(tsm_op opA, tsm_dtype dtype, int M, int N, int64_t K,
                          const double *alpha, const void *A, int64_t lda,
                          const void *B, int64_t ldb, const double *beta,
                          void *C, int64_t ldc, int variant, int grid,
                          tsm_stream_t stream);
tsm_status tsm_tsmm_ex(tsm_op opC, tsm_dtype dtype, int M, int N, int64_t K,
                       const double *alpha, const void *A, int64_t lda,
                       const void *C, int64_t ldc, const double *beta, void *B,
                       int64_t ldb, int variant, int grid, tsm_stream_t stream);

/*
 * One block Gram-Schmidt projection step, the use that motivates TSMTTSM
 * and TSMM in the paper (Sec. 1.1): with A (K x M) holding orthonormal
 * columns,
 *     C = A^H B        (TSMTTSM, op C; A^T B for real data)
 *     B = B - A C      (TSMM, alpha = -1, beta = 1)
 * removes from B (K x N, in place) its components in span(A) and leaves
 * the coefficients in C (M x N, ldc >= N), a caller-owned DEVICE buffer.
 * C does not travel to the host between the two products: the TSMM kernel
 * reads it from device memory once per CTA into shared memory.  Both
 * products use the variants the tuning table selects; the two launches are
 * enqueued on `stream` back to back (no host synchronisation, capturable in
 * a CUDA graph).  For K <= 2^15 the step runs as one fused cooperative
 * kernel instead (tsm_gs_step_ex).  With A not orthonormal the same two products run (one
 * classical Gram-Schmidt projection).
 * Errors: as tsm_tsmttsm / tsm_tsmm; C == NULL -> INVALID_VALUE; every check
 * runs before the first launch, so on an error B and C are untouched.  C must
 * not alias A or B.  K == 0 sets C to zero and leaves B unchanged.
 */
tsm_status tsm_gs_step(tsm_dtype dtype, int M, int N, int64_t K, const void *A,
                       int64_t lda, void *B, int64_t ldb, void *C, int64_t ldc,
                       tsm_stream_t stream);

/* How tsm_gs_step_ex runs the step. */
typedef enum {
    TSM_GS_AUTO = 0,         /* fused for K <= 2^15, else two products */
    TSM_GS_TWO_PRODUCTS = 1, /* the TSMTTSM and TSMM launches described above */
    TSM_GS_FUSED = 2         /* one cooperative kernel (below) */
} tsm_gs_mode;

/*
 * tsm_gs_step with a choice of path; tsm_gs_step is TSM_GS_AUTO.  The fused
 * path is one cooperative launch in which every CTA owns a contiguous range
 * of rows: it forms its partial of C over its rows, all CTAs meet at a grid
 * barrier, CTA b sums a slice of C's entries over the partials in a fixed
 * order and stores them in C, all meet again, and each CTA then updates its
 * own rows of B with -C staged in shared memory.  At small K the second pass
 * finds its rows in L2, and the step is one launch instead of two.  The
 * barrier waits are bounded (tsm_gs_set_timeout); a wait that gives up
 * leaves B and C unspecified and an error word that tsm_gs_status reports.
 * Results of both paths are deterministic (fixed reduction orders) but not
 * bitwise equal to each other.  Arguments, layout, ownership and errors as
 * tsm_gs_step; an unknown mode -> INVALID_VALUE.
 */
tsm_status tsm_gs_step_ex(tsm_dtype dtype, int M, int N, int64_t K, const void *A,
                          int64_t lda, void *B, int64_t ldb, void *C, int64_t ldc,
                          tsm_gs_mode mode, tsm_stream_t stream);

/*
 * Synchronizes `stream` and reports whether a fused Gram-Schmidt step on it
 * hit a barrier wait that gave up (TSM_ERR_TIMEOUT), TSM_OK otherwise.
 * Clears the word.
 */
tsm_status tsm_gs_status(tsm_stream_t stream);

/*
 * Test hook: every barrier wait of later fused steps (all streams) limited
 * to `timeout_cycles` SM clock cycles; <= 0 restores the default of about
 * two seconds.
 */
tsm_status tsm_gs_set_timeout(int64_t timeout_cycles);

/* The variant index and grid the library would use for this shape
 * (tuning table first, then the built-in heuristic). */
tsm_status tsm_choose(tsm_kind kind, tsm_dtype dtype, int M, int N, int64_t K,
                      int *variant, int *grid);

/* ------------------------------------------------------ synthetic inputs */

/*
 * Fills a row-major block vector with the seeded synthetic inputs used by
 * the tests and the benchmark: element (k, c) of a `rows` x `ld` buffer
 * (rows row0 .. row0 + rows - 1 of the full matrix) takes SplitMix64 output
 * number i = (row0 + k) * ld + c of the stream seeded with `seed`
 * (complex: outputs 2i and 2i + 1).  dist: 0 uniform [-1, 1), 1 log-uniform
 * magnitudes 2^-20 .. 2^20, 2 integers in [-8, 7], 3 all ones.  This is
 * input generation only, not part of either product.  dst is a device
 * pointer.  INVALID_VALUE on a bad dist or negative sizes.
 */
tsm_status tsm_fill_random(void *dst, tsm_dtype dtype, int64_t rows, int64_t ld,
                           int64_t row0, uint64_t seed, int dist,
                           tsm_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TSM_H */
