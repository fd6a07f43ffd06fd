/*
 * tsm_split.h -- split-precision TSMTTSM on the tensor cores.
 *
 * The paper computes both products in binary64 on the FP64 units.  On GB300
 * the FP64 rate is about 1.25 TFLOP/s, so TSMTTSM is FP64-bound for every
 * width above one.  This entry point computes the same product,
 *     C = alpha * op(A)^T B + beta * C            (op = T, or C for A^H)
 * with error-free splitting in the style of Ozaki, Ogita, Oishi and Rump
 * ("Error-free transformations of matrix multiplication by using fast
 * routines of matrix multiplication and its applications", Numer. Algorithms
 * 59, 2012): every input column is scaled by a power of two and cut into six
 * signed 8-bit integer slices held exactly in fp16, the slice products
 * run on the tensor cores (tcgen05, FP32 accumulation in tensor memory kept
 * exact by bounding the rows per accumulation tile), and the slice products
 * are recombined and reduced over K in binary64.  Complex data is handled
 * as the real product of the interleaved (re, im) columns.
 *
 * Accuracy: with S slices each input keeps 8S - 1 bits below its column's
 * running maximum and slice products of combined weight below 2^-(8S+6)
 * are dropped, so |C_split - C_exact| is a few units of 2^-(8S-1) relative
 * to sum |a||b| per entry.  S = 6 (tsm_tsmttsm_split): normwise relative
 * error against the FP64 oracle about 1e-14 on uniform and log-uniform
 * inputs, within the 1e-12 bar of the FP64 path; S = 5: about 4e-12;
 * S = 4: about 1e-9 (fewer tensor-core products, fewer accumulator
 * columns, faster).  Inputs that are small integers (or any values with at
 * most 8S - 1 significant bits below the column maximum) give the exact
 * result.  Inputs must be finite (NaN/Inf are not propagated; use
 * tsm_tsmttsm for them).  Results are deterministic for a fixed problem,
 * slice count and device.
 *
 * Arguments, layout, ownership and argument errors as tsm_tsmttsm (tsm.h);
 * any alignment and leading dimension is accepted.  Work is asynchronous on
 * `stream` (two kernels: the split product and a fixed-order reduction of
 * the per-CTA partials); the library's per-(device, stream) workspace holds
 * the partial sums and an error word that tsm_split_status() reads.
 */
#ifndef TSM_SPLIT_H
#define TSM_SPLIT_H

#include "tsm.h"

#ifdef __cplusplus
extern "C" {
#endif

tsm_status tsm_tsmttsm_split(tsm_op opA, tsm_dtype dtype, int M, int N,
                             int64_t K, const double *alpha, const void *A,
                             int64_t lda, const void *B, int64_t ldb,
                             const double *beta, void *C, int64_t ldc,
                             tsm_stream_t stream);

/*
 * How inputs are split for the tensor cores.  TSM_SPLIT_DIGITS_F16: signed
 * 8-bit digits held exactly in fp16, products on tcgen05 kind::f16 with
 * FP32 accumulation (the only kind on sm_103a: the toolchain rejects
 * kind::i8 there, and bf16 or fp8 digits would hold fewer bits per slice
 * for the same product rate).
 */
typedef enum { TSM_SPLIT_DIGITS_F16 = 0 } tsm_split_kind;

/*
 * tsm_tsmttsm_split with the precision knobs: `kind` (TSM_SPLIT_DIGITS_F16)
 * and `slices` S in [4, 6] per input (tsm_tsmttsm_split is S = 6).  Fewer
 * slices trade accuracy (see above) for fewer tensor-core products per row
 * (S (S + 1) / 2 digit pairs).  Errors: as tsm_tsmttsm_split; an unknown
 * kind -> INVALID_VALUE; slices outside [4, 6] -> NOT_SUPPORTED.
 */
tsm_status tsm_tsmttsm_split_ex(tsm_op opA, tsm_dtype dtype, int M, int N,
                                int64_t K, const double *alpha, const void *A,
                                int64_t lda, const void *B, int64_t ldb,
                                const double *beta, void *C, int64_t ldc,
                                tsm_split_kind kind, int slices,
                                tsm_stream_t stream);

/*
 * Launch plan of tsm_tsmttsm_split for a shape (no work is done).  Narrow
 * products (accumulators of 6 slices x the Y chunk width in few tensor-memory
 * columns) run several CTAs per SM so that one CTA's tensor-memory drain
 * overlaps another's conversion; wide ones run one CTA per SM and split B's
 * columns into two chunks when they exceed tensor memory.
 * Errors: info == NULL, bad dtype or K < 1 -> INVALID_VALUE; M, N outside
 * [1, 64] -> NOT_SUPPORTED; no sm_103 device -> NO_DEVICE.
 */
typedef struct {
    int ctas;              /* CTAs of the split kernel */
    int ctas_per_sm;       /* co-resident CTAs per SM (1..4) */
    int column_chunks;     /* B column chunks (1 or 2) */
    int converter_threads; /* threads per CTA that split the inputs */
    int epilogue_warps;    /* warps per CTA that drain tensor memory */
    int threads_per_cta;
    int digit_stages;      /* depth of the converter -> tensor-core ring */
    int tmem_columns;      /* tensor-memory columns allocated per CTA */
    int smem_bytes;        /* dynamic shared memory per CTA */
} tsm_split_plan_info;

tsm_status tsm_split_plan(tsm_dtype dtype, int M, int N, int64_t K,
                          tsm_split_plan_info *info);

/* The plan of tsm_tsmttsm_split_ex with `slices` S (tsm_split_plan is
 * S = 6).  slices outside [4, 6] -> NOT_SUPPORTED, else as tsm_split_plan. */
tsm_status tsm_split_plan_ex(tsm_dtype dtype, int M, int N, int64_t K, int slices,
                             tsm_split_plan_info *info);

/*
 * Synchronizes `stream` and reports whether the most recent
 * tsm_tsmttsm_split on it hit a bounded device-side wait that gave up
 * (TSM_ERR_TIMEOUT; that call's C then holds NaN) -- TSM_OK otherwise.
 * Clears the word.
 */
tsm_status tsm_split_status(tsm_stream_t stream);

/*
 * Test hook: the same kernel with every device-side wait limited to
 * `timeout_cycles` SM clock cycles (<= 0 restores the default of about
 * two seconds).  Affects later calls on all streams.
 */
tsm_status tsm_split_set_timeout(int64_t timeout_cycles);

#ifdef __cplusplus
}
#endif

#endif /* TSM_SPLIT_H */
