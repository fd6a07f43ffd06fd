/*
 * Uncompensated CPU TSMTTSM and TSMM: the timed CPU baseline.  TEST INFRASTRUCTURE
 * ONLY, like tsm_oracle.c: the benchmark's CPU leg and the tests use it; the
 * library never calls it and shares no code with it.
 *
 * This is the definition of Sec. 1.1 / Listing 1 of the paper (C[m][n] =
 * sum_k A[k][m] * B[k][n]) as the plain k-outer triple loop a CPU user would
 * write: each product is rounded to binary64 and added to a plain running
 * sum (no FMA contraction: built with -ffp-contract=off), with the
 * BLAS-style alpha/beta update on top.  Its error grows like K * u, which is
 * why the parity tests use the compensated oracle instead; this one exists
 * to be timed.
 *
 * Threads: the K range is cut into `nthreads` contiguous chunks of nearly
 * equal length (chunk t = [t*K/T, (t+1)*K/T)); every thread sums its chunk
 * into a private M x N array, and the partial arrays are added in chunk
 * order afterwards, so the result depends on nthreads but not on thread
 * timing.
 *
 * Layout and op as in tsm_oracle.c: row-major, leading dimensions in
 * elements, complex data interleaved (re, im); op 1 = A^T B, 2 = A^H B.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    int op, is_complex, M, N;
    int64_t k0, k1;
    const double *A, *B;
    int64_t lda, ldb;
    double *sum; /* M * N * c plain sums of this chunk */
} chunk_t;

static void *sum_chunk(void *arg) {
    chunk_t *t = (chunk_t *)arg;
    const int M = t->M, N = t->N;
    const int c = t->is_complex ? 2 : 1;
    for (int64_t k = t->k0; k < t->k1; ++k) {
        const double *a = t->A + (size_t)k * t->lda * c;
        const double *b = t->B + (size_t)k * t->ldb * c;
        for (int m = 0; m < M; ++m) {
            for (int n = 0; n < N; ++n) {
                double *s = t->sum + ((size_t)m * N + n) * c;
                if (!t->is_complex) {
                    s[0] += a[m] * b[n];
                } else {
                    double ar = a[2 * m], ai = a[2 * m + 1];
                    double br = b[2 * n], bi = b[2 * n + 1];
                    if (t->op == 2) ai = -ai; /* conj(a) */
                    s[0] += ar * br - ai * bi;
                    s[1] += ar * bi + ai * br;
                }
            }
        }
    }
    return NULL;
}

int oracle_tsmttsm_plain(int op, int is_complex, int M, int N, int64_t K,
                         const double *alpha, const double *A, int64_t lda,
                         const double *B, int64_t ldb, const double *beta,
                         double *C, int64_t ldc, int nthreads) {
    if (M < 1 || N < 1 || K < 0 || nthreads < 1 || nthreads > 1024) return 1;
    const int c = is_complex ? 2 : 1;
    const size_t per = (size_t)M * N * c;
    double *sums = (double *)calloc(per * (size_t)nthreads, sizeof(double));
    chunk_t *ch = (chunk_t *)calloc((size_t)nthreads, sizeof(chunk_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int *started = (int *)calloc((size_t)nthreads, sizeof(int));
    if (!sums || !ch || !th || !started) {
        free(sums);
        free(ch);
        free(th);
        free(started);
        return 2;
    }
    for (int t = 0; t < nthreads; ++t) {
        ch[t].op = op;
        ch[t].is_complex = is_complex;
        ch[t].M = M;
        ch[t].N = N;
        ch[t].k0 = K * t / nthreads;
        ch[t].k1 = K * (t + 1) / nthreads;
        ch[t].A = A;
        ch[t].B = B;
        ch[t].lda = lda;
        ch[t].ldb = ldb;
        ch[t].sum = sums + per * t;
    }
    /* chunk 0 runs on the calling thread; a chunk whose thread cannot be
     * started also runs here, so the result never depends on that */
    for (int t = 1; t < nthreads; ++t)
        started[t] = pthread_create(&th[t], NULL, sum_chunk, &ch[t]) == 0;
    sum_chunk(&ch[0]);
    for (int t = 1; t < nthreads; ++t) {
        if (started[t])
            pthread_join(th[t], NULL);
        else
            sum_chunk(&ch[t]);
    }
    for (int m = 0; m < M; ++m)
        for (int n = 0; n < N; ++n) {
            double v[2] = {0.0, 0.0};
            for (int t = 0; t < nthreads; ++t)
                for (int j = 0; j < c; ++j) v[j] += ch[t].sum[((size_t)m * N + n) * c + j];
            if (!is_complex) {
                double *out = C + (size_t)m * ldc + n;
                double r = alpha[0] * v[0];
                if (beta[0] != 0.0) r += beta[0] * (*out);
                *out = r;
            } else {
                double *out = C + ((size_t)m * ldc + n) * 2;
                double rr = alpha[0] * v[0] - alpha[1] * v[1];
                double ri = alpha[0] * v[1] + alpha[1] * v[0];
                if (beta[0] != 0.0 || beta[1] != 0.0) {
                    double o_r = out[0], o_i = out[1];
                    rr += beta[0] * o_r - beta[1] * o_i;
                    ri += beta[0] * o_i + beta[1] * o_r;
                }
                out[0] = rr;
                out[1] = ri;
            }
        }
    free(sums);
    free(ch);
    free(th);
    free(started);
    return 0;
}

/*
 * Uncompensated CPU TSMM: B = alpha * A C + beta * B as the plain row loop
 * (each output a plain sum over m of rounded products).  Rows are
 * independent, so `nthreads` contiguous row ranges run in parallel and the
 * result does not depend on nthreads.
 */
typedef struct {
    int is_complex, M, N;
    int64_t k0, k1;
    const double *A, *Cm, *alpha, *beta;
    int64_t lda, ldc, ldb;
    double *B;
} rows_t;

static void *tsmm_rows(void *arg) {
    rows_t *t = (rows_t *)arg;
    const int M = t->M, N = t->N;
    const double *al = t->alpha, *be = t->beta;
    for (int64_t k = t->k0; k < t->k1; ++k) {
        if (!t->is_complex) {
            const double *a = t->A + (size_t)k * t->lda;
            double *b = t->B + (size_t)k * t->ldb;
            for (int n = 0; n < N; ++n) {
                double s = 0.0;
                for (int m = 0; m < M; ++m) s += a[m] * t->Cm[(size_t)m * t->ldc + n];
                double r = al[0] * s;
                if (be[0] != 0.0) r += be[0] * b[n];
                b[n] = r;
            }
        } else {
            const double *a = t->A + (size_t)k * t->lda * 2;
            double *b = t->B + (size_t)k * t->ldb * 2;
            for (int n = 0; n < N; ++n) {
                double sr = 0.0, si = 0.0;
                for (int m = 0; m < M; ++m) {
                    const double *c = t->Cm + ((size_t)m * t->ldc + n) * 2;
                    sr += a[2 * m] * c[0] - a[2 * m + 1] * c[1];
                    si += a[2 * m] * c[1] + a[2 * m + 1] * c[0];
                }
                double rr = al[0] * sr - al[1] * si;
                double ri = al[0] * si + al[1] * sr;
                if (be[0] != 0.0 || be[1] != 0.0) {
                    double o_r = b[2 * n], o_i = b[2 * n + 1];
                    rr += be[0] * o_r - be[1] * o_i;
                    ri += be[0] * o_i + be[1] * o_r;
                }
                b[2 * n] = rr;
                b[2 * n + 1] = ri;
            }
        }
    }
    return NULL;
}

int oracle_tsmm_plain(int is_complex, int M, int N, int64_t K, const double *alpha,
                      const double *A, int64_t lda, const double *Cm, int64_t ldc,
                      const double *beta, double *B, int64_t ldb, int nthreads) {
    if (M < 1 || N < 1 || K < 0 || nthreads < 1 || nthreads > 1024) return 1;
    rows_t *ch = (rows_t *)calloc((size_t)nthreads, sizeof(rows_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int *started = (int *)calloc((size_t)nthreads, sizeof(int));
    if (!ch || !th || !started) {
        free(ch);
        free(th);
        free(started);
        return 2;
    }
    for (int t = 0; t < nthreads; ++t) {
        rows_t r = {is_complex, M, N, K * t / nthreads, K * (t + 1) / nthreads,
                    A, Cm, alpha, beta, lda, ldc, ldb, B};
        ch[t] = r;
    }
    for (int t = 1; t < nthreads; ++t)
        started[t] = pthread_create(&th[t], NULL, tsmm_rows, &ch[t]) == 0;
    tsmm_rows(&ch[0]);
    for (int t = 1; t < nthreads; ++t) {
        if (started[t])
            pthread_join(th[t], NULL);
        else
            tsmm_rows(&ch[t]);
    }
    free(ch);
    free(th);
    free(started);
    return 0;
}
