/*
 * CPU oracle for the tall & skinny products.  TEST INFRASTRUCTURE ONLY:
 * tests, the package's smoke check and the benchmark's CPU-baseline leg use
 * it; the library never calls it and shares no code with it.
 *
 * It is the plain definition written out, in binary64 (Sec. 1.1 and
 * Listing 1 of the paper: C[m][n] = sum_k A[k][m] * B[k][n]; TSMM:
 * B = A C), with the BLAS-style alpha/beta update added on top and the
 * complex product taken element by element.  The long sum over k is
 * accumulated with Neumaier's compensated summation (A. Neumaier, ZAMM 54,
 * 1974) applied to every rounded product (each product itself is made
 * exact with an FMA-based TwoProduct, Ogita/Rump/Oishi 2005), so the
 * oracle's own error is about one unit roundoff of the result instead of
 * the sqrt(K) growth of naive summation.
 *
 * Layout: row-major block vectors.  Element (k, m) of A sits at
 * A[k * lda + m]; complex data is interleaved (re, im) pairs and the leading
 * dimensions count complex elements.  alpha and beta point to one double
 * (real) or two doubles (complex).
 *
 * op: 1 = transpose (A^T B), 2 = conjugate transpose (A^H B).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double s; /* running sum */
    double c; /* running compensation */
} acc_t;

/* Neumaier's variant of Kahan summation: add x to (s, c). */
static inline void acc_add(acc_t *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

/* Add the exact product u*v: the rounded product and its FMA residual. */
static inline void acc_add_prod(acc_t *a, double u, double v) {
    double p = u * v;
    double e = fma(u, v, -p);
    acc_add(a, p);
    acc_add(a, e);
}

static inline double acc_value(const acc_t *a) { return a->s + a->c; }

/* out = alpha * value + beta * old, with beta == 0 meaning "old not read". */
static void axpby_real(double alpha, double value, double beta, double *out) {
    double r = alpha * value;
    if (beta != 0.0) r += beta * (*out);
    *out = r;
}

static void axpby_cplx(const double *alpha, double vr, double vi,
                       const double *beta, double *out) {
    double rr = alpha[0] * vr - alpha[1] * vi;
    double ri = alpha[0] * vi + alpha[1] * vr;
    if (beta[0] != 0.0 || beta[1] != 0.0) {
        double o_r = out[0], o_i = out[1];
        rr += beta[0] * o_r - beta[1] * o_i;
        ri += beta[0] * o_i + beta[1] * o_r;
    }
    out[0] = rr;
    out[1] = ri;
}

/*
 * TSMTTSM: C = alpha * op(A)^T B + beta * C, A is K x M, B is K x N,
 * C is M x N (row-major, ldc).  The loop nest is k-outer so that both
 * block vectors stream row by row, with one compensated accumulator per
 * entry of C.
 */
int oracle_tsmttsm(int op, int is_complex, int M, int N, int64_t K,
                   const double *alpha, const double *A, int64_t lda,
                   const double *B, int64_t ldb, const double *beta,
                   double *C, int64_t ldc) {
    if (M < 1 || N < 1 || K < 0) return 1;
    const int c = is_complex ? 2 : 1;
    acc_t *acc = (acc_t *)calloc((size_t)M * N * c, sizeof(acc_t));
    if (!acc) return 2;
    for (int64_t k = 0; k < K; ++k) {
        const double *a = A + (size_t)k * lda * c;
        const double *b = B + (size_t)k * ldb * c;
        for (int m = 0; m < M; ++m) {
            for (int n = 0; n < N; ++n) {
                acc_t *x = acc + ((size_t)m * N + n) * c;
                if (!is_complex) {
                    acc_add_prod(x, a[m], b[n]);
                } else {
                    double ar = a[2 * m], ai = a[2 * m + 1];
                    double br = b[2 * n], bi = b[2 * n + 1];
                    if (op == 2) ai = -ai; /* conj(a) */
                    /* (ar + i ai)(br + i bi) */
                    acc_add_prod(&x[0], ar, br);
                    acc_add_prod(&x[0], -ai, bi);
                    acc_add_prod(&x[1], ar, bi);
                    acc_add_prod(&x[1], ai, br);
                }
            }
        }
    }
    for (int m = 0; m < M; ++m)
        for (int n = 0; n < N; ++n) {
            acc_t *x = acc + ((size_t)m * N + n) * c;
            if (!is_complex) {
                axpby_real(alpha[0], acc_value(x), beta[0], C + (size_t)m * ldc + n);
            } else {
                axpby_cplx(alpha, acc_value(&x[0]), acc_value(&x[1]), beta,
                           C + ((size_t)m * ldc + n) * 2);
            }
        }
    free(acc);
    return 0;
}

/*
 * TSMM: B = alpha * A C + beta * B, A is K x M, C is M x N (ldc), B is
 * K x N.  Each output row is an independent short sum over m.
 */
int oracle_tsmm(int is_complex, int M, int N, int64_t K, const double *alpha,
                const double *A, int64_t lda, const double *Cm, int64_t ldc,
                const double *beta, double *B, int64_t ldb) {
    if (M < 1 || N < 1 || K < 0) return 1;
    for (int64_t k = 0; k < K; ++k) {
        const double *a = A + (size_t)k * lda * (is_complex ? 2 : 1);
        double *b = B + (size_t)k * ldb * (is_complex ? 2 : 1);
        for (int n = 0; n < N; ++n) {
            if (!is_complex) {
                acc_t x = {0.0, 0.0};
                for (int m = 0; m < M; ++m) acc_add_prod(&x, a[m], Cm[(size_t)m * ldc + n]);
                axpby_real(alpha[0], acc_value(&x), beta[0], &b[n]);
            } else {
                acc_t xr = {0.0, 0.0}, xi = {0.0, 0.0};
                for (int m = 0; m < M; ++m) {
                    double ar = a[2 * m], ai = a[2 * m + 1];
                    double cr = Cm[((size_t)m * ldc + n) * 2];
                    double ci = Cm[((size_t)m * ldc + n) * 2 + 1];
                    acc_add_prod(&xr, ar, cr);
                    acc_add_prod(&xr, -ai, ci);
                    acc_add_prod(&xi, ar, ci);
                    acc_add_prod(&xi, ai, cr);
                }
                axpby_cplx(alpha, acc_value(&xr), acc_value(&xi), beta, &b[2 * n]);
            }
        }
    }
    return 0;
}

/*
 * One entry of A^T B (or A^H B) from two columns given as contiguous
 * vectors of length K: used to check sampled entries of products too tall
 * to hold on the host.  Same compensated sum as above.
 */
void oracle_dot(int op, int is_complex, int64_t K, const double *a,
                const double *b, double *out) {
    acc_t xr = {0.0, 0.0}, xi = {0.0, 0.0};
    for (int64_t k = 0; k < K; ++k) {
        if (!is_complex) {
            acc_add_prod(&xr, a[k], b[k]);
        } else {
            double ar = a[2 * k], ai = a[2 * k + 1];
            double br = b[2 * k], bi = b[2 * k + 1];
            if (op == 2) ai = -ai;
            acc_add_prod(&xr, ar, br);
            acc_add_prod(&xr, -ai, bi);
            acc_add_prod(&xi, ar, bi);
            acc_add_prod(&xi, ai, br);
        }
    }
    out[0] = acc_value(&xr);
    if (is_complex) out[1] = acc_value(&xi);
}
