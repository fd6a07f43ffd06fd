"""Pins for the uncompensated CPU TSMTTSM and TSMM (``oracle/tsm_plain.c``),
the loops the benchmark times as its CPU baseline.  It is checked against exact
rational arithmetic (within the textbook bound of a plain recursive sum,
|error| <= gamma_K * sum |a| |b|, Higham, Accuracy and Stability, Sec. 3.1),
exact integer arithmetic (bit for bit, for any thread count), the
conjugation and transpose definitions, and the BLAS beta rule.  Planted
mistakes in its source must make one of these pins fail.
"""

import ctypes
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

U = 2.0 ** -53


def _exact(A, B, op):
    K, M = A.shape
    N = B.shape[1]
    out = np.zeros((M, N), dtype=complex)
    for m in range(M):
        for n in range(N):
            if not np.iscomplexobj(A):
                out[m, n] = float(sum(Fraction(float(A[k, m])) * Fraction(float(B[k, n])) for k in range(K)))
            else:
                sr = si = Fraction(0)
                for k in range(K):
                    ar, ai = Fraction(A[k, m].real), Fraction(A[k, m].imag)
                    if op == "C":
                        ai = -ai
                    br, bi = Fraction(B[k, n].real), Fraction(B[k, n].imag)
                    sr += ar * br - ai * bi
                    si += ar * bi + ai * br
                out[m, n] = complex(float(sr), float(si))
    return out


def pin_plain_rational():
    """Tiny shapes against exact rational sums, within gamma_(K+2)."""
    for cplx in (False, True):
        for (K, M, N, T) in ((1, 1, 1, 1), (9, 3, 2, 2), (23, 4, 5, 3), (40, 2, 3, 7)):
            for op in (("T", "C") if cplx else ("T",)):
                A = synth.block_vector(111, K, M, complex_=cplx)
                B = synth.block_vector(112, K, N, complex_=cplx, dist="loguniform")
                got = oracle.gram_plain(A, B, op, threads=T)
                ex = _exact(A, B, op)
                scale = np.abs(A).T @ np.abs(B)
                bound = (K + 2) * U / (1 - (K + 2) * U) * scale * (2 if cplx else 1)
                assert np.all(np.abs(got - (ex if cplx else ex.real)) <= bound + 1e-300), (cplx, op, K, M, N, T)


def pin_plain_smallint():
    """Small integers: every partial sum is exact, so any thread count gives
    the exact integer product bit for bit."""
    K = 2501
    for (M, N) in ((1, 1), (3, 7), (8, 5)):
        A = synth.block_vector(121, K, M, dist="smallint")
        B = synth.block_vector(122, K, N, dist="smallint")
        exact = (A.astype(np.int64).T @ B.astype(np.int64)).astype(np.float64)
        for T in (1, 4, 13):
            assert np.array_equal(oracle.gram_plain(A, B, threads=T), exact), (M, N, T)
        Az = synth.block_vector(123, K, M, complex_=True, dist="smallint")
        Bz = synth.block_vector(124, K, N, complex_=True, dist="smallint")
        ar, ai = Az.real.astype(np.int64), Az.imag.astype(np.int64)
        br, bi = Bz.real.astype(np.int64), Bz.imag.astype(np.int64)
        ex_t = (ar.T @ br - ai.T @ bi) + 1j * (ar.T @ bi + ai.T @ br)
        ex_c = (ar.T @ br + ai.T @ bi) + 1j * (ar.T @ bi - ai.T @ br)
        for T in (1, 6):
            assert np.array_equal(oracle.gram_plain(Az, Bz, "T", threads=T), ex_t)
            assert np.array_equal(oracle.gram_plain(Az, Bz, "C", threads=T), ex_c)


def pin_plain_more_threads_than_rows():
    """Empty chunks (threads > K) and K = 0 leave the sum unchanged."""
    A = synth.block_vector(131, 3, 2, dist="smallint")
    B = synth.block_vector(132, 3, 4, dist="smallint")
    exact = (A.astype(np.int64).T @ B.astype(np.int64)).astype(np.float64)
    assert np.array_equal(oracle.gram_plain(A, B, threads=8), exact)
    C = np.full((2, 4), 3.0)
    oracle.tsmttsm_plain("T", 2, 4, 0, 1.0, np.zeros(0), 2, np.zeros(0), 4, 0.5, C, 4, 3)
    assert np.array_equal(C, np.full((2, 4), 1.5))


def pin_plain_alpha_beta():
    """alpha, beta as in BLAS; beta = 0 does not read C (NaN stays out)."""
    K, M, N = 301, 3, 4
    for cplx in (False, True):
        A = synth.block_vector(141, K, M, complex_=cplx, dist="smallint")
        B = synth.block_vector(142, K, N, complex_=cplx, dist="smallint")
        g = oracle.gram_plain(A, B, "C" if cplx else "T", threads=3)
        alpha, beta = (2.0 - 1.0j, 0.5 + 0.25j) if cplx else (2.0, -0.5)
        C0 = synth.small_matrix(143, M, N, complex_=cplx, dist="smallint")
        C = C0.copy()
        oracle.tsmttsm_plain("C" if cplx else "T", M, N, K, alpha, A, M, B, N, beta, C, N, 3)
        assert np.array_equal(C, alpha * g + beta * C0)
        nan = np.full((M, N), np.nan, dtype=C0.dtype)
        oracle.tsmttsm_plain("C" if cplx else "T", M, N, K, 1.0, A, M, B, N, 0.0, nan, N, 2)
        assert np.array_equal(nan, g)


def pin_plain_tsmm():
    """TSMM rows: exact rational row sums within gamma_(M+2); small
    integers bit for bit for any thread count; beta = 0 does not read B."""
    for cplx in (False, True):
        K, M, N = 11, 6, 3
        A = synth.block_vector(161, K, M, complex_=cplx, dist="loguniform")
        Cm = synth.small_matrix(162, M, N, complex_=cplx)
        B0 = synth.block_vector(163, K, N, complex_=cplx)
        alpha, beta = (0.5 + 1j, -1.0 + 0.5j) if cplx else (0.5, 3.0)
        got = oracle.apply_plain(A, Cm, alpha, beta, B0, threads=4)
        for k in range(K):
            for n in range(N):
                if cplx:
                    s = sum(Fraction(A[k, m].real) * Fraction(Cm[m, n].real)
                            - Fraction(A[k, m].imag) * Fraction(Cm[m, n].imag) for m in range(M))
                    t = sum(Fraction(A[k, m].real) * Fraction(Cm[m, n].imag)
                            + Fraction(A[k, m].imag) * Fraction(Cm[m, n].real) for m in range(M))
                    ex = complex(alpha) * complex(float(s), float(t)) + complex(beta) * complex(B0[k, n])
                else:
                    s = sum(Fraction(float(A[k, m])) * Fraction(float(Cm[m, n])) for m in range(M))
                    ex = float(Fraction(alpha) * s + Fraction(beta) * Fraction(float(B0[k, n])))
                scale = abs(alpha) * (np.abs(A[k]) @ np.abs(Cm[:, n])) + abs(beta) * abs(B0[k, n])
                assert abs(got[k, n] - ex) <= 4 * (M + 4) * U * scale, (cplx, k, n)
        Ai = synth.block_vector(164, 999, M, complex_=cplx, dist="smallint")
        Ci = synth.small_matrix(165, M, N, complex_=cplx, dist="smallint")
        if cplx:
            ar, ai = Ai.real.astype(np.int64), Ai.imag.astype(np.int64)
            cr, ci = Ci.real.astype(np.int64), Ci.imag.astype(np.int64)
            exact = (ar @ cr - ai @ ci) + 1j * (ar @ ci + ai @ cr)
        else:
            exact = (Ai.astype(np.int64) @ Ci.astype(np.int64)).astype(np.float64)
        for T in (1, 7):
            assert np.array_equal(oracle.apply_plain(Ai, Ci, threads=T), exact)
        nan = np.full((999, N), np.nan, dtype=Ai.dtype)
        assert np.array_equal(oracle.apply_plain(Ai, Ci, beta=0.0, B0=nan, threads=3), exact)


PLAIN_PINS = [pin_plain_rational, pin_plain_smallint, pin_plain_more_threads_than_rows, pin_plain_alpha_beta,
              pin_plain_tsmm]


@pytest.mark.parametrize("pin", PLAIN_PINS, ids=[p.__name__ for p in PLAIN_PINS])
def test_plain_pin(pin):
    pin()


def test_plain_agrees_with_compensated_oracle():
    """On uniform data both loops agree to within the plain loop's bound."""
    K, M, N = 20000, 5, 6
    for cplx in (False, True):
        A = synth.block_vector(151, K, M, complex_=cplx)
        B = synth.block_vector(152, K, N, complex_=cplx)
        op = "C" if cplx else "T"
        ref = oracle.gram(A, B, op)
        got = oracle.gram_plain(A, B, op, threads=4)
        assert oracle.rel_fro(got, ref) <= K * U


MUTATIONS = {
    "drop_conj": ("if (t->op == 2) ai = -ai; /* conj(a) */", ""),
    "sign_flip": ("s[0] += ar * br - ai * bi;", "s[0] += ar * br + ai * bi;"),
    "transpose": ("s[0] += a[m] * b[n];", "s[0] += a[n % M] * b[m % N];"),
    "chunk_bound": ("ch[t].k1 = K * (t + 1) / nthreads;", "ch[t].k1 = K * (t + 1) / nthreads - (t > 0);"),
    "skip_partial": ("for (int t = 0; t < nthreads; ++t)\n                for (int j",
                     "for (int t = 1; t < nthreads; ++t)\n                for (int j"),
    "beta_read": ("if (beta[0] != 0.0) r += beta[0] * (*out);", "r += beta[0] * (*out);"),
    "tsmm_index": ("s += a[m] * t->Cm[(size_t)m * t->ldc + n];", "s += a[m] * t->Cm[(size_t)n * t->ldc + m % N];"),
    "tsmm_sign": ("sr += a[2 * m] * c[0] - a[2 * m + 1] * c[1];", "sr += a[2 * m] * c[0] + a[2 * m + 1] * c[1];"),
    "tsmm_rows": ("K * t / nthreads, K * (t + 1) / nthreads,", "K * t / nthreads, K * (t + 1) / nthreads - 1,"),
    "tsmm_beta_read": ("if (be[0] != 0.0) r += be[0] * b[n];", "r += be[0] * b[n];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_plain_pins_catch_planted_mistakes(name, monkeypatch):
    with open(oracle._SRC_PLAIN) as f:
        src = f.read()
    old, new = MUTATIONS[name]
    assert old in src, "mutation anchor for %s not found" % name
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "plain.c")
        so = os.path.join(d, "libplain.so")
        with open(c, "w") as f:
            f.write(src.replace(old, new, 1))
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o", so, c])
        real = oracle._load()
        lib = ctypes.CDLL(so)
        lib.oracle_tsmttsm_plain.argtypes = real.oracle_tsmttsm_plain.argtypes
        lib.oracle_tsmttsm_plain.restype = ctypes.c_int
        lib.oracle_tsmm_plain.argtypes = real.oracle_tsmm_plain.argtypes
        lib.oracle_tsmm_plain.restype = ctypes.c_int

        class Mixed:
            def __getattr__(self, n):
                return getattr(lib if n.endswith("_plain") else real, n)

        monkeypatch.setattr(oracle, "_lib", Mixed())
        failed = []
        for pin in PLAIN_PINS:
            try:
                pin()
            except AssertionError:
                failed.append(pin.__name__)
        assert failed, "no pin caught the planted mistake %s" % name
