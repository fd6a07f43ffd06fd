"""Pins for the CPU oracle: each check compares the oracle with something
other than itself (exact rational arithmetic, exact integer arithmetic,
closed forms from an independent QR, algebraic invariants, published
generator outputs).  ``test_pins_catch_planted_mistakes`` recompiles the C
oracle with a deliberate mistake and shows that the pins fail on it.
"""

import math
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
U = 2.0 ** -53


# ---------------------------------------------------------------- generator

def test_splitmix64_published_outputs():
    rows = []
    with open(os.path.join(HERE, "golden", "splitmix64_seed0.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                i, v = line.split()
                rows.append((int(i), int(v, 16)))
    got = synth.splitmix64(0, [i for i, _ in rows])
    assert [int(x) for x in got] == [v for _, v in rows]


def test_generator_ranges():
    x = synth.values(3, np.arange(1 << 16), "uniform")
    assert x.min() >= -1.0 and x.max() < 1.0
    y = np.abs(synth.values(3, np.arange(1 << 16), "loguniform"))
    assert y.min() >= 2.0 ** -20 and y.max() < 2.0 ** 20
    z = synth.values(3, np.arange(1 << 12), "smallint")
    assert set(np.unique(z)) <= set(range(-8, 8))


# ---------------------------------------------------------------- helpers

def _exact_gram(A, B, op, alpha, beta, C0):
    """alpha * op(A)^T B + beta * C0 in exact rational arithmetic."""
    K, M = A.shape
    N = B.shape[1]
    cplx = np.iscomplexobj(A)
    out = []
    for m in range(M):
        row = []
        for n in range(N):
            if not cplx:
                s = sum(Fraction(float(A[k, m])) * Fraction(float(B[k, n])) for k in range(K))
                v = Fraction(alpha) * s + (Fraction(beta) * Fraction(float(C0[m, n])) if beta else 0)
                row.append(v)
            else:
                sr = Fraction(0)
                si = Fraction(0)
                for k in range(K):
                    ar, ai = Fraction(A[k, m].real), Fraction(A[k, m].imag)
                    if op == "C":
                        ai = -ai
                    br, bi = Fraction(B[k, n].real), Fraction(B[k, n].imag)
                    sr += ar * br - ai * bi
                    si += ar * bi + ai * br
                al = complex(alpha)
                ar_, ai_ = Fraction(al.real), Fraction(al.imag)
                vr = ar_ * sr - ai_ * si
                vi = ar_ * si + ai_ * sr
                if beta:
                    be = complex(beta)
                    cr, ci = Fraction(C0[m, n].real), Fraction(C0[m, n].imag)
                    vr += Fraction(be.real) * cr - Fraction(be.imag) * ci
                    vi += Fraction(be.real) * ci + Fraction(be.imag) * cr
                row.append((vr, vi))
        out.append(row)
    return out


def _abs_sum(A, B):
    return np.abs(A).T @ np.abs(B)


# ---------------------------------------------------------------- pins as functions

def pin_rational_tsmttsm():
    """P1: tiny shapes against exact rational arithmetic."""
    for cplx in (False, True):
        for (K, M, N) in ((1, 1, 1), (7, 3, 2), (17, 5, 4), (33, 2, 5)):
            for op in (("T", "C") if cplx else ("T",)):
                A = synth.block_vector(11, K, M, complex_=cplx)
                B = synth.block_vector(12, K, N, complex_=cplx, dist="loguniform")
                C0 = synth.small_matrix(13, M, N, complex_=cplx)
                alpha, beta = (1.5 - 0.25j, 0.5 + 2j) if cplx else (1.5, -0.75)
                got = oracle.gram(A, B, op, alpha, beta, C0)
                ex = _exact_gram(A, B, op, alpha, beta, C0)
                scale = abs(alpha) * _abs_sum(A, B) + abs(beta) * np.abs(C0)
                for m in range(M):
                    for n in range(N):
                        if cplx:
                            err = abs(complex(got[m, n]) - complex(float(ex[m][n][0]), float(ex[m][n][1])))
                        else:
                            err = abs(got[m, n] - float(ex[m][n]))
                        assert err <= 8 * U * scale[m, n] + 1e-300, (cplx, op, K, M, N, m, n, err)


def pin_rational_tsmm():
    """P1 for TSMM: rows against exact rational dot products."""
    for cplx in (False, True):
        K, M, N = 9, 5, 3
        A = synth.block_vector(21, K, M, complex_=cplx, dist="loguniform")
        Cm = synth.small_matrix(22, M, N, complex_=cplx)
        B0 = synth.block_vector(23, K, N, complex_=cplx)
        alpha, beta = (0.5 + 1j, -1.0 + 0.5j) if cplx else (0.5, 3.0)
        got = oracle.apply(A, Cm, alpha, beta, B0)
        for k in range(K):
            for n in range(N):
                if cplx:
                    s = sum((Fraction(A[k, m].real) + 0) * Fraction(Cm[m, n].real)
                            - Fraction(A[k, m].imag) * Fraction(Cm[m, n].imag) for m in range(M))
                    t = sum(Fraction(A[k, m].real) * Fraction(Cm[m, n].imag)
                            + Fraction(A[k, m].imag) * Fraction(Cm[m, n].real) for m in range(M))
                    ex = complex(alpha) * complex(float(s), float(t)) + complex(beta) * complex(B0[k, n])
                    scale = abs(alpha) * np.abs(A[k]) @ np.abs(Cm[:, n]) + abs(beta) * abs(B0[k, n])
                    assert abs(got[k, n] - ex) <= 16 * U * scale
                else:
                    s = sum(Fraction(float(A[k, m])) * Fraction(float(Cm[m, n])) for m in range(M))
                    ex = Fraction(alpha) * s + Fraction(beta) * Fraction(float(B0[k, n]))
                    scale = abs(alpha) * np.abs(A[k]) @ np.abs(Cm[:, n]) + abs(beta) * abs(B0[k, n])
                    assert abs(got[k, n] - float(ex)) <= 8 * U * scale


def pin_ones():
    """P2: all-ones inputs give C = K and B = M exactly."""
    K, M, N = 1000, 3, 4
    for cplx in (False, True):
        dt = np.complex128 if cplx else np.float64
        A = np.ones((K, M), dt)
        B = np.ones((K, N), dt)
        C = oracle.gram(A, B, "T")
        assert np.array_equal(C, np.full((M, N), K, dt))
        Bo = oracle.apply(A, np.ones((M, N), dt))
        assert np.array_equal(Bo, np.full((K, N), M, dt))


def pin_smallint_exact():
    """P3: small-integer inputs make every partial sum an exact integer, so
    the oracle must equal exact integer arithmetic bit for bit."""
    K = 3001
    for (M, N) in ((1, 1), (3, 7), (8, 5)):
        A = synth.block_vector(31, K, M, dist="smallint")
        B = synth.block_vector(32, K, N, dist="smallint")
        exact = A.astype(np.int64).T @ B.astype(np.int64)
        assert np.array_equal(oracle.gram(A, B), exact.astype(np.float64))
        Cm = synth.small_matrix(33, M, N, dist="smallint")
        exact_b = A.astype(np.int64) @ Cm.astype(np.int64)
        assert np.array_equal(oracle.apply(A, Cm), exact_b.astype(np.float64))
        # complex: (ar + i ai)(br + i bi) with integer parts
        Az = synth.block_vector(34, K, M, complex_=True, dist="smallint")
        Bz = synth.block_vector(35, K, N, complex_=True, dist="smallint")
        ar, ai = Az.real.astype(np.int64), Az.imag.astype(np.int64)
        br, bi = Bz.real.astype(np.int64), Bz.imag.astype(np.int64)
        ex_t = (ar.T @ br - ai.T @ bi) + 1j * (ar.T @ bi + ai.T @ br)
        ex_c = (ar.T @ br + ai.T @ bi) + 1j * (ar.T @ bi - ai.T @ br)
        assert np.array_equal(oracle.gram(Az, Bz, "T"), ex_t)
        assert np.array_equal(oracle.gram(Az, Bz, "C"), ex_c)


def pin_orthonormal():
    """P4: columns of Q from an (independent, LAPACK) QR: Q^T Q = I and
    Q^H Q = I for complex Q."""
    K, M = 4000, 9
    X = synth.block_vector(41, K, M)
    Q, _ = np.linalg.qr(X)
    G = oracle.gram(np.ascontiguousarray(Q), np.ascontiguousarray(Q))
    assert np.abs(G - np.eye(M)).max() < 1e-13
    Z = synth.block_vector(42, K, M, complex_=True)
    Qz, _ = np.linalg.qr(Z)
    Qz = np.ascontiguousarray(Qz)
    Gz = oracle.gram(Qz, Qz, "C")
    assert np.abs(Gz - np.eye(M)).max() < 1e-13
    # The plain transpose of a complex orthonormal basis is NOT the identity.
    assert np.abs(oracle.gram(Qz, Qz, "T") - np.eye(M)).max() > 1e-3


def pin_special_tsmm():
    """P5: C = I reproduces A bit for bit; M = 1 is a scaled outer product."""
    K, M = 777, 6
    for cplx in (False, True):
        A = synth.block_vector(51, K, M, complex_=cplx)
        I = np.eye(M, dtype=np.complex128 if cplx else np.float64)
        assert np.array_equal(oracle.apply(A, I), A)
        a = synth.block_vector(52, K, 1, complex_=cplx)
        c = synth.small_matrix(53, 1, 5, complex_=cplx)
        got = oracle.apply(a, c)
        if cplx:
            # one rounding per part in the oracle vs two in a plain complex
            # multiply: equal to within a couple of units of roundoff
            ref = a[:, :1] * c[:1, :]
            assert np.all(np.abs(got - ref) <= 4 * U * np.abs(a[:, :1]) * np.abs(c[:1, :]))
        else:
            assert np.array_equal(got, a[:, :1] * c[:1, :])


def pin_dot():
    """P6: M = N = 1 is a dot product; compare with math.fsum of the exact
    products split into rounded product + FMA-free residual via Fractions."""
    K = 5000
    a = synth.block_vector(61, K, 1)[:, 0]
    b = synth.block_vector(62, K, 1, dist="loguniform")[:, 0]
    ex = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
    got = oracle.gram(a[:, None].copy(), b[:, None].copy())[0, 0]
    scale = float(np.abs(a) @ np.abs(b))
    assert abs(got - float(ex)) <= 4 * U * scale
    assert abs(oracle.dot("T", a, b) - float(ex)) <= 4 * U * scale
    # the naive sum of rounded products is a much weaker bound
    assert abs(math.fsum(a * b) - float(ex)) <= K * U * scale


def pin_invariants():
    """P7: (A^T B)^T = B^T A; (A^H B)^H = B^H A; A^H B = (A-bar)^T B;
    real data embedded as complex gives the real result."""
    K, M, N = 2049, 5, 3
    A = synth.block_vector(71, K, M)
    B = synth.block_vector(72, K, N)
    assert np.array_equal(oracle.gram(A, B).T, oracle.gram(B, A))
    Az = synth.block_vector(73, K, M, complex_=True)
    Bz = synth.block_vector(74, K, N, complex_=True)
    g1 = oracle.gram(Az, Bz, "C").conj().T
    g2 = oracle.gram(Bz, Az, "C")
    assert np.abs(g1 - g2).max() <= 4 * U * np.abs(g2).max()
    g3 = oracle.gram(np.ascontiguousarray(Az.conj()), Bz, "T")
    assert np.abs(oracle.gram(Az, Bz, "C") - g3).max() <= 4 * U * np.abs(g3).max()
    gz = oracle.gram(A.astype(np.complex128), B.astype(np.complex128), "C")
    assert np.array_equal(gz.real, oracle.gram(A, B)) and not np.any(gz.imag)
    Cm = synth.small_matrix(75, M, N)
    bz = oracle.apply(A.astype(np.complex128), Cm.astype(np.complex128))
    assert np.array_equal(bz.real, oracle.apply(A, Cm)) and not np.any(bz.imag)


def pin_gram_schmidt():
    """P8: one classical Gram-Schmidt step B' = B - Q (Q^H B) built from the
    two oracle products leaves Q^H B' ~ 0 (Sec. 1.2's use case), and TSMM
    rows match an independent per-row dot loop."""
    K, M, N = 6000, 6, 5
    for cplx in (False, True):
        X = synth.block_vector(81, K, M, complex_=cplx)
        Q = np.ascontiguousarray(np.linalg.qr(X)[0])
        B = synth.block_vector(82, K, N, complex_=cplx)
        C = oracle.gram(Q, B, "C")
        B2 = oracle.apply(Q, C, alpha=-1.0, beta=1.0, B0=B)
        R = oracle.gram(Q, B2, "C")
        assert np.abs(R).max() < 1e-13 * np.linalg.norm(B)
        for k in (0, 1, K // 2, K - 1):
            for n in range(N):
                ref = B[k, n] - sum(Q[k, m] * C[m, n] for m in range(M))
                assert abs(B2[k, n] - ref) <= 1e-14 * (abs(B[k, n]) + 1)


def pin_linearity():
    """P9: alpha scaling by a power of two is exact; beta = 0 never reads C
    (NaNs in C do not propagate); beta = 1 adds the old C."""
    K, M, N = 999, 4, 6
    A = synth.block_vector(91, K, M)
    B = synth.block_vector(92, K, N)
    g = oracle.gram(A, B)
    assert np.array_equal(oracle.gram(A, B, alpha=2.0), 2.0 * g)
    nan = np.full((M, N), np.nan)
    assert np.array_equal(oracle.gram(A, B, beta=0.0, C0=nan), g)
    X = synth.small_matrix(93, M, N)
    assert np.abs(oracle.gram(A, B, beta=1.0, C0=X) - (g + X)).max() <= 4 * U * (np.abs(g).max() + 1)
    Cm = synth.small_matrix(94, M, N)
    nanb = np.full((K, N), np.nan)
    assert np.array_equal(oracle.apply(A, Cm, beta=0.0, B0=nanb), oracle.apply(A, Cm))
    # K = 0 leaves beta * C
    empty = np.zeros((0, M))
    assert np.array_equal(oracle.tsmttsm("T", M, N, 0, 1.0, empty, M, np.zeros((0, N)), N, 0.5,
                                         X.copy(), N), 0.5 * X)


def pin_ill_conditioned():
    """Sums whose exact value survives only if both the product residuals and
    the summation carries are kept: with e = 2**-30,
    (1+e)^2 + (1-e)^2 - 1 - 1 = 2 e^2 = 2**-59 exactly, while rounding each
    product to binary64 loses the e^2 terms and a naive sum returns 0; and
    2**60 + 1 - 2**60 = 1 exactly while naive left-to-right summation
    returns 0.  The oracle must reproduce the exact values (rational
    arithmetic gives them) in TSMTTSM, TSMM and the dot product."""
    e = 2.0 ** -30
    a = np.array([[1 + e], [1 - e], [-1.0], [-1.0]])
    b = np.array([[1 + e], [1 - e], [1.0], [1.0]])
    exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a[:, 0], b[:, 0]))
    assert exact == Fraction(2, 2 ** 60)
    assert oracle.gram(a, b)[0, 0] == 2.0 ** -59
    assert oracle.dot("T", a[:, 0], b[:, 0]) == 2.0 ** -59
    assert oracle.gram(a.astype(np.complex128), b.astype(np.complex128), "C")[0, 0] == 2.0 ** -59
    # imaginary route: (i a)^H (i b) = a^T b, (i a)^T (i b) = -a^T b
    ia, ib = 1j * a, 1j * b
    assert oracle.gram(ia, ib, "C")[0, 0] == 2.0 ** -59
    assert oracle.gram(ia, ib, "T")[0, 0] == -(2.0 ** -59)
    # TSMM: the same sum along a row of A times a column of C
    row = np.ascontiguousarray(a.T)
    assert oracle.apply(row, b)[0, 0] == 2.0 ** -59
    big = np.array([[2.0 ** 60], [1.0], [-(2.0 ** 60)]])
    ones = np.ones((3, 1))
    assert oracle.gram(big, ones)[0, 0] == 1.0
    assert oracle.apply(np.ascontiguousarray(big.T), ones)[0, 0] == 1.0


PINS = [pin_rational_tsmttsm, pin_rational_tsmm, pin_ones, pin_smallint_exact, pin_orthonormal,
        pin_special_tsmm, pin_dot, pin_invariants, pin_gram_schmidt, pin_linearity,
        pin_ill_conditioned]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


# ---------------------------------------------------------------- planted mistakes

MUTATIONS = {
    # a dropped conjugation
    "drop_conj": ("if (op == 2) ai = -ai; /* conj(a) */", ""),
    # a wrong sign in the complex product
    "sign_flip": ("acc_add_prod(&x[0], -ai, bi);", "acc_add_prod(&x[0], ai, bi);"),
    # a transposed operand (reads B with A's index)
    "transpose": ("acc_add_prod(x, a[m], b[n]);", "acc_add_prod(x, a[n % M], b[m % N]);"),
    # a dropped correction term of the compensated sum
    "drop_term": ("acc_add(a, e);", ""),
    # an off-by-one row range
    "row_range": ("for (int64_t k = 0; k < K; ++k) {\n        const double *a = A",
                  "for (int64_t k = 1; k < K; ++k) {\n        const double *a = A"),
    # TSMM reading the wrong element of C
    "tsmm_index": ("Cm[(size_t)m * ldc + n]", "Cm[(size_t)n * ldc + m % N]"),
    # beta applied even when zero (NaN propagation)
    "beta_read": ("if (beta != 0.0) r += beta * (*out);", "r += beta * (*out);"),
}


def _compile_mutant(src, tmpdir, name):
    path = os.path.join(tmpdir, f"lib_{name}.so")
    c = os.path.join(tmpdir, f"{name}.c")
    with open(c, "w") as f:
        f.write(src)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", path, c, "-lm"])
    return path


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistakes(name, monkeypatch):
    """Each planted mistake in the C oracle must make at least one pin fail."""
    import ctypes
    with open(oracle._SRC) as f:
        src = f.read()
    old, new = MUTATIONS[name]
    assert old in src, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new, 1)
    with tempfile.TemporaryDirectory() as d:
        path = _compile_mutant(mutated, d, name)
        real = oracle._load()
        lib = ctypes.CDLL(path)
        for fn in ("oracle_tsmttsm", "oracle_tsmm", "oracle_dot"):
            getattr(lib, fn).argtypes = getattr(real, fn).argtypes
            getattr(lib, fn).restype = getattr(real, fn).restype
        monkeypatch.setattr(oracle, "_lib", lib)
        failed = []
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                failed.append(pin.__name__)
        assert failed, f"no pin caught the planted mistake {name}"
