"""Parity of the FP64 CUDA kernels against the CPU oracle (GPU required).

Every compiled variant that supports a shape is run through the C ABI on the
same seeded inputs as the oracle and compared element by element:
normwise relative Frobenius error <= 1e-12 for random data (the bound the
method must meet), bit-exact for small-integer data (every partial sum is
an exact integer, so any summation order gives the same bits).
"""

import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def tsm():
    import paper_1905_03136_gb300 as t
    from paper_1905_03136_gb300 import build, _lib
    import os
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    t.load()
    return t


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _variants_for(tsm, kind, dt, M, N):
    lib = tsm.load()
    return [i for i in range(lib.tsm_variant_count(kind)) if lib.tsm_variant_supports(kind, i, dt, M, N)]


TSMTTSM_SHAPES = [(1, 1), (2, 2), (2, 3), (3, 3), (4, 4), (7, 5), (8, 8), (16, 16), (33, 17), (32, 32), (64, 64),
                  (1, 64), (64, 1), (8, 32), (32, 8), (13, 64), (49, 25)]
TSMM_SHAPES = [(1, 1), (2, 2), (3, 3), (3, 5), (4, 4), (8, 8), (16, 16), (31, 7), (32, 32), (64, 64), (4, 64),
               (64, 4), (1, 64), (64, 1), (54, 17), (28, 39)]


@pytest.mark.parametrize("cplx", [False, True], ids=["r64", "c64"])
@pytest.mark.parametrize("shape", TSMTTSM_SHAPES, ids=lambda s: "%dx%d" % s)
def test_tsmttsm_every_variant(tsm, shape, cplx):
    M, N = shape
    K = 4097
    A = synth.block_vector(0, K, M, complex_=cplx)
    B = synth.block_vector(1, K, N, complex_=cplx)
    dA, dB = dev(A), dev(B)
    dt = tsm.C64 if cplx else tsm.R64
    ops = ("T", "C") if cplx else ("T",)
    vs = _variants_for(tsm, tsm.KIND_TSMTTSM, dt, M, N)
    assert vs
    for op in ops:
        ref = oracle.gram(A, B, op)
        for v in vs:
            for grid in (0, 7):
                C = tsm.tsmttsm(dA, dB, op=op, variant=v, grid=grid)
                err = oracle.rel_fro(host(C), ref)
                assert err <= TOL, (tsm.variants(tsm.KIND_TSMTTSM)[v]["name"], op, grid, err)


@pytest.mark.parametrize("cplx", [False, True], ids=["r64", "c64"])
@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (16, 16), (64, 64), (64, 1)], ids=lambda s: "%dx%d" % s)
def test_tsmttsm_integer_inputs_bitwise(tsm, shape, cplx):
    M, N = shape
    K = 3001
    A = synth.block_vector(5, K, M, complex_=cplx, dist="smallint")
    B = synth.block_vector(6, K, N, complex_=cplx, dist="smallint")
    dA, dB = dev(A), dev(B)
    dt = tsm.C64 if cplx else tsm.R64
    for op in (("T", "C") if cplx else ("T",)):
        ref = oracle.gram(A, B, op)
        for v in _variants_for(tsm, tsm.KIND_TSMTTSM, dt, M, N):
            C = host(tsm.tsmttsm(dA, dB, op=op, variant=v))
            assert np.array_equal(C, ref), tsm.variants(tsm.KIND_TSMTTSM)[v]["name"]


@pytest.mark.parametrize("cplx", [False, True], ids=["r64", "c64"])
def test_tsmttsm_alpha_beta_ld_and_nan(tsm, cplx):
    import torch
    M, N, K = 6, 5, 20011
    lda, ldb, ldc = M + 3, N + 1, N + 2
    A = synth.block_vector(11, K, M, ld=lda, complex_=cplx)
    B = synth.block_vector(12, K, N, ld=ldb, complex_=cplx, dist="loguniform")
    C0 = synth.block_vector(13, M, N, ld=ldc, complex_=cplx)
    alpha, beta = (0.5 - 1.25j, 2.0 + 0.5j) if cplx else (0.5, -2.0)
    ref = C0.copy()
    oracle.tsmttsm("C" if cplx else "T", M, N, K, alpha, A, lda, B, ldb, beta, ref, ldc)
    dA, dB = dev(A), dev(B)
    dC = dev(C0)
    tsm.tsmttsm(dA[:, :M], dB[:, :N], dC[:, :N], alpha, beta, op="C" if cplx else "T")
    got = host(dC)
    assert oracle.rel_fro(got[:, :N], ref[:, :N]) <= TOL
    assert np.array_equal(got[:, N:], C0[:, N:]), "padding columns of C were written"
    # beta = 0: NaNs in C must not propagate
    nanC = dev(np.full((M, ldc), np.nan, dtype=C0.dtype))
    tsm.tsmttsm(dA[:, :M], dB[:, :N], nanC[:, :N], alpha, 0.0, op="C" if cplx else "T")
    ref0 = np.zeros((M, N), dtype=C0.dtype)
    oracle.tsmttsm("C" if cplx else "T", M, N, K, alpha, A, lda, B, ldb, 0.0, ref0, N)
    assert oracle.rel_fro(host(nanC)[:, :N], ref0) <= TOL
    # K = 0 and alpha = 0: C = beta * C exactly
    dC2 = dev(C0)
    tsm.tsmttsm(dA[:0, :M], dB[:0, :N], dC2[:, :N], alpha, beta, op="T")
    exp = C0.copy()
    exp[:, :N] = beta * C0[:, :N]
    assert np.allclose(host(dC2), exp, rtol=1e-15, atol=0)
    dC3 = dev(C0)
    tsm.tsmttsm(dA[:, :M], dB[:, :N], dC3[:, :N], 0.0, beta, op="T")
    assert np.allclose(host(dC3), exp, rtol=1e-15, atol=0)
    del torch


def test_tsmttsm_small_k_and_determinism(tsm):
    import torch
    for K in (1, 2, 3, 5, 151, 1217):
        A = synth.block_vector(21, K, 8)
        B = synth.block_vector(22, K, 3)
        C = host(tsm.tsmttsm(dev(A), dev(B)))
        assert oracle.rel_fro(C, oracle.gram(A, B)) <= TOL, K
    A = dev(synth.block_vector(23, 300007, 16, complex_=True))
    B = dev(synth.block_vector(24, 300007, 16, complex_=True))
    c1 = host(tsm.tsmttsm(A, B, op="C"))
    for _ in range(3):
        assert np.array_equal(host(tsm.tsmttsm(A, B, op="C")), c1)
    del torch


@pytest.mark.parametrize("cplx", [False, True], ids=["r64", "c64"])
@pytest.mark.parametrize("shape", TSMM_SHAPES, ids=lambda s: "%dx%d" % s)
def test_tsmm_every_variant(tsm, shape, cplx):
    M, N = shape
    K = 5003
    A = synth.block_vector(31, K, M, complex_=cplx)
    Cm = synth.small_matrix(32, M, N, complex_=cplx)
    B0 = synth.block_vector(33, K, N, complex_=cplx)
    dA, dC = dev(A), dev(Cm)
    dt = tsm.C64 if cplx else tsm.R64
    alpha, beta = (1.5 + 0.5j, -0.5 + 1j) if cplx else (1.5, -0.5)
    ref0 = oracle.apply(A, Cm)
    ref1 = oracle.apply(A, Cm, alpha, beta, B0)
    ref2 = oracle.apply(A, Cm, alpha, 1.0, B0)
    vs = _variants_for(tsm, tsm.KIND_TSMM, dt, M, N)
    assert vs
    for v in vs:
        for grid in (0, 5):
            B = tsm.tsmm(dA, dC, variant=v, grid=grid)
            err = oracle.rel_fro(host(B), ref0)
            assert err <= TOL, (tsm.variants(tsm.KIND_TSMM)[v]["name"], grid, err)
        dB = dev(B0)
        tsm.tsmm(dA, dC, dB, alpha, beta, variant=v)
        err = oracle.rel_fro(host(dB), ref1)
        assert err <= TOL, (tsm.variants(tsm.KIND_TSMM)[v]["name"], "alpha/beta", err)
        # beta = 1 exactly: the old B value opens the FMA chain unscaled
        dB = dev(B0)
        tsm.tsmm(dA, dC, dB, alpha, 1.0, variant=v)
        err = oracle.rel_fro(host(dB), ref2)
        assert err <= TOL, (tsm.variants(tsm.KIND_TSMM)[v]["name"], "beta = 1", err)


@pytest.mark.parametrize("cplx", [False, True], ids=["r64", "c64"])
def test_tsmm_integer_bitwise_identity_and_ld(tsm, cplx):
    M, N, K = 12, 9, 4099
    A = synth.block_vector(41, K, M, complex_=cplx, dist="smallint")
    Cm = synth.small_matrix(42, M, N, complex_=cplx, dist="smallint")
    dt = tsm.C64 if cplx else tsm.R64
    ref = oracle.apply(A, Cm)
    dA, dC = dev(A), dev(Cm)
    for v in _variants_for(tsm, tsm.KIND_TSMM, dt, M, N):
        assert np.array_equal(host(tsm.tsmm(dA, dC, variant=v)), ref)
    # C = I reproduces A bit for bit
    I = np.eye(M, dtype=A.dtype)
    assert np.array_equal(host(tsm.tsmm(dev(synth.block_vector(43, K, M, complex_=cplx)), dev(I))),
                          synth.block_vector(43, K, M, complex_=cplx))
    # padded leading dimensions; padding of B untouched; NaN B with beta = 0
    lda, ldc, ldb = M + 5, N + 3, N + 4
    A2 = synth.block_vector(44, K, M, ld=lda, complex_=cplx)
    C2 = synth.block_vector(45, M, N, ld=ldc, complex_=cplx)
    B2 = np.full((K, ldb), np.nan, dtype=A2.dtype)
    dB2 = dev(B2)
    tsm.tsmm(dev(A2)[:, :M], dev(C2)[:, :N], dB2[:, :N], 1.0, 0.0)
    got = host(dB2)
    ref2 = np.zeros((K, N), dtype=A2.dtype)
    oracle.tsmm(M, N, K, 1.0, A2, lda, C2, ldc, 0.0, ref2, N)
    assert oracle.rel_fro(got[:, :N], ref2) <= TOL
    assert np.all(np.isnan(got[:, N:]))


NARROW = [(False, 1, 1), (False, 2, 2), (False, 3, 3), (False, 4, 4), (True, 1, 1), (True, 2, 2)]


def _narrow(tsm, kind, cplx, M, N):
    pre = "%s_%s_narrow_m%dn%d_" % ("tsmttsm" if kind == tsm.KIND_TSMTTSM else "tsmm", "c64" if cplx else "r64", M, N)
    vs = [v["index"] for v in tsm.variants(kind) if v["name"].startswith(pre)]
    assert len(vs) == (7 if kind == tsm.KIND_TSMTTSM else 5), pre
    return vs


@pytest.mark.parametrize("case", NARROW, ids=lambda c: "%s%dx%d" % ("c64_" if c[0] else "r64_", c[1], c[2]))
def test_narrow_variants_every_layout(tsm, case):
    """The vector-streaming narrow kernels on every layout they meet: rows
    stored without padding and vector-aligned (vector path), a base pointer
    one element off the vector boundary and a padded leading dimension (both
    the scalar row path), with row counts that leave a ragged group at the
    end and grids from 1 CTA to more CTAs than groups."""
    cplx, M, N = case
    dt = np.complex128 if cplx else np.float64
    ops = ("T", "C") if cplx else ("T",)
    for K in (4099, 1, 3, 37):
        A = synth.block_vector(61, K + 1, M + 1, complex_=cplx)
        B = synth.block_vector(62, K + 1, N + 1, complex_=cplx)
        Cm = synth.small_matrix(63, M, N, complex_=cplx)
        B0 = synth.block_vector(64, K + 1, N + 1, complex_=cplx)
        dA_pad, dB_pad = dev(A), dev(B)
        flatA = dev(np.concatenate([np.zeros(1, dt), np.ascontiguousarray(A[:K, :M]).ravel()]))
        flatB = dev(np.concatenate([np.zeros(1, dt), np.ascontiguousarray(B[:K, :N]).ravel()]))
        views = {
            "packed": (dev(A[:K, :M]), dev(B[:K, :N])),
            "offset": (flatA[1:].view(K, M), flatB[1:].view(K, N)),
            "padded": (dA_pad[:K, :M], dB_pad[:K, :N]),
        }
        for op in ops:
            ref = oracle.gram(A[:K, :M], B[:K, :N], op)
            for lay, (a, b) in views.items():
                for v in _narrow(tsm, tsm.KIND_TSMTTSM, cplx, M, N):
                    for grid in (0, 1, 5, 400):
                        C = host(tsm.tsmttsm(a, b, op=op, variant=v, grid=grid))
                        err = oracle.rel_fro(C, ref)
                        assert err <= TOL, (tsm.variants(tsm.KIND_TSMTTSM)[v]["name"], K, lay, op, grid, err)
        # TSMM: B = A C and B = alpha A C + beta B on the same layouts
        alpha, beta = (0.75 - 0.5j, 1.0 - 2.0j) if cplx else (0.75, -2.0)
        ref0 = oracle.apply(A[:K, :M], Cm)
        ref1 = oracle.apply(A[:K, :M], Cm, alpha, beta, B0[:K, :N])
        dC = dev(Cm)
        for lay in ("packed", "offset", "padded"):
            a = views[lay][0]
            for v in _narrow(tsm, tsm.KIND_TSMM, cplx, M, N):
                for grid in (0, 1, 5, 400):
                    if lay == "padded":
                        outbuf = dev(np.full((K + 1, N + 1), np.nan, dtype=dt))
                        out = outbuf[:K, :N]
                    elif lay == "offset":
                        outbuf = dev(np.full(K * N + 1, np.nan, dtype=dt))
                        out = outbuf[1:].view(K, N)
                    else:
                        outbuf = dev(np.full((K, N), np.nan, dtype=dt))
                        out = outbuf
                    tsm.tsmm(a, dC, out, variant=v, grid=grid)
                    got = host(out)
                    assert oracle.rel_fro(got, ref0) <= TOL, (tsm.variants(tsm.KIND_TSMM)[v]["name"], K, lay, grid)
                    if lay == "padded":
                        assert np.all(np.isnan(host(outbuf)[:, N:])), "padding of B written"
                    if lay == "offset":
                        assert np.isnan(host(outbuf)[0]), "element before B written"
                # beta != 0 reads B
                if lay == "padded":
                    ob = dev(B0)
                    out = ob[:K, :N]
                elif lay == "offset":
                    ob = dev(np.concatenate([np.zeros(1, dt), np.ascontiguousarray(B0[:K, :N]).ravel()]))
                    out = ob[1:].view(K, N)
                else:
                    ob = dev(np.ascontiguousarray(B0[:K, :N]))
                    out = ob
                tsm.tsmm(a, dC, out, alpha, beta, variant=v)
                err = oracle.rel_fro(host(out), ref1)
                assert err <= TOL, (tsm.variants(tsm.KIND_TSMM)[v]["name"], K, lay, "beta", err)


@pytest.mark.parametrize("cplx", [False, True], ids=["r64", "c64"])
def test_every_width_fixed_shape_kernels(tsm, cplx):
    """Every width-specialised kernel (the code generator's and the narrow
    family's) for every square width 1..64: TSMTTSM and TSMM (beta = 0 and
    beta != 0) against the oracle on a ragged row count."""
    K = 1031
    dt = tsm.C64 if cplx else tsm.R64
    alpha, beta = (0.5 + 0.25j, -1.0 + 0.5j) if cplx else (0.5, -1.0)
    tv = tsm.variants(tsm.KIND_TSMTTSM)
    mv = tsm.variants(tsm.KIND_TSMM)
    seen = 0
    for w in range(1, 65):
        A = synth.block_vector(71, K, w, complex_=cplx)
        B = synth.block_vector(72, K, w, complex_=cplx)
        Cm = synth.small_matrix(73, w, w, complex_=cplx)
        dA, dB, dC = dev(A), dev(B), dev(Cm)
        ref_t = oracle.gram(A, B, "C" if cplx else "T")
        fixed_t = [v for v in _variants_for(tsm, tsm.KIND_TSMTTSM, dt, w, w) if tv[v]["fixed_m"] == w]
        fixed_m = [v for v in _variants_for(tsm, tsm.KIND_TSMM, dt, w, w) if mv[v]["fixed_m"] == w]
        # every width has a TSMM kernel of its own; so has every TSMTTSM width
        # except complex 64, whose 64 x 64 x 2 accumulators are served by the
        # hand-written 8 x 4 tiles (tested above)
        assert fixed_m and (fixed_t or (cplx and w == 64)), ("no width-specialised kernel", w)
        for v in fixed_t:
            C = host(tsm.tsmttsm(dA, dB, op="C" if cplx else "T", variant=v))
            assert oracle.rel_fro(C, ref_t) <= TOL, (tv[v]["name"], w)
            seen += 1
        ref0 = oracle.apply(A, Cm)
        ref1 = oracle.apply(A, Cm, alpha, beta, B)
        ref2 = oracle.apply(A, Cm, 1.0, 1.0, B)
        for v in fixed_m:
            assert oracle.rel_fro(host(tsm.tsmm(dA, dC, variant=v)), ref0) <= TOL, (mv[v]["name"], w)
            out = dev(B)
            tsm.tsmm(dA, dC, out, alpha, beta, variant=v)
            assert oracle.rel_fro(host(out), ref1) <= TOL, (mv[v]["name"], w, "beta")
            out = dev(B)
            tsm.tsmm(dA, dC, out, 1.0, 1.0, variant=v)
            assert oracle.rel_fro(host(out), ref2) <= TOL, (mv[v]["name"], w, "beta = 1")
            seen += 1
    assert seen >= 127


def test_tsmm_beta_tuning_key(tsm, tmp_path):
    """TSMM with beta != 0 has a tuning key of its own: tsm_tune with kind
    TSMM_BETA times the TSMM variants with beta = 1 and records the winner
    under that key, tsm_choose returns it for that key, and calls with
    beta != 0 still match the oracle.  The loaded table is restored."""
    import ctypes
    from paper_1905_03136_gb300 import _lib
    lib = tsm.load()
    saved = str(tmp_path / "table.txt").encode()
    _lib.call("tsm_save_tuning", saved)
    try:
        lib.tsm_clear_tuning()
        K, M, N = 70001, 3, 3
        A = synth.block_vector(81, K, M)
        Cm = synth.small_matrix(82, M, N)
        B0 = synth.block_vector(83, K, N)
        dA, dC = dev(A), dev(Cm)
        Z = dev(B0)
        samples = tsm.tune(tsm.KIND_TSMM_BETA, dA, dC, Z, reps=1)
        assert samples
        best = min(samples, key=lambda s: s[2])
        assert tsm.choose(tsm.KIND_TSMM_BETA, tsm.R64, M, N, K) == (best[0], best[1])
        # the search wrote its own key (2) and no beta = 0 entry (1)
        after = str(tmp_path / "after.txt")
        _lib.call("tsm_save_tuning", after.encode())
        keys = [tuple(int(x) for x in line.split()[:4]) for line in open(after) if not line.startswith("#")]
        assert (2, 0, M, N) in keys and (1, 0, M, N) not in keys
        out = dev(B0)
        tsm.tsmm(dA, dC, out, 1.5, -0.5)
        assert oracle.rel_fro(host(out), oracle.apply(A, Cm, 1.5, -0.5, B0)) <= TOL
    finally:
        lib.tsm_clear_tuning()
        _lib.call("tsm_load_tuning", saved)


def test_device_fill_matches_host_generator(tsm):
    import torch
    for dist in ("uniform", "loguniform", "smallint", "ones"):
        for cplx in (False, True):
            rows, ld, row0 = 1031, 7, 12345
            t = torch.empty((rows, ld), dtype=torch.complex128 if cplx else torch.float64, device="cuda")
            tsm.fill_random(t, seed=9, dist=dist, row0=row0)
            ref = synth.block_vector(9, rows, ld, complex_=cplx, dist=dist, row0=row0)
            assert np.array_equal(host(t), ref), (dist, cplx)


def test_gram_schmidt_step_on_device(tsm):
    """B' = B - Q (Q^H B) with both products on the GPU leaves Q^H B' ~ 0."""
    K, M, N = 200003, 8, 6
    X = synth.block_vector(51, K, M, complex_=True)
    Q = np.ascontiguousarray(np.linalg.qr(X)[0])
    B = synth.block_vector(52, K, N, complex_=True)
    dQ, dB = dev(Q), dev(B)
    C = tsm.tsmttsm(dQ, dB, op="C")
    tsm.tsmm(dQ, C, dB, -1.0, 1.0)
    R = host(tsm.tsmttsm(dQ, dB, op="C"))
    assert np.abs(R).max() < 1e-12 * np.linalg.norm(B)
