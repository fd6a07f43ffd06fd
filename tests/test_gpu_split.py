"""Split-precision TSMTTSM (tensor cores) against the FP64 oracle.

Pins: small-integer inputs are represented exactly by the slices, so the
split product must equal the oracle bit for bit; random uniform and
log-uniform inputs must meet the normwise 1e-12 bar; a forced expiry of the
device-side waits must surface as TSM_ERR_TIMEOUT with NaN output and leave
the context usable.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def sp():
    import os
    import paper_1905_03136_gb300 as t
    from paper_1905_03136_gb300 import build, _lib, split
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    t.load()
    return split


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


SHAPES = [(False, 1, 1), (False, 7, 5), (False, 32, 32), (False, 64, 64), (False, 64, 1), (False, 33, 17),
          (True, 1, 1), (True, 8, 8), (True, 32, 32), (True, 48, 48), (True, 64, 64), (True, 1, 64),
          (True, 64, 7), (True, 33, 41)]


@pytest.mark.parametrize("case", SHAPES, ids=lambda c: "%s_%dx%d" % ("c64" if c[0] else "r64", c[1], c[2]))
def test_split_integer_inputs_bitwise(sp, case):
    cplx, M, N = case
    K = 4097
    A = synth.block_vector(3, K, M, complex_=cplx, dist="smallint")
    B = synth.block_vector(4, K, N, complex_=cplx, dist="smallint")
    for op in (("T", "C") if cplx else ("T",)):
        got = host(sp.tsmttsm_split(dev(A), dev(B), op=op))
        assert np.array_equal(got, oracle.gram(A, B, op)), op
    assert sp.status() == 0


@pytest.mark.parametrize("dist", ["uniform", "loguniform"])
@pytest.mark.parametrize("case", SHAPES, ids=lambda c: "%s_%dx%d" % ("c64" if c[0] else "r64", c[1], c[2]))
def test_split_random_inputs(sp, case, dist):
    cplx, M, N = case
    K = 20011
    A = synth.block_vector(0, K, M, complex_=cplx, dist=dist)
    B = synth.block_vector(1, K, N, complex_=cplx, dist=dist)
    for op in (("T", "C") if cplx else ("T",)):
        got = host(sp.tsmttsm_split(dev(A), dev(B), op=op))
        err = oracle.rel_fro(got, oracle.gram(A, B, op))
        assert err <= TOL, (op, err)


SLICE_SHAPES = [(False, 7, 5), (False, 64, 64), (False, 33, 17), (True, 8, 8), (True, 32, 32), (True, 48, 48),
                (True, 64, 64), (True, 33, 41)]


@pytest.mark.parametrize("slices", [4, 5, 6])
@pytest.mark.parametrize("case", SLICE_SHAPES, ids=lambda c: "%s_%dx%d" % ("c64" if c[0] else "r64", c[1], c[2]))
def test_split_slice_count(sp, case, slices):
    """Each slice count S keeps 8S - 1 bits per input: small integers stay
    exact (bit for bit), uniform inputs meet a normwise bound of
    32 * 2^-(8S-1) against the oracle (S = 6: the 1e-12 bar with room), and
    the default call is S = 6 bit for bit."""
    cplx, M, N = case
    K = 4099
    op = "C" if cplx else "T"
    Ai = synth.block_vector(5, K, M, complex_=cplx, dist="smallint")
    Bi = synth.block_vector(6, K, N, complex_=cplx, dist="smallint")
    got = host(sp.tsmttsm_split(dev(Ai), dev(Bi), op=op, slices=slices))
    assert np.array_equal(got, oracle.gram(Ai, Bi, op))
    A = synth.block_vector(7, K, M, complex_=cplx)
    B = synth.block_vector(8, K, N, complex_=cplx)
    dA, dB = dev(A), dev(B)
    got = host(sp.tsmttsm_split(dA, dB, op=op, slices=slices))
    err = oracle.rel_fro(got, oracle.gram(A, B, op))
    assert err <= 32 * 2.0 ** -(8 * slices - 1), (slices, err)
    if slices == 6:
        assert err <= TOL
        assert np.array_equal(got, host(sp.tsmttsm_split(dA, dB, op=op)))
    else:
        # fewer slices: never more accurate than the full split
        assert err >= oracle.rel_fro(host(sp.tsmttsm_split(dA, dB, op=op)), oracle.gram(A, B, op))
    pl = sp.plan(int(cplx), M, N, K, slices)
    assert pl["tmem_columns"] <= 512
    assert sp.status() == 0


def test_split_alpha_beta_ld_nan_and_k0(sp):
    M, N, K = 24, 40, 30011
    lda, ldb, ldc = M + 3, N + 5, N + 2
    A = synth.block_vector(11, K, M, ld=lda, complex_=True)
    B = synth.block_vector(12, K, N, ld=ldb, complex_=True)
    C0 = synth.block_vector(13, M, N, ld=ldc, complex_=True)
    alpha, beta = 0.5 - 1.25j, 2.0 + 0.5j
    ref = C0.copy()
    oracle.tsmttsm("C", M, N, K, alpha, A, lda, B, ldb, beta, ref, ldc)
    dC = dev(C0)
    sp.tsmttsm_split(dev(A)[:, :M], dev(B)[:, :N], dC[:, :N], alpha, beta, op="C")
    got = host(dC)
    assert oracle.rel_fro(got[:, :N], ref[:, :N]) <= TOL
    assert np.array_equal(got[:, N:], C0[:, N:])
    nanC = dev(np.full((M, N), np.nan + 0j))
    sp.tsmttsm_split(dev(A)[:, :M], dev(B)[:, :N], nanC, 1.0, 0.0, op="C")
    assert oracle.rel_fro(host(nanC), oracle.gram(A[:, :M].copy(), B[:, :N].copy(), "C")) <= TOL
    dC2 = dev(C0)
    sp.tsmttsm_split(dev(A)[:0, :M], dev(B)[:0, :N], dC2[:, :N], alpha, beta)
    assert np.allclose(host(dC2)[:, :N], beta * C0[:, :N], rtol=1e-15, atol=0)


def test_split_small_k_ragged_and_deterministic(sp):
    for K in (1, 15, 16, 17, 255, 257, 4095):
        A = synth.block_vector(21, K, 64, dist="loguniform")
        B = synth.block_vector(22, K, 64)
        got = host(sp.tsmttsm_split(dev(A), dev(B)))
        assert oracle.rel_fro(got, oracle.gram(A, B)) <= TOL, K
    A = dev(synth.block_vector(23, 300007, 64, complex_=True))
    B = dev(synth.block_vector(24, 300007, 64, complex_=True))
    c1 = host(sp.tsmttsm_split(A, B, op="C"))
    for _ in range(2):
        assert np.array_equal(host(sp.tsmttsm_split(A, B, op="C")), c1)


def test_split_magnitude_jumps_along_k(sp):
    """Column magnitudes that grow and shrink along K force accumulation
    tiles to end early (running exponents increase); the result must still
    meet the bar."""
    K, M, N = 12000, 16, 16
    A = synth.block_vector(31, K, M)
    B = synth.block_vector(32, K, N)
    scale = np.ldexp(1.0, (np.arange(K) // 700) % 9 * 3 - 12)[:, None]
    A = np.ascontiguousarray(A * scale)
    B = np.ascontiguousarray(B * scale[::-1])
    got = host(sp.tsmttsm_split(dev(A), dev(B)))
    assert oracle.rel_fro(got, oracle.gram(A, B)) <= TOL


def test_split_wait_expiry_reports_timeout(sp):
    """Every device-side wait limited to a few cycles: the kernel must give
    up, report TSM_ERR_TIMEOUT, write NaN, and the next call must work."""
    import torch
    K = 50000
    A = synth.block_vector(41, K, 32, complex_=True)
    B = synth.block_vector(42, K, 32, complex_=True)
    dA, dB = dev(A), dev(B)
    try:
        sp.set_timeout(4)
        C = sp.tsmttsm_split(dA, dB, op="C")
        assert sp.status() == 5
        assert np.all(np.isnan(host(C)))
    finally:
        sp.set_timeout(0)
    C = sp.tsmttsm_split(dA, dB, op="C")
    assert sp.status() == 0
    assert oracle.rel_fro(host(C), oracle.gram(A, B, "C")) <= TOL
    torch.cuda.synchronize()


K_FULL = 1 << 24


def test_split_plan(sp):
    """Narrow products share SMs (several CTAs, smaller tensor-memory
    allocations); wide ones take one CTA per SM and two column chunks."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for (dt, M, N) in [(0, 1, 1), (0, 16, 16), (1, 8, 8), (0, 32, 32), (1, 16, 16), (0, 64, 64), (1, 32, 32),
                       (1, 48, 48), (1, 64, 64), (1, 33, 41)]:
        p = sp.plan(dt, M, N, K_FULL)
        assert 1 <= p["ctas_per_sm"] <= 4
        assert p["ctas"] == p["ctas_per_sm"] * sms // p["column_chunks"] * p["column_chunks"]
        assert p["tmem_columns"] * p["ctas_per_sm"] <= 512
        assert p["ctas_per_sm"] * (p["smem_bytes"] + 1024) <= 228 * 1024
        assert p["digit_stages"] >= 2 and p["epilogue_warps"] in (4, 8)
        assert p["threads_per_cta"] == p["converter_threads"] + 32 * (1 + p["epilogue_warps"])
    assert sp.plan(0, 16, 16, K_FULL)["ctas_per_sm"] >= 2
    wide = sp.plan(1, 64, 64, K_FULL)
    assert wide["ctas_per_sm"] == 1 and wide["column_chunks"] == 2


@pytest.mark.parametrize("case", [(True, 64, 64), (True, 32, 32), (True, 48, 48), (False, 64, 64), (False, 16, 16)],
                         ids=lambda c: "%s_%dx%d" % ("c64" if c[0] else "r64", c[1], c[2]))
@pytest.mark.parametrize("dist", ["uniform", "loguniform"])
def test_split_full_size_sampled(sp, case, dist):
    import torch
    import paper_1905_03136_gb300 as tsm
    cplx, M, N = case
    op = "C" if cplx else "T"
    dt = torch.complex128 if cplx else torch.float64
    A = torch.empty((K_FULL, M), dtype=dt, device="cuda")
    B = torch.empty((K_FULL, N), dtype=dt, device="cuda")
    tsm.fill_random(A, synth.SEED_A, dist)
    tsm.fill_random(B, synth.SEED_B, dist)
    Ch = host(sp.tsmttsm_split(A, B, op=op))
    assert sp.status() == 0
    del A, B
    torch.cuda.empty_cache()
    ms, ns = sorted({0, M - 1}), sorted({0, N // 2, N - 1})
    ca = {m: synth.column(synth.SEED_A, K_FULL, m, M, cplx, dist) for m in ms}
    cb = {n: synth.column(synth.SEED_B, K_FULL, n, N, cplx, dist) for n in ns}
    got = [Ch[m, n] for m in ms for n in ns]
    ref = [oracle.dot(op, ca[m], cb[n]) for m in ms for n in ns]
    assert oracle.rel_fro(np.array(got), np.array(ref)) <= TOL
