"""Products launched back to back on one stream (GPU required).

The product kernels are launched with programmatic dependent launch: the
next product on a stream is scheduled while the previous one drains, reads
its inputs early only when the host found that the previous product wrote
none of them, and waits for it before writing.  Every chain below is run
twice -- once with the stream drained after every call, once with no
synchronisation at all -- and the results must agree bit for bit (the
reductions are deterministic, so any read of stale data or write racing the
previous call shows up as a difference).  The drained results are checked
against the oracle, so both runs are also correct.
"""

import os

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
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    t.load()
    return t


def _dev(tsm, rows, cols, cplx, seed):
    import torch
    t = torch.empty((rows, cols), dtype=torch.complex128 if cplx else torch.float64, device="cuda")
    tsm.fill_random(t, seed=seed)
    return t


def _run_twice(chain):
    import torch
    torch.cuda.synchronize()
    drained = [x.cpu().numpy() for x in chain(True)]
    torch.cuda.synchronize()
    free = [x.cpu().numpy() for x in chain(False)]
    assert len(drained) == len(free)
    for i, (d, f) in enumerate(zip(drained, free)):
        assert np.array_equal(d, f), "result %d differs when the calls are not drained" % i
    return drained


@pytest.mark.parametrize("cplx", [False, True], ids=["r64", "c64"])
def test_tsmm_then_tsmttsm_reads_fresh_output(tsm, cplx):
    """V = A C_i (TSMM writes V), then G_i = op(A)^T V reads it at once."""
    import torch
    K, M, N = 1 << 20, 4, 6
    A = _dev(tsm, K, M, cplx, 11)
    Cs = [_dev(tsm, M, N, cplx, 20 + i) for i in range(6)]
    V = torch.empty((K, N), dtype=A.dtype, device="cuda")
    op = "C" if cplx else "T"

    def chain(drain):
        out = []
        for Ci in Cs:
            tsm.tsmm(A, Ci, V)
            if drain:
                torch.cuda.synchronize()
            out.append(tsm.tsmttsm(A, V, op=op))
            if drain:
                torch.cuda.synchronize()
        return out
    res = _run_twice(chain)
    Ah = A.cpu().numpy()
    for Ci, G in zip(Cs, res):
        V_ref = oracle.apply(Ah, Ci.cpu().numpy())
        assert oracle.rel_fro(G, oracle.gram(Ah, V_ref, op)) <= TOL


@pytest.mark.parametrize("cplx", [False, True], ids=["r64", "c64"])
def test_tsmm_accumulation_chain(tsm, cplx):
    """B <- B + A C_i, each call reading the previous call's output."""
    import torch
    K, M, N = 1 << 19, 3, 5
    A = _dev(tsm, K, M, cplx, 31)
    Cs = [_dev(tsm, M, N, cplx, 40 + i) for i in range(5)]
    B0 = _dev(tsm, K, N, cplx, 32)

    def chain(drain):
        B = B0.clone()
        for Ci in Cs:
            tsm.tsmm(A, Ci, B, 1.0, 1.0)
            if drain:
                torch.cuda.synchronize()
        return [B]
    (got,) = _run_twice(chain)
    Ah = A.cpu().numpy()
    ref = B0.cpu().numpy()
    for Ci in Cs:
        ref = oracle.apply(Ah, Ci.cpu().numpy(), 1.0, 1.0, ref)
    assert oracle.rel_fro(got, ref) <= TOL


def test_tsmttsm_output_feeds_next_tsmttsm(tsm):
    """C_1 = A^T B (K = 2^20), then C_2 = C_1^T C_1 with C_1 as a 64-row block
    vector: the second call's inputs are the first call's output."""
    import torch
    K, W = 1 << 20, 64
    A = _dev(tsm, K, W, False, 51)
    B = _dev(tsm, K, W, False, 52)

    def chain(drain):
        out = []
        for _ in range(4):
            C1 = tsm.tsmttsm(A, B)
            if drain:
                torch.cuda.synchronize()
            out.append(tsm.tsmttsm(C1, C1))
            if drain:
                torch.cuda.synchronize()
        return out
    res = _run_twice(chain)
    c1 = oracle.gram(A.cpu().numpy(), B.cpu().numpy())
    assert oracle.rel_fro(res[0], oracle.gram(c1, c1)) <= 1e-11


@pytest.mark.parametrize("w", [1, 2, 8, 64])
def test_independent_products_read_early(tsm, w):
    """Products on the same inputs into separate outputs: each may read its
    inputs before the previous one completes (the early path)."""
    import torch
    K = 1 << 22 if w <= 2 else 1 << 20
    A = _dev(tsm, K, w, False, 61)
    B = _dev(tsm, K, w, False, 62)
    outs = [torch.empty((w, w), dtype=torch.float64, device="cuda") for _ in range(6)]

    def chain(drain):
        for C in outs:
            C.fill_(np.nan)
        torch.cuda.synchronize()
        for C in outs:
            tsm.tsmttsm(A, B, C)
            if drain:
                torch.cuda.synchronize()
        return outs
    res = _run_twice(chain)
    for r in res[1:]:
        assert np.array_equal(r, res[0])
    ref = oracle.gram(synth.block_vector(61, K, w), synth.block_vector(62, K, w))
    assert oracle.rel_fro(res[0], ref) <= TOL


@pytest.mark.parametrize("cplx", [False, True], ids=["r64", "c64"])
def test_gram_schmidt_steps_back_to_back(tsm, cplx):
    """Repeated C = A^H B, B <- B - A C on the same B (each product depends
    on the other's output)."""
    import torch
    K, M, N = 1 << 20, 8, 8
    A = _dev(tsm, K, M, cplx, 71)
    B0 = _dev(tsm, K, N, cplx, 72)

    def chain(drain):
        B = B0.clone()
        out = []
        for _ in range(3):
            out.append(tsm.gs_step(A, B))
            if drain:
                torch.cuda.synchronize()
        out.append(B)
        return out
    _run_twice(chain)

