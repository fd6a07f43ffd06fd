"""Batched persistent launch: every instance against the oracle; graph
replays bitwise identical; every per-instance configuration code correct."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _make(seed, n, kmax_log2=15):
    """n random instances: TSMTTSM/TSMM, real/complex, M, N in [1, 64],
    K log-uniform in [2^8, 2^kmax_log2] (small enough for the oracle)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = int(rng.integers(0, 2))
        cplx = bool(rng.integers(0, 2))
        M, N = int(rng.integers(1, 65)), int(rng.integers(1, 65))
        K = int(2 ** rng.uniform(8, kmax_log2))
        out.append((kind, cplx, M, N, K))
    return out


def _build(insts, configs=None, beta=0.0):
    import torch
    from paper_1905_03136_gb300 import batched as bt
    descs, host, dev = [], [], []
    for i, (kind, cplx, M, N, K) in enumerate(insts):
        A = synth.block_vector(100 + i, K, M, complex_=cplx)
        if kind == bt.TSMTTSM:
            B = synth.block_vector(300 + i, K, N, complex_=cplx)
            O = synth.small_matrix(500 + i, M, N, complex_=cplx)
        else:
            B = synth.small_matrix(300 + i, M, N, complex_=cplx)
            O = synth.block_vector(500 + i, K, N, complex_=cplx)
        dA, dB, dO = (torch.from_numpy(x).cuda() for x in (A, B, O))
        op = ("C" if cplx else "T") if kind == bt.TSMTTSM else "N"
        descs.append(bt.desc(kind, dA, dB, dO, 1.5, beta, op, configs[i] if configs else 0))
        host.append((A, B, O, op))
        dev.append((dA, dB, dO))
    return bt.Batch(descs), host, dev


def _ref(kind, A, B, O, op, beta):
    if kind == 0:
        return oracle.gram(A, B, op, 1.5, beta, O)
    return oracle.apply(A, B, 1.5, beta, O)


@pytest.fixture(scope="module")
def lib():
    import os
    import paper_1905_03136_gb300 as t
    from paper_1905_03136_gb300 import build, _lib
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return t.load()


def test_batched_random_instances_and_replay(lib):
    import torch
    insts = _make(1, 40)
    batch, host, dev = _build(insts, beta=0.0)
    batch.run()
    torch.cuda.synchronize()
    first = [d[2].cpu().numpy().copy() for d in dev]
    for (kind, cplx, M, N, K), (A, B, O, op), got in zip(insts, host, first):
        assert oracle.rel_fro(got, _ref(kind, A, B, O, op, 0.0)) <= TOL, (kind, cplx, M, N, K)
    for _ in range(3):  # replays: bit for bit (outputs are overwritten since beta = 0)
        batch.run()
        torch.cuda.synchronize()
        for d, f in zip(dev, first):
            assert np.array_equal(d[2].cpu().numpy(), f)
    batch.run_direct()
    torch.cuda.synchronize()
    for d, f in zip(dev, first):
        assert np.array_equal(d[2].cpu().numpy(), f)
    items, ctas = batch.info()
    assert items >= len(insts) and ctas >= 152


@pytest.mark.parametrize("code", list(range(1, 15)))
def test_batched_every_tsmttsm_tile_code(lib, code):
    """Every tile code on shapes that pad it and shapes it cannot take (more
    than 256 threads: the default tile runs instead)."""
    import torch
    insts = [(0, c, M, N, 20000) for c in (False, True)
             for (M, N) in ((1, 1), (5, 7), (16, 16), (64, 64), (3, 64), (37, 53), (64, 61))]
    configs = [code | (12 << 8)] * len(insts)  # 4096-row items
    batch, host, dev = _build(insts, configs, beta=0.5)
    batch.run()
    torch.cuda.synchronize()
    for (kind, cplx, M, N, K), (A, B, O, op), d in zip(insts, host, dev):
        assert oracle.rel_fro(d[2].cpu().numpy(), _ref(kind, A, B, O, op, 0.5)) <= TOL, (code, cplx, M, N)


@pytest.mark.parametrize("code", [1, 2, 3, 4])
def test_batched_every_tsmm_code(lib, code):
    import torch
    insts = [(1, c, M, N, 9000) for c in (False, True)
             for (M, N) in ((1, 1), (7, 5), (64, 64), (4, 64), (64, 4), (13, 39), (54, 17))]
    batch, host, dev = _build(insts, [code | (10 << 8)] * len(insts), beta=-1.0)
    batch.run()
    torch.cuda.synchronize()
    for (kind, cplx, M, N, K), (A, B, O, op), d in zip(insts, host, dev):
        assert oracle.rel_fro(d[2].cpu().numpy(), _ref(kind, A, B, O, op, -1.0)) <= TOL, (code, cplx, M, N)


def test_batched_rejects_bad_descriptor(lib):
    import torch
    from paper_1905_03136_gb300 import batched as bt
    from paper_1905_03136_gb300._lib import TsmError
    A = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
    B = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    O = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    d = bt.desc(0, A, B, O)
    d.M = 65
    with pytest.raises(TsmError):
        bt.Batch([d])
    d = bt.desc(1, A, torch.zeros((4, 3), dtype=torch.float64, device="cuda"), B, op="N")
    d.op = 1
    with pytest.raises(TsmError):
        bt.Batch([d])
