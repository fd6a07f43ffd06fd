"""Full-size parity at K = 2^24 (the benchmark workload), GPU required.

Inputs are generated on the device with the library's SplitMix64 fill (a
separate test checks it bit for bit against the host generator) and the
products run in the same launch configuration as the benchmark (the
library's default choice).  The oracle cannot hold these matrices, so it
recomputes samples one by one from host-generated columns and rows:
  * TSMTTSM: entries C[m][n] on the corners and a middle row/column of C,
    each a 2^24-term compensated dot product of two generated columns;
  * TSMM: the first and last 4096 rows and 2^14 random rows of B, each
    recomputed from the generated row of A.
The bar is the normwise relative error over the sample, <= 1e-12.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
K_FULL = 1 << 24
TOL = 1e-12


@pytest.fixture(scope="module")
def tsm():
    import os
    import paper_1905_03136_gb300 as t
    from paper_1905_03136_gb300 import build, _lib
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    t.load()
    return t


def _fill(tsm, rows, cols, cplx, seed, dist="uniform"):
    import torch
    t = torch.empty((rows, cols), dtype=torch.complex128 if cplx else torch.float64, device="cuda")
    tsm.fill_random(t, seed=seed, dist=dist)
    return t


TSMTTSM_CASES = [(False, 1, 1), (False, 4, 4), (False, 64, 64), (False, 1, 64), (False, 64, 1),
                 (False, 8, 32), (True, 1, 1), (True, 32, 32), (True, 64, 64), (True, 32, 8)]


@pytest.mark.parametrize("case", TSMTTSM_CASES, ids=lambda c: "%s_%dx%d" % ("c64" if c[0] else "r64", c[1], c[2]))
def test_tsmttsm_full_size_sampled(tsm, case):
    import torch
    cplx, M, N = case
    op = "C" if cplx else "T"
    A = _fill(tsm, K_FULL, M, cplx, synth.SEED_A)
    B = _fill(tsm, K_FULL, N, cplx, synth.SEED_B)
    C = tsm.tsmttsm(A, B, op=op)
    torch.cuda.synchronize()
    Ch = C.cpu().numpy()
    del A, B
    torch.cuda.empty_cache()
    ms = sorted({0, M // 2, M - 1})
    ns = sorted({0, N // 2, N - 1})
    cols_a = {m: synth.column(synth.SEED_A, K_FULL, m, M, cplx) for m in ms}
    cols_b = {n: synth.column(synth.SEED_B, K_FULL, n, N, cplx) for n in ns}
    got, ref = [], []
    for m in ms:
        for n in ns:
            ref.append(oracle.dot(op, cols_a[m], cols_b[n]))
            got.append(Ch[m, n])
    assert oracle.rel_fro(np.array(got), np.array(ref)) <= TOL


TSMM_CASES = [(False, 1, 1, 0.0), (False, 64, 64, 0.0), (False, 64, 64, 1.0), (False, 4, 64, 0.0),
              (True, 64, 64, 1.0), (True, 7, 7, 0.0), (True, 64, 4, 0.0)]


@pytest.mark.parametrize("case", TSMM_CASES,
                         ids=lambda c: "%s_%dx%d_b%g" % ("c64" if c[0] else "r64", c[1], c[2], c[3]))
def test_tsmm_full_size_sampled_rows(tsm, case):
    import torch
    cplx, M, N, beta = case
    A = _fill(tsm, K_FULL, M, cplx, synth.SEED_A)
    Cm = _fill(tsm, M, N, cplx, synth.SEED_C)
    B = _fill(tsm, K_FULL, N, cplx, synth.SEED_B)
    tsm.tsmm(A, Cm, B, 1.0, beta)
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([np.arange(4096), np.arange(K_FULL - 4096, K_FULL),
                                     rng.integers(0, K_FULL, 1 << 14)]))
    idx = torch.from_numpy(rows).cuda()
    got = B.index_select(0, idx).cpu().numpy()
    del A, B
    torch.cuda.empty_cache()
    Ah = synth.rows_at(synth.SEED_A, rows, M, cplx)
    Ch = synth.small_matrix(synth.SEED_C, M, N, complex_=cplx)
    B0 = synth.rows_at(synth.SEED_B, rows, N, cplx)
    ref = oracle.apply(Ah, Ch, 1.0, beta, B0)
    assert oracle.rel_fro(got, ref) <= TOL
