"""Full-size parity for every configuration of the width sweeps, GPU required.

Two checks per configuration, both at the production launch configuration
(the kernel variant and grid the library chooses for K = 2^24, i.e. what the
benchmark runs):
  * at K = 2^20 the whole output (all of C for TSMTTSM, all 2^20 rows of B
    for TSMM) is compared with the oracle's full product;
  * at K = 2^24 (the benchmark's size) sampled outputs are recomputed by the
    oracle one by one from host-generated columns and rows: five entries of
    C (corners and middle) for every TSMTTSM configuration, a full row and a
    full column of C for the 64 x 64 ones, and the first and last 4096 rows
    plus 2^14 random rows of B for TSMM.
Device inputs come from the library's SplitMix64 fill (checked bit for bit
against the host generator elsewhere); the oracle's inputs come from the
host generator only.  The bar is the normwise relative error over what is
compared, <= 1e-12.  The oracle products of the K = 2^20 checks run on a
thread pool (the C oracle releases the GIL) while the GPU tests proceed.
"""

import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
K_FULL = 1 << 24
K_MID = 1 << 20
TOL = 1e-12

SQUARE = (1, 2, 4, 8, 16, 32, 64)
TSMTTSM_SWEEP = [(c, m, n) for c in (False, True) for (m, n) in [(w, w) for w in SQUARE] +
                 [(1, 64), (64, 1), (8, 32), (32, 8)]]
TSMM_SWEEP = [(c, m, n, b) for c in (False, True) for (m, n) in [(w, w) for w in SQUARE] + [(4, 64), (64, 4)]
              for b in (0.0, 1.0)]


def _id3(c):
    return "%s_%dx%d" % ("c64" if c[0] else "r64", c[1], c[2])


def _id4(c):
    return "%s_%dx%d_b%g" % ("c64" if c[0] else "r64", c[1], c[2], c[3])


@pytest.fixture(scope="module")
def tsm():
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


class _MidRefs:
    """Host inputs at K = 2^20; the oracle's TSMTTSM products are computed on
    a thread pool as soon as the module starts, its TSMM products on demand
    with the rows split over threads (rows are independent, so this is the
    same arithmetic as one call)."""

    def __init__(self):
        # flat buffers: the first K*w(*2) doubles are the seeded input of
        # every width w (and complex width) with ld = w
        self.flatA = synth.block_vector(synth.SEED_A, K_MID, 128).reshape(-1)
        self.flatB = synth.block_vector(synth.SEED_B, K_MID, 128).reshape(-1)
        self.flatC = synth.block_vector(synth.SEED_C, 64, 128).reshape(-1)
        self.pool = cf.ThreadPoolExecutor(max(2, min(16, os.cpu_count() or 2)))
        self.jobs = {}
        # largest jobs first, so that they are ready in time
        work = [("tsmttsm",) + c for c in TSMTTSM_SWEEP]
        work.sort(key=lambda w: -w[2] * w[3] * (4 if w[1] else 1))
        for w in work:
            self.jobs[w] = self.pool.submit(self._ref, w)

    def view(self, flat, rows, cols, cplx):
        dt = np.complex128 if cplx else np.float64
        return flat[: rows * cols * (2 if cplx else 1)].view(dt).reshape(rows, cols)

    def _ref(self, w):
        _, cplx, M, N = w
        return oracle.gram(self.view(self.flatA, K_MID, M, cplx), self.view(self.flatB, K_MID, N, cplx),
                           "C" if cplx else "T")

    def tsmm_ref(self, cplx, M, N, beta):
        A = self.view(self.flatA, K_MID, M, cplx)
        Cm = np.ascontiguousarray(self.view(self.flatC, M, N, cplx))
        B = self.view(self.flatB, K_MID, N, cplx).copy() if beta else \
            np.zeros((K_MID, N), dtype=A.dtype)
        nt = 16
        cuts = [K_MID * t // nt for t in range(nt + 1)]

        def rows(t):
            k0, k1 = cuts[t], cuts[t + 1]
            oracle.tsmm(M, N, k1 - k0, 1.0, A[k0:k1], M, Cm, N, beta, B[k0:k1], N)

        with cf.ThreadPoolExecutor(nt) as ex:
            list(ex.map(rows, range(nt)))
        return B

    def result(self, w):
        return self.jobs.pop(w).result()


@pytest.fixture(scope="module")
def mid_refs():
    r = _MidRefs()
    yield r
    r.pool.shutdown(wait=False, cancel_futures=True)


@pytest.mark.parametrize("case", TSMTTSM_SWEEP, ids=_id3)
def test_tsmttsm_production_config_full_c(tsm, mid_refs, case):
    """All of C at K = 2^20 with the variant and grid chosen for K = 2^24."""
    import torch
    cplx, M, N = case
    dt = tsm.C64 if cplx else tsm.R64
    var, grid = tsm.choose(tsm.KIND_TSMTTSM, dt, M, N, K_FULL)
    A = _fill(tsm, K_MID, M, cplx, synth.SEED_A)
    B = _fill(tsm, K_MID, N, cplx, synth.SEED_B)
    C = tsm.tsmttsm(A, B, op="C" if cplx else "T", variant=var, grid=grid)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    ref = mid_refs.result(("tsmttsm", cplx, M, N))
    assert oracle.rel_fro(got, ref) <= TOL, (var, grid)


@pytest.mark.parametrize("case", TSMM_SWEEP, ids=_id4)
def test_tsmm_production_config_full_b(tsm, mid_refs, case):
    """All 2^20 rows of B with the variant and grid chosen for K = 2^24."""
    import torch
    cplx, M, N, beta = case
    dt = tsm.C64 if cplx else tsm.R64
    var, grid = tsm.choose(tsm.KIND_TSMM_BETA if beta else tsm.KIND_TSMM, dt, M, N, K_FULL)
    A = _fill(tsm, K_MID, M, cplx, synth.SEED_A)
    Cm = _fill(tsm, M, N, cplx, synth.SEED_C)
    B = _fill(tsm, K_MID, N, cplx, synth.SEED_B)
    tsm.tsmm(A, Cm, B, 1.0, beta, variant=var, grid=grid)
    torch.cuda.synchronize()
    got = B.cpu().numpy()
    del A, B
    ref = mid_refs.tsmm_ref(cplx, M, N, beta)
    assert oracle.rel_fro(got, ref) <= TOL, (var, grid)


def _columns(seed, K, cols, ld, cplx):
    with cf.ThreadPoolExecutor(max(2, min(16, os.cpu_count() or 2))) as ex:
        futs = {c: ex.submit(synth.column, seed, K, c, ld, cplx) for c in cols}
        return {c: f.result() for c, f in futs.items()}


def _dots(op, pairs, cols_a, cols_b):
    with cf.ThreadPoolExecutor(max(2, min(16, os.cpu_count() or 2))) as ex:
        futs = [ex.submit(oracle.dot, op, cols_a[m], cols_b[n]) for (m, n) in pairs]
        return [f.result() for f in futs]


@pytest.mark.parametrize("case", TSMTTSM_SWEEP, ids=_id3)
def test_tsmttsm_full_size_sampled(tsm, case):
    """K = 2^24 as the benchmark runs it: sampled entries of C against
    oracle dot products of host-generated columns (a full row and a full
    column of C for the 64 x 64 shapes)."""
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
    if M == N == 64:
        pairs = sorted({(0, n) for n in range(N)} | {(m, 0) for m in range(M)})
    else:
        pairs = sorted({(0, 0), (0, N - 1), (M - 1, 0), (M - 1, N - 1), (M // 2, N // 2)})
    cols_a = _columns(synth.SEED_A, K_FULL, sorted({m for m, _ in pairs}), M, cplx)
    cols_b = _columns(synth.SEED_B, K_FULL, sorted({n for _, n in pairs}), N, cplx)
    ref = _dots(op, pairs, cols_a, cols_b)
    got = [Ch[m, n] for (m, n) in pairs]
    assert oracle.rel_fro(np.array(got), np.array(ref)) <= TOL


TSMM_CASES = [(False, 1, 1, 0.0), (False, 64, 64, 0.0), (False, 64, 64, 1.0), (False, 4, 64, 0.0),
              (True, 64, 64, 1.0), (True, 7, 7, 0.0), (True, 64, 4, 0.0), (True, 1, 1, 1.0), (False, 2, 2, 1.0)]


@pytest.mark.parametrize("case", TSMM_CASES, ids=_id4)
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
