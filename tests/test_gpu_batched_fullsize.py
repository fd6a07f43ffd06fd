"""The 256-instance mixed batched workload exactly as the benchmark times it
(`bench.batched_workload`: op and dtype 50/50, M, N uniform in [1, 64], K
log-uniform in [2^16, 2^22]; operands read from the two seeded pools, the
default configurations and item split, one graph launch), GPU required.

Every instance is checked on sampled outputs that the oracle computes one by
one from host-generated data: for each TSMTTSM instance the entries (0, 0),
(M-1, N-1) and (M/2, N/2) as oracle dot products of the host-generated
columns; for each TSMM instance its first and last rows and 30 random rows
through the oracle's row product.  Each instance must meet the normwise bar
on its own samples, so one wrong instance cannot hide among the others.
"""

import concurrent.futures as cf
import os

import numpy as np
import pytest

import bench
import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _pool():
    return cf.ThreadPoolExecutor(max(2, min(16, os.cpu_count() or 2)))


def test_batched_workload_full_size_sampled():
    import torch
    import paper_1905_03136_gb300 as tsm
    tsm.load()
    insts = bench.batched_workload()
    KK = max(i[4] for i in insts)
    flatA = torch.empty(KK * 128, dtype=torch.float64, device="cuda")
    flatB = torch.empty(KK * 128, dtype=torch.float64, device="cuda")
    tsm.fill_random(flatA.view(KK, 128), synth.SEED_A)
    tsm.fill_random(flatB.view(KK, 128), synth.SEED_B)
    views = bench.batched_views(flatA, flatB, insts)
    batch = bench.batched_make(insts, views, [0] * len(insts))
    batch.run()
    torch.cuda.synchronize()
    items, ctas = batch.info()
    batch.close()
    assert items >= len(insts) and ctas >= 152

    rng = np.random.default_rng(3)
    samples = []  # (instance, got, reference job)
    with _pool() as ex:
        for i, ((kind, cplx, M, N, K), (A, B, O)) in enumerate(zip(insts, views)):
            if kind == 0:
                Ch = O.cpu().numpy()
                pairs = sorted({(0, 0), (M - 1, N - 1), (M // 2, N // 2)})
                op = "C" if cplx else "T"
                for (m, n) in pairs:
                    a = ex.submit(synth.column, synth.SEED_A, K, m, M, cplx)
                    b = ex.submit(synth.column, synth.SEED_B, K, n, N, cplx)
                    job = ex.submit(lambda a=a, b=b, op=op: oracle.dot(op, a.result(), b.result()))
                    samples.append((i, np.array([Ch[m, n]]), job))
            else:
                rows = np.unique(np.concatenate([[0, K - 1], rng.integers(0, K, 30)]))
                got = O.index_select(0, torch.from_numpy(rows).cuda()).cpu().numpy()
                Ah = synth.rows_at(synth.SEED_A, rows, M, cplx)
                Cm = synth.small_matrix(synth.SEED_B, M, N, complex_=cplx)
                job = ex.submit(oracle.apply, Ah, Cm)
                samples.append((i, got.ravel(), job))
        per = {}
        for i, got, job in samples:
            g, r = per.setdefault(i, ([], []))
            g.extend(np.ravel(got))
            r.extend(np.ravel(job.result()))
    del views
    torch.cuda.empty_cache()
    assert len(per) == len(insts)
    bad = []
    for i, (g, r) in per.items():
        err = oracle.rel_fro(np.array(g), np.array(r))
        if not err <= TOL:
            bad.append((insts[i], err))
    assert not bad, bad[:5]
