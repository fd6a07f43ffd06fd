"""Multi-rank host logic on CPU (gloo, world size 2).

The library runs one process per GPU as independent replicas; the only
cross-rank steps are the benchmark's barrier and its max-over-ranks time.
The K-partitioned TSMTTSM (each rank a contiguous range of rows, partials
summed in rank order) is checked here with oracle partials: the rank-order
sum must equal the single-process oracle to rounding, and be bitwise the
same on every rank.
"""

import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # max over ranks: every rank sees the slowest rank's time
        got = bench.max_over_ranks(1.5 + rank)
        assert got == 1.5 + (world - 1), got

        # K-partitioned TSMTTSM, complex A^H B, ragged split of K
        K, M, N = 1001, 5, 3
        A = synth.block_vector(synth.SEED_A, K, M, complex_=True)
        B = synth.block_vector(synth.SEED_B, K, N, complex_=True)
        bounds = [0, 613, K]  # deliberately uneven ranges
        r0, r1 = bounds[rank], bounds[rank + 1]
        part = oracle.gram(A[r0:r1], B[r0:r1], op="C")
        parts = [torch.zeros((M, N), dtype=torch.complex128) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(np.ascontiguousarray(part)))
        total = np.zeros((M, N), dtype=np.complex128)
        for p in parts:  # fixed rank order
            total = total + p.numpy()
        ref = oracle.gram(A, B, op="C")
        assert oracle.rel_fro(total, ref) < 1e-14
        np.save(os.path.join(out_dir, "total_%d.npy" % rank), total)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_partition_and_max_over_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    oracle.build()  # compile once in the parent, not concurrently in both ranks
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    t0 = np.load(tmp_path / "total_0.npy")
    t1 = np.load(tmp_path / "total_1.npy")
    assert np.array_equal(t0.view(np.float64), t1.view(np.float64))  # bitwise, every rank


def test_max_over_ranks_single_process():
    pytest.importorskip("torch")
    import bench
    assert bench.max_over_ranks(3.25) == 3.25


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
