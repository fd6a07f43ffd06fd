"""Block Gram-Schmidt step through the C ABI (GPU required).

tsm_gs_step computes C = A^H B and B <- B - A C.  Checked against the CPU
oracle (both products), and by the property the step exists for: with A's
columns orthonormal (from a host QR factorisation, independent code), the
updated B is orthogonal to span(A) to rounding, A^H B' ~ 0 relative to B.
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
    import os
    import paper_1905_03136_gb300 as t
    from paper_1905_03136_gb300 import build, _lib
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    t.load()
    return t


def _orthonormal(K, M, cplx, ld=None):
    X = synth.block_vector(synth.SEED_A, K, M, complex_=cplx)
    Q, _ = np.linalg.qr(X)
    if ld is None or ld == M:
        return np.ascontiguousarray(Q)
    P = np.zeros((K, ld), dtype=Q.dtype)
    P[:, :M] = Q
    return P


@pytest.mark.parametrize("cplx,M,N,ldpad", [(True, 8, 8, 0), (True, 32, 16, 3), (False, 64, 64, 0),
                                            (False, 5, 3, 2), (True, 1, 64, 0), (False, 64, 1, 1)],
                         ids=["c64-8x8", "c64-32x16-ld", "r64-64x64", "r64-5x3-ld", "c64-1x64", "r64-64x1-ld"])
@pytest.mark.parametrize("mode", ["two_products", "fused"])
def test_gs_step_matches_oracle_and_orthogonalises(tsm, cplx, M, N, ldpad, mode):
    import torch
    K = (1 << 16) + 3
    Ap = _orthonormal(K, M, cplx, M + ldpad)
    A = Ap[:, :M]
    B0 = synth.block_vector(synth.SEED_B, K, N, complex_=cplx)
    Bp = np.zeros((K, N + ldpad), dtype=B0.dtype)
    Bp[:, :N] = B0
    dA = torch.from_numpy(Ap).cuda()[:, :M]
    dBp = torch.from_numpy(Bp).cuda()
    dB = dBp[:, :N]
    C = tsm.gs_step(dA, dB, mode=mode)
    torch.cuda.synchronize()
    C_ref = oracle.gram(A, B0, op="C")
    assert oracle.rel_fro(C.cpu().numpy(), C_ref) <= TOL
    B1 = dB.cpu().numpy()
    B_ref = oracle.apply(A, C_ref, alpha=-1.0, beta=1.0, B0=B0)
    assert oracle.rel_fro(B1, B_ref) <= TOL
    # B' is orthogonal to span(A): ||A^H B'|| <= a few ulps x ||B||
    resid = np.linalg.norm(oracle.gram(A, B1, op="C")) / np.linalg.norm(B0)
    assert resid <= 1e-13, resid
    # the padding columns between rows of B are never written
    if ldpad:
        assert torch.count_nonzero(dBp[:, N:]).item() == 0


def test_gs_step_k0_and_errors(tsm):
    import torch
    from paper_1905_03136_gb300 import _lib
    M, N = 4, 3
    A = torch.zeros((0, M), dtype=torch.float64, device="cuda")
    B = torch.zeros((0, N), dtype=torch.float64, device="cuda")
    C = torch.full((M, N), 7.0, dtype=torch.float64, device="cuda")
    tsm.gs_step(A, B, C)
    torch.cuda.synchronize()
    assert torch.count_nonzero(C).item() == 0  # K = 0: C = A^H B = 0

    K = 1000
    A = torch.ones((K, M), dtype=torch.float64, device="cuda")
    B = torch.ones((K, N), dtype=torch.float64, device="cuda")
    lib = tsm.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # C == NULL, ld too small, width out of range: nothing is launched, B unchanged
    assert lib.tsm_gs_step(0, M, N, K, ctypes.c_void_p(A.data_ptr()), M, ctypes.c_void_p(B.data_ptr()), N,
                           None, N, s) == 1
    assert lib.tsm_gs_step(0, M, N, K, ctypes.c_void_p(A.data_ptr()), M, ctypes.c_void_p(B.data_ptr()), N,
                           ctypes.c_void_p(C.data_ptr()), N - 1, s) == 1
    assert lib.tsm_gs_step(0, 65, N, K, ctypes.c_void_p(A.data_ptr()), 65, ctypes.c_void_p(B.data_ptr()), N,
                           ctypes.c_void_p(C.data_ptr()), N, s) == 2
    torch.cuda.synchronize()
    assert torch.all(B == 1.0).item()


def test_gs_step_twice_reorthogonalises(tsm):
    """A second pass removes what rounding left: the coefficients of the
    second pass are at rounding level relative to the first."""
    import torch
    K, M, N = (1 << 15) + 7, 16, 16
    A = _orthonormal(K, M, True)
    B0 = synth.block_vector(synth.SEED_B, K, N, complex_=True)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B0).cuda()
    C1 = tsm.gs_step(dA, dB)
    C2 = tsm.gs_step(dA, dB)
    torch.cuda.synchronize()
    r = (torch.linalg.norm(C2) / torch.linalg.norm(C1)).item()
    assert r <= 1e-13, r


@pytest.mark.parametrize("cplx,M,N", [(False, 1, 1), (True, 1, 1), (False, 17, 3), (True, 3, 17), (True, 64, 64),
                                      (False, 64, 64), (False, 8, 8), (False, 63, 63), (True, 37, 53)])
@pytest.mark.parametrize("K", [1, 31, 1000, (1 << 20) + 5])
def test_gs_fused_matches_oracle_and_repeats(tsm, cplx, M, N, K):
    """The fused kernel at row counts below, near and far above the grid
    (fewer rows than CTAs, ragged ranges): C and B against the oracle, and
    bit for bit the same on a second run from the same B."""
    import torch
    if K > 100000 and M * N > 64:
        K = (1 << 17) + 5  # keeps the oracle's product within seconds
    A = synth.block_vector(synth.SEED_A, K, M, complex_=cplx)
    B0 = synth.block_vector(synth.SEED_B, K, N, complex_=cplx)
    dA = torch.from_numpy(A).cuda()
    outs = []
    for _ in range(2):
        dB = torch.from_numpy(B0).cuda()
        C = tsm.gs_step(dA, dB, mode="fused")
        torch.cuda.synchronize()
        outs.append((C.cpu().numpy(), dB.cpu().numpy()))
    tsm.gs_status()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    C_ref = oracle.gram(A, B0, op="C")
    assert oracle.rel_fro(outs[0][0], C_ref) <= TOL
    B_ref = oracle.apply(A, C_ref, alpha=-1.0, beta=1.0, B0=B0)
    assert oracle.rel_fro(outs[0][1], B_ref) <= TOL


def test_gs_fused_k0_sets_c_to_zero(tsm):
    import torch
    A = torch.zeros((0, 5), dtype=torch.complex128, device="cuda")
    B = torch.zeros((0, 4), dtype=torch.complex128, device="cuda")
    C = torch.full((5, 4), 3.0 + 1.0j, dtype=torch.complex128, device="cuda")
    tsm.gs_step(A, B, C, mode="fused")
    torch.cuda.synchronize()
    assert torch.count_nonzero(C).item() == 0


def test_gs_fused_barrier_timeout_is_reported(tsm):
    """A one-cycle barrier budget makes the waiting CTAs give up (no fault,
    no hang: the last CTA to arrive still releases the barrier); the status
    call reports TIMEOUT once, and the next step with the default budget is
    correct again."""
    import torch
    from paper_1905_03136_gb300 import _lib
    K, M, N = (1 << 18) + 3, 8, 8
    A = synth.block_vector(synth.SEED_A, K, M)
    B0 = synth.block_vector(synth.SEED_B, K, N)
    dA = torch.from_numpy(A).cuda()
    try:
        tsm.gs_set_timeout(1)
        tsm.gs_step(dA, torch.from_numpy(B0).cuda(), mode="fused")
        with pytest.raises(_lib.TsmError) as e:
            tsm.gs_status()
        assert e.value.status == 5  # TSM_ERR_TIMEOUT
        tsm.gs_status()  # the word was cleared
    finally:
        tsm.gs_set_timeout(0)
    dB = torch.from_numpy(B0).cuda()
    C = tsm.gs_step(dA, dB, mode="fused")
    tsm.gs_status()
    C_ref = oracle.gram(A, B0, op="C")
    assert oracle.rel_fro(C.cpu().numpy(), C_ref) <= TOL
    assert oracle.rel_fro(dB.cpu().numpy(), oracle.apply(A, C_ref, alpha=-1.0, beta=1.0, B0=B0)) <= TOL


def test_gs_step_ex_rejects_unknown_mode(tsm):
    import torch
    lib = tsm.load()
    A = torch.ones((100, 2), dtype=torch.float64, device="cuda")
    B = torch.ones((100, 2), dtype=torch.float64, device="cuda")
    C = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.tsm_gs_step_ex(0, 2, 2, 100, ctypes.c_void_p(A.data_ptr()), 2, ctypes.c_void_p(B.data_ptr()), 2,
                              ctypes.c_void_p(C.data_ptr()), 2, 7, s) == 1
    torch.cuda.synchronize()
    assert torch.all(B == 1.0).item()
