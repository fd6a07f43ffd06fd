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
def test_gs_step_matches_oracle_and_orthogonalises(tsm, cplx, M, N, ldpad):
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
    C = tsm.gs_step(dA, dB)
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
