"""The allocation-free TSMTTSM entry point, through the C ABI.

It exists for callers that may not allocate device memory (a pool or arena
that owns the GPU, code that must not hit the device synchronization of a
cudaMalloc).  It must give the oracle's products within the 1e-12
normwise tolerance of the other parity tests, the same bits as tsm_tsmttsm
(it runs the same kernel, grid and reduction order), and the same bits on
two consecutive calls that reuse its fixed scratch array.  The shapes cover
the vector-streamed narrow kernels (real widths <= 4, complex <= 2), the
generated and hand-written tiles, the final-kernel reduction (complex
64 x 64) and the scale-only branch (K = 0, alpha = 0).  Kept in its own
file, named to be collected last.
"""

import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 1e-12

CASES = [(False, 1, 1), (False, 4, 4), (True, 2, 2), (True, 1, 1), (False, 64, 64), (True, 64, 64),
         (False, 7, 5), (True, 1, 64), (True, 33, 9)]


def _call(fn_name, op, dt, M, N, K, alpha, A, B, beta, C, cplx, stream):
    from paper_1905_03136_gb300 import _lib
    from paper_1905_03136_gb300._lib import scalar
    import paper_1905_03136_gb300.noalloc  # noqa: F401  (registers the signature)
    fn = _lib.raw(fn_name)
    return fn(op, dt, M, N, K, scalar(alpha, cplx), ctypes.c_void_p(A.data_ptr() if A is not None else 0), M,
              ctypes.c_void_p(B.data_ptr() if B is not None else 0), N, scalar(beta, cplx),
              ctypes.c_void_p(C.data_ptr()), N, stream)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s_%dx%d" % ("c64" if c[0] else "r64", c[1], c[2]))
def test_noalloc_matches_oracle_and_allocating_entry_point(case):
    import torch
    import paper_1905_03136_gb300 as tsm
    tsm.load()
    cplx, M, N = case
    K = 50021
    dt = 1 if cplx else 0
    op = 2 if cplx else 1
    hA = synth.block_vector(0, K, M, complex_=cplx)
    hB = synth.block_vector(1, K, N, complex_=cplx)
    A = torch.from_numpy(hA).cuda()
    B = torch.from_numpy(hB).cuda()
    C0 = synth.small_matrix(2, M, N, complex_=cplx)
    alpha, beta = (0.75 + 0.5j, -1.5 + 0.25j) if cplx else (0.75, -1.5)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    want = oracle.gram(hA, hB, "C" if cplx else "T", alpha, beta, C0)

    ref = torch.from_numpy(C0.copy()).cuda()
    assert _call("tsm_tsmttsm", op, dt, M, N, K, alpha, A, B, beta, ref, cplx, stream) == 0
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    outs = []
    for _ in range(2):  # two calls in a row share the scratch array
        out = torch.from_numpy(C0.copy()).cuda()
        assert _call("tsm_tsmttsm_noalloc", op, dt, M, N, K, alpha, A, B, beta, out, cplx, stream) == 0
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    for got in outs:
        assert oracle.rel_fro(got, want) <= TOL
        # same kernel, grid and reduction order as tsm_tsmttsm on this GPU
        assert np.array_equal(got, ref)
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("cplx", [False, True], ids=["r64", "c64"])
def test_noalloc_scale_only(cplx):
    """K = 0 and alpha = 0 leave C = beta * C (the inputs are not read)."""
    import torch
    import paper_1905_03136_gb300 as tsm
    tsm.load()
    M, N = 5, 3
    dt = 1 if cplx else 0
    op = 2 if cplx else 1
    C0 = synth.small_matrix(2, M, N, complex_=cplx, dist="smallint")
    beta = (0.5 - 2.0j) if cplx else -0.5
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    A = torch.from_numpy(synth.block_vector(0, 16, M, complex_=cplx)).cuda()
    B = torch.from_numpy(synth.block_vector(1, 16, N, complex_=cplx)).cuda()
    for (K, alpha, a, b) in ((0, 1.0, None, None), (16, 0.0, A, B)):
        out = torch.from_numpy(C0.copy()).cuda()
        assert _call("tsm_tsmttsm_noalloc", op, dt, M, N, K, alpha, a, b, beta, out, cplx, stream) == 0
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), beta * C0)
