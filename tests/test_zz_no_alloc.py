"""The allocation-free TSMTTSM entry point, through the C ABI.

It exists for callers that may not allocate device memory (a pool or arena
that owns the GPU, code that must not hit the device synchronization of a
cudaMalloc).  It must give the same products as tsm_tsmttsm -- within the
1e-12 normwise tolerance of the other parity tests -- on consecutive calls
that reuse its fixed scratch array.  Kept in its own file, named to be
collected last.
"""

import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _rel(x, ref):
    return np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel())


@pytest.mark.parametrize("case", [(False, 64, 64), (True, 64, 64), (False, 7, 5), (True, 1, 64), (True, 33, 9)],
                         ids=lambda c: "%s_%dx%d" % ("c64" if c[0] else "r64", c[1], c[2]))
def test_noalloc_matches_allocating_entry_point(case):
    import torch
    import paper_1905_03136_gb300 as tsm
    from paper_1905_03136_gb300 import _lib
    from paper_1905_03136_gb300._lib import scalar
    import paper_1905_03136_gb300.noalloc  # noqa: F401  (registers the signature)
    lib = tsm.load()
    cplx, M, N = case
    K = 50021
    dt = 1 if cplx else 0
    op = 2 if cplx else 1
    A = torch.from_numpy(synth.block_vector(0, K, M, complex_=cplx)).cuda()
    B = torch.from_numpy(synth.block_vector(1, K, N, complex_=cplx)).cuda()
    C0 = synth.small_matrix(2, M, N, complex_=cplx)
    alpha, beta = (0.75 + 0.5j, -1.5 + 0.25j) if cplx else (0.75, -1.5)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    ref = torch.from_numpy(C0.copy()).cuda()
    st = lib.tsm_tsmttsm(op, dt, M, N, K, scalar(alpha, cplx), ctypes.c_void_p(A.data_ptr()), M,
                         ctypes.c_void_p(B.data_ptr()), N, scalar(beta, cplx), ctypes.c_void_p(ref.data_ptr()),
                         N, stream)
    assert st == 0
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for _ in range(2):  # two calls in a row share the scratch array
        out = torch.from_numpy(C0.copy()).cuda()
        st = _lib.raw("tsm_tsmttsm_noalloc")(op, dt, M, N, K, scalar(alpha, cplx), ctypes.c_void_p(A.data_ptr()),
                                             M, ctypes.c_void_p(B.data_ptr()), N, scalar(beta, cplx),
                                             ctypes.c_void_p(out.data_ptr()), N, stream)
        assert st == 0
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy(), ref) <= TOL
