"""Binding of the allocation-free TSMTTSM entry point (include/tsm_noalloc.h),
for callers that cannot let a library allocate device memory."""

import ctypes

from . import _lib
from ._lib import scalar

_lib.extend_signatures({
    "tsm_tsmttsm_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p]),
})

SCRATCH_BYTES = 16 * 1024 * 1024
_OPS = {"T": 1, "C": 2}


def tsmttsm_noalloc(A, B, C, alpha=1.0, beta=0.0, op="T", stream=None):
    """C = alpha * op(A)^T B + beta * C into the caller's C, using only the
    library's fixed scratch array (no device allocation by the call)."""
    from . import _dtype_code, _ld, _stream
    dt = _dtype_code(A)
    K, M = A.shape
    N = B.shape[1]
    cplx = dt == 1
    _lib.call("tsm_tsmttsm_noalloc", _OPS[op], dt, M, N, K, scalar(alpha, cplx), ctypes.c_void_p(A.data_ptr()),
              _ld(A, "A"), ctypes.c_void_p(B.data_ptr()), _ld(B, "B"), scalar(beta, cplx),
              ctypes.c_void_p(C.data_ptr()), _ld(C, "C"), _stream(stream))
    return C
