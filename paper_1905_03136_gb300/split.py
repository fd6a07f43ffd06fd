"""Binding of the split-precision TSMTTSM (include/tsm_split.h)."""

import ctypes

from . import _lib
from ._lib import scalar

class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("ctas", "ctas_per_sm", "column_chunks", "converter_threads",
                                              "epilogue_warps", "threads_per_cta", "digit_stages", "tmem_columns",
                                              "smem_bytes")]


_lib.extend_signatures({
    "tsm_split_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                      ctypes.POINTER(PlanInfo)]),
    "tsm_tsmttsm_split": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "tsm_tsmttsm_split_ex": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_void_p]),
    "tsm_split_plan_ex": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                         ctypes.POINTER(PlanInfo)]),
    "tsm_split_status": (ctypes.c_int, [ctypes.c_void_p]),
    "tsm_split_set_timeout": (ctypes.c_int, [ctypes.c_int64]),
})

_OPS = {"T": 1, "C": 2}


DIGITS_F16 = 0


def tsmttsm_split(A, B, C=None, alpha=1.0, beta=0.0, op="T", stream=None, slices=6, kind=DIGITS_F16):
    """C = alpha * op(A)^T B + beta * C with the tensor-core split path
    (`slices` 8-bit slices per input, 4..6)."""
    import torch
    from . import _dtype_code, _ld, _stream
    dt = _dtype_code(A)
    K, M = A.shape
    N = B.shape[1]
    if C is None:
        C = torch.zeros((M, N), dtype=A.dtype, device=A.device)
        beta = 0.0
    cplx = dt == 1
    _lib.call("tsm_tsmttsm_split_ex", _OPS[op], dt, M, N, K, scalar(alpha, cplx), ctypes.c_void_p(A.data_ptr()),
              _ld(A, "A"), ctypes.c_void_p(B.data_ptr()), _ld(B, "B"), scalar(beta, cplx),
              ctypes.c_void_p(C.data_ptr()), _ld(C, "C"), int(kind), int(slices), _stream(stream))
    return C


def status(stream=None):
    """Raw status of the last split call on the stream (0 OK, 5 timeout)."""
    from . import _stream
    return _lib.raw("tsm_split_status")(_stream(stream))


def set_timeout(cycles):
    _lib.call("tsm_split_set_timeout", int(cycles))


def plan(dtype, M, N, K, slices=6):
    """The launch plan (dict) tsm_tsmttsm_split(_ex) would use for a shape;
    dtype is 0 (real) or 1 (complex)."""
    info = PlanInfo()
    _lib.call("tsm_split_plan_ex", int(dtype), int(M), int(N), int(K), int(slices), ctypes.byref(info))
    return {n: getattr(info, n) for n, _ in PlanInfo._fields_}
