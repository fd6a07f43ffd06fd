"""Binding of the batched persistent launch (include/tsm_batched.h)."""

import ctypes

from . import _lib


class BatchDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("op", ctypes.c_int), ("dtype", ctypes.c_int), ("M", ctypes.c_int),
                ("N", ctypes.c_int), ("K", ctypes.c_int64), ("alpha", ctypes.c_double * 2),
                ("beta", ctypes.c_double * 2), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("out", ctypes.c_void_p),
                ("ldo", ctypes.c_int64), ("config", ctypes.c_int)]


_lib.extend_signatures({
    "tsm_batched_create": (ctypes.c_int, [ctypes.POINTER(BatchDesc), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "tsm_batched_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "tsm_batched_run_direct": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "tsm_batched_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]),
    "tsm_batched_destroy": (None, [ctypes.c_void_p]),
})

TSMTTSM, TSMM = 0, 1
OPS = {"N": 0, "T": 1, "C": 2}


def desc(kind, A, B, out, alpha=1.0, beta=0.0, op=None, config=0):
    """One instance from device tensors: TSMTTSM (A: K x M, B: K x N, out: M x N)
    or TSMM (A: K x M, B = C: M x N, out: K x N)."""
    import torch
    cplx = A.dtype == torch.complex128
    d = BatchDesc()
    d.kind = kind
    d.op = OPS[op or ("T" if kind == TSMTTSM else "N")]
    d.dtype = 1 if cplx else 0
    d.M = A.shape[1]
    d.N = B.shape[1]
    d.K = A.shape[0]
    a, b = complex(alpha), complex(beta)
    d.alpha[0], d.alpha[1] = a.real, a.imag
    d.beta[0], d.beta[1] = b.real, b.imag
    d.A, d.lda = A.data_ptr(), max(A.stride(0), A.shape[1])
    d.B, d.ldb = B.data_ptr(), max(B.stride(0), B.shape[1])
    d.out, d.ldo = out.data_ptr(), max(out.stride(0), out.shape[1])
    d.config = int(config)
    return d


class Batch:
    def __init__(self, descs):
        arr = (BatchDesc * len(descs))(*descs)
        h = ctypes.c_void_p()
        _lib.call("tsm_batched_create", arr, len(descs), ctypes.byref(h))
        self.h = h

    def _stream(self, stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(s.cuda_stream)

    def run(self, stream=None):
        _lib.call("tsm_batched_run", self.h, self._stream(stream))

    def run_direct(self, stream=None):
        _lib.call("tsm_batched_run_direct", self.h, self._stream(stream))

    def info(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _lib.call("tsm_batched_info", self.h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def close(self):
        if self.h:
            _lib.load().tsm_batched_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
