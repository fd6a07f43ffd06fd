"""CPU oracle for TSMTTSM and TSMM (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The CUDA library never calls it, and it
shares no code with the library: the products are computed by the plain C
file ``tsm_oracle.c`` (the definition of Sec. 1.1 / Listing 1 written out
in binary64 with compensated summation), compiled here with gcc.
``tsm_plain.c`` holds both products as plain uncompensated loops, threaded
over K: the timed CPU baseline (``tsmttsm_plain``, ``tsmm_plain``), never a
parity reference.

Functions take host numpy arrays laid out exactly like the C-ABI's device
buffers: row-major block vectors with leading dimensions in elements,
complex data as complex128 (interleaved re/im doubles).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(exact rational arithmetic on tiny inputs, integer-exact cases, closed forms,
invariants, the Gram-Schmidt identity); none is "parity unpinned".
"""

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsm_oracle.c")
_SRC_PLAIN = os.path.join(_HERE, "tsm_plain.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OP_T, OP_C = 1, 2
_OPS = {"T": OP_T, "C": OP_C, OP_T: OP_T, OP_C: OP_C}


def build(force=False):
    """Compile the C oracle (plain -O2, no fast-math so rounding is IEEE)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_PLAIN))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off",
                           "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, _SRC_PLAIN, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.oracle_tsmttsm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64,
                                           dp, dp, i64, dp, i64, dp, dp, i64]
            lib.oracle_tsmttsm.restype = ctypes.c_int
            lib.oracle_tsmm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64,
                                        dp, dp, i64, dp, i64, dp, dp, i64]
            lib.oracle_tsmm.restype = ctypes.c_int
            lib.oracle_dot.argtypes = [ctypes.c_int, ctypes.c_int, i64, dp, dp, dp]
            lib.oracle_dot.restype = None
            lib.oracle_tsmttsm_plain.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64,
                                                 dp, dp, i64, dp, i64, dp, dp, i64, ctypes.c_int]
            lib.oracle_tsmttsm_plain.restype = ctypes.c_int
            lib.oracle_tsmm_plain.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64,
                                              dp, dp, i64, dp, i64, dp, dp, i64, ctypes.c_int]
            lib.oracle_tsmm_plain.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _scalar(x, cplx):
    if cplx:
        z = complex(x)
        return np.array([z.real, z.imag], dtype=np.float64)
    return np.array([float(np.real(x))], dtype=np.float64)


def _check(arr, cplx, name):
    want = np.complex128 if cplx else np.float64
    if arr.dtype != want or not arr.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous {np.dtype(want).name} array")


def tsmttsm(op, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc):
    """C = alpha * op(A)^T B + beta * C on host arrays (C updated in place).

    op is "T" (A^T B) or "C" (A^H B; same as "T" for real data).  A holds at
    least K*lda elements, B at least K*ldb, C at least M*ldc."""
    cplx = np.iscomplexobj(A)
    for arr, name in ((A, "A"), (B, "B"), (C, "C")):
        _check(arr, cplx, name)
    if A.size < K * lda or B.size < K * ldb or C.size < (M - 1) * ldc + N:
        raise ValueError("buffer too small")
    al, be = _scalar(alpha, cplx), _scalar(beta, cplx)
    rc = _load().oracle_tsmttsm(_OPS[op], int(cplx), M, N, K, _dptr(al), _dptr(A.view(np.float64)),
                                lda, _dptr(B.view(np.float64)), ldb, _dptr(be),
                                _dptr(C.view(np.float64)), ldc)
    if rc:
        raise ValueError(f"oracle_tsmttsm rejected its arguments ({rc})")
    return C


def tsmttsm_plain(op, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, threads=1):
    """As ``tsmttsm`` but with the plain uncompensated sum of rounded
    products, K cut into ``threads`` contiguous chunks summed in chunk
    order: the CPU baseline that is timed, not a parity reference."""
    cplx = np.iscomplexobj(A)
    for arr, name in ((A, "A"), (B, "B"), (C, "C")):
        _check(arr, cplx, name)
    if A.size < K * lda or B.size < K * ldb or C.size < (M - 1) * ldc + N:
        raise ValueError("buffer too small")
    al, be = _scalar(alpha, cplx), _scalar(beta, cplx)
    rc = _load().oracle_tsmttsm_plain(_OPS[op], int(cplx), M, N, K, _dptr(al), _dptr(A.view(np.float64)),
                                      lda, _dptr(B.view(np.float64)), ldb, _dptr(be),
                                      _dptr(C.view(np.float64)), ldc, int(threads))
    if rc:
        raise ValueError(f"oracle_tsmttsm_plain rejected its arguments ({rc})")
    return C


def gram_plain(A, B, op="T", threads=1):
    """op(A)^T B by the plain threaded loop, for 2-D arrays."""
    K, M = A.shape
    N = B.shape[1]
    C = np.zeros((M, N), dtype=A.dtype)
    return tsmttsm_plain(op, M, N, K, 1.0, np.ascontiguousarray(A), M, np.ascontiguousarray(B), N, 0.0, C, N,
                         threads)


def tsmm_plain(M, N, K, alpha, A, lda, Cm, ldc, beta, B, ldb, threads=1):
    """As ``tsmm`` with plain uncompensated row sums, rows split over
    ``threads`` threads: the timed CPU baseline, not a parity reference."""
    cplx = np.iscomplexobj(A)
    for arr, name in ((A, "A"), (Cm, "C"), (B, "B")):
        _check(arr, cplx, name)
    if A.size < K * lda or B.size < K * ldb or Cm.size < (M - 1) * ldc + N:
        raise ValueError("buffer too small")
    al, be = _scalar(alpha, cplx), _scalar(beta, cplx)
    rc = _load().oracle_tsmm_plain(int(cplx), M, N, K, _dptr(al), _dptr(A.view(np.float64)), lda,
                                   _dptr(Cm.view(np.float64)), ldc, _dptr(be),
                                   _dptr(B.view(np.float64)), ldb, int(threads))
    if rc:
        raise ValueError(f"oracle_tsmm_plain rejected its arguments ({rc})")
    return B


def apply_plain(A, Cm, alpha=1.0, beta=0.0, B0=None, threads=1):
    """alpha * A C + beta * B0 by the plain threaded loop, for 2-D arrays."""
    K, M = A.shape
    N = Cm.shape[1]
    B = np.zeros((K, N), dtype=A.dtype) if B0 is None else np.array(B0, dtype=A.dtype, order="C")
    return tsmm_plain(M, N, K, alpha, np.ascontiguousarray(A), M, np.ascontiguousarray(Cm), N, beta, B, N,
                      threads)


def tsmm(M, N, K, alpha, A, lda, Cm, ldc, beta, B, ldb):
    """B = alpha * A C + beta * B on host arrays (B updated in place)."""
    cplx = np.iscomplexobj(A)
    for arr, name in ((A, "A"), (Cm, "C"), (B, "B")):
        _check(arr, cplx, name)
    if A.size < K * lda or B.size < K * ldb or Cm.size < (M - 1) * ldc + N:
        raise ValueError("buffer too small")
    al, be = _scalar(alpha, cplx), _scalar(beta, cplx)
    rc = _load().oracle_tsmm(int(cplx), M, N, K, _dptr(al), _dptr(A.view(np.float64)), lda,
                             _dptr(Cm.view(np.float64)), ldc, _dptr(be),
                             _dptr(B.view(np.float64)), ldb)
    if rc:
        raise ValueError(f"oracle_tsmm rejected its arguments ({rc})")
    return B


def dot(op, a, b):
    """sum_k op(a_k) * b_k for two contiguous columns (op "C" conjugates a)."""
    cplx = np.iscomplexobj(a)
    a = np.ascontiguousarray(a, dtype=np.complex128 if cplx else np.float64)
    b = np.ascontiguousarray(b, dtype=a.dtype)
    if a.shape != b.shape or a.ndim != 1:
        raise ValueError("dot wants two 1-D columns of equal length")
    out = np.zeros(2, dtype=np.float64)
    _load().oracle_dot(_OPS[op], int(cplx), a.shape[0], _dptr(a.view(np.float64)),
                       _dptr(b.view(np.float64)), _dptr(out))
    return complex(out[0], out[1]) if cplx else float(out[0])


# Convenience forms on 2-D arrays (K x M etc.), returning fresh results.

def gram(A, B, op="T", alpha=1.0, beta=0.0, C0=None):
    """alpha * op(A)^T B + beta * C0 for 2-D arrays A (K x M), B (K x N)."""
    K, M = A.shape
    N = B.shape[1]
    cplx = np.iscomplexobj(A) or np.iscomplexobj(B)
    dt = np.complex128 if cplx else np.float64
    A = np.ascontiguousarray(A, dtype=dt)
    B = np.ascontiguousarray(B, dtype=dt)
    C = np.zeros((M, N), dtype=dt) if C0 is None else np.array(C0, dtype=dt, order="C")
    return tsmttsm(op, M, N, K, alpha, A, M, B, N, beta, C, N)


def apply(A, Cm, alpha=1.0, beta=0.0, B0=None):
    """alpha * A C + beta * B0 for 2-D arrays A (K x M), C (M x N)."""
    K, M = A.shape
    N = Cm.shape[1]
    cplx = np.iscomplexobj(A) or np.iscomplexobj(Cm)
    dt = np.complex128 if cplx else np.float64
    A = np.ascontiguousarray(A, dtype=dt)
    Cm = np.ascontiguousarray(Cm, dtype=dt)
    B = np.zeros((K, N), dtype=dt) if B0 is None else np.array(B0, dtype=dt, order="C")
    return tsmm(M, N, K, alpha, A, M, Cm, N, beta, B, N)


def rel_fro(x, ref):
    """Normwise relative Frobenius error ||x - ref||_F / ||ref||_F (absolute
    norm when ||ref||_F == 0)."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    num = np.linalg.norm((x - ref).ravel())
    den = np.linalg.norm(ref.ravel())
    return num / den if den > 0 else num
