"""GB300-native tall & skinny FP64 matrix products (arXiv:1905.03136).

Thin Python layer over ``libtsm.so``: the functions below only turn torch
tensors into the pointers, sizes and leading dimensions of the C ABI
(``include/tsm*.h``) and raise on a non-zero status.  All arithmetic runs in
the library's CUDA kernels; there is no CPU or PyTorch fallback.

Tensors are row-major 2-D views (stride(1) == 1, leading dimension =
stride(0)) of float64 or complex128 device memory.
"""

import ctypes

from . import _lib
from ._lib import (C64, KIND_TSMM, KIND_TSMM_BETA, KIND_TSMTTSM, OP_C, OP_N, OP_T, R64, TsmError, VariantInfo,
                   TuneSample, call, load, raw, scalar)

__all__ = ["tsmttsm", "tsmm", "gs_step", "fill_random", "variants", "variant_shape", "choose", "tune", "time_variant",
           "TsmError", "load", "R64", "C64", "OP_T", "OP_C", "OP_N"]

_OPS = {"T": OP_T, "C": OP_C, "N": OP_N, OP_T: OP_T, OP_C: OP_C, OP_N: OP_N}


def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float64:
        return R64
    if t.dtype == torch.complex128:
        return C64
    raise TypeError("tensors must be float64 or complex128, got %s" % t.dtype)


def _ld(t, name):
    if t.dim() != 2:
        raise ValueError("%s must be 2-D" % name)
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError("%s must be row-major (stride(1) == 1)" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    return max(int(t.stride(0)), int(t.shape[1]))


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def tsmttsm(A, B, C=None, alpha=1.0, beta=0.0, op="T", stream=None, variant=-1, grid=0):
    """C = alpha * op(A)^T B + beta * C  (A: K x M, B: K x N, C: M x N)."""
    torch = _torch()
    dt = _dtype_code(A)
    K, M = A.shape
    N = B.shape[1]
    if B.shape[0] != K or _dtype_code(B) != dt:
        raise ValueError("A and B must have the same row count and dtype")
    if C is None:
        C = torch.zeros((M, N), dtype=A.dtype, device=A.device)
        beta = 0.0
    cplx = dt == C64
    call("tsm_tsmttsm_ex", _OPS[op], dt, M, N, K, scalar(alpha, cplx), ctypes.c_void_p(A.data_ptr()),
         _ld(A, "A"), ctypes.c_void_p(B.data_ptr()), _ld(B, "B"), scalar(beta, cplx),
         ctypes.c_void_p(C.data_ptr()), _ld(C, "C"), int(variant), int(grid), _stream(stream))
    return C


def tsmm(A, Cm, B=None, alpha=1.0, beta=0.0, stream=None, variant=-1, grid=0):
    """B = alpha * A C + beta * B  (A: K x M, C: M x N, B: K x N)."""
    torch = _torch()
    dt = _dtype_code(A)
    K, M = A.shape
    N = Cm.shape[1]
    if Cm.shape[0] != M or _dtype_code(Cm) != dt:
        raise ValueError("C must be M x N with A's dtype")
    if B is None:
        B = torch.empty((K, N), dtype=A.dtype, device=A.device)
        beta = 0.0
    cplx = dt == C64
    call("tsm_tsmm_ex", OP_N, dt, M, N, K, scalar(alpha, cplx), ctypes.c_void_p(A.data_ptr()), _ld(A, "A"),
         ctypes.c_void_p(Cm.data_ptr()), _ld(Cm, "C"), scalar(beta, cplx), ctypes.c_void_p(B.data_ptr()),
         _ld(B, "B"), int(variant), int(grid), _stream(stream))
    return B


GS_MODES = {"auto": 0, "two_products": 1, "fused": 2}


def gs_step(A, B, C=None, stream=None, mode="auto"):
    """One block Gram-Schmidt projection in place: C = A^H B, B -= A C.
    Returns C (M x N, on the device).  mode: "auto", "two_products" or
    "fused" (tsm_gs_step_ex)."""
    torch = _torch()
    dt = _dtype_code(A)
    K, M = A.shape
    N = B.shape[1]
    if B.shape[0] != K or _dtype_code(B) != dt:
        raise ValueError("A and B must have the same row count and dtype")
    if C is None:
        C = torch.empty((M, N), dtype=A.dtype, device=A.device)
    elif C.shape != (M, N) or _dtype_code(C) != dt:
        raise ValueError("C must be M x N with A's dtype")
    call("tsm_gs_step_ex", dt, M, N, K, ctypes.c_void_p(A.data_ptr()), _ld(A, "A"), ctypes.c_void_p(B.data_ptr()),
         _ld(B, "B"), ctypes.c_void_p(C.data_ptr()), _ld(C, "C"), GS_MODES[mode], _stream(stream))
    return C


def gs_status(stream=None):
    """Synchronizes the stream; raises TSM_ERR_TIMEOUT if a fused step on it
    gave up a barrier wait (tsm_gs_status)."""
    call("tsm_gs_status", _stream(stream))


def gs_set_timeout(cycles):
    """Test hook: barrier wait budget of later fused steps (<= 0: default)."""
    call("tsm_gs_set_timeout", int(cycles))


DIST = {"uniform": 0, "loguniform": 1, "smallint": 2, "ones": 3}


def fill_random(t, seed, dist="uniform", row0=0, stream=None):
    """Fills a row-major float64/complex128 device tensor (rows x ld) with the
    seeded synthetic inputs (same values as the host generator ``synth``)."""
    dt = _dtype_code(t)
    rows = t.shape[0] if t.dim() == 2 else 1
    ld = t.stride(0) if t.dim() == 2 else t.numel()
    call("tsm_fill_random", ctypes.c_void_p(t.data_ptr()), dt, rows, ld, int(row0), ctypes.c_uint64(seed),
         DIST[dist], _stream(stream))
    return t


def variants(kind):
    """List of dicts describing the compiled variants of a product."""
    lib = load()
    out = []
    for i in range(lib.tsm_variant_count(kind)):
        info = VariantInfo()
        call("tsm_variant_get", kind, i, ctypes.byref(info))
        d = {f: getattr(info, f) for f, _ in VariantInfo._fields_}
        d["name"] = info.name.decode()
        d["index"] = i
        out.append(d)
    return out


def variant_shape(kind, index, dtype, M, N):
    """Variant `index` described for shape (M, N): runtime-tile variants
    report the tile (TSMTTSM) or threads per row and results per thread
    (TSMM) their launch picks for it."""
    info = VariantInfo()
    call("tsm_variant_shape", kind, index, dtype, M, N, ctypes.byref(info))
    d = {f: getattr(info, f) for f, _ in VariantInfo._fields_}
    d["name"] = info.name.decode()
    d["index"] = index
    return d


def choose(kind, dtype, M, N, K):
    v, g = ctypes.c_int(), ctypes.c_int()
    call("tsm_choose", kind, dtype, M, N, K, ctypes.byref(v), ctypes.byref(g))
    return v.value, g.value


def tune(kind, X, Y, Z, reps=3, stream=None, max_samples=512):
    """Exhaustive search (tsm_tune) on device tensors; returns the samples.
    kind KIND_TSMM_BETA times the TSMM variants with beta = 1 (Z is read)."""
    dt = _dtype_code(X)
    if kind == KIND_TSMTTSM:
        K, M = X.shape
        N = Y.shape[1]
    else:
        K, M = X.shape
        N = Y.shape[1]
    buf = (TuneSample * max_samples)()
    n = ctypes.c_int()
    call("tsm_tune", kind, dt, M, N, K, ctypes.c_void_p(X.data_ptr()), _ld(X, "X"),
         ctypes.c_void_p(Y.data_ptr()), _ld(Y, "Y"), ctypes.c_void_p(Z.data_ptr()), _ld(Z, "Z"), reps, buf,
         max_samples, ctypes.byref(n), _stream(stream))
    return [(buf[i].variant, buf[i].grid, buf[i].ms) for i in range(min(n.value, max_samples))]


def time_variant(kind, X, Y, Z, variant, grid=0, reps=3, stream=None):
    dt = _dtype_code(X)
    K, M = X.shape
    N = Y.shape[1]
    ms = ctypes.c_float()
    call("tsm_time_variant", kind, dt, M, N, K, ctypes.c_void_p(X.data_ptr()), _ld(X, "X"),
         ctypes.c_void_p(Y.data_ptr()), _ld(Y, "Y"), ctypes.c_void_p(Z.data_ptr()), _ld(Z, "Z"),
         int(variant), int(grid), int(reps), ctypes.byref(ms), _stream(stream))
    return ms.value
