"""Bindings of the machine-peak probes (include/tsm_probe.h)."""

import ctypes

from . import _lib

_lib.extend_signatures({
    "tsm_probe_fp64": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_void_p]),
    "tsm_probe_bandwidth": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_void_p]),
})


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def fp64_peak(mode=0, iters=20000, stream=None):
    """Measured FP64 GFLOP/s: mode 0 DFMA register tile, mode 1 FP64 MMA,
    mode 2 the constant-operand DFMA chain of the first probe."""
    out = ctypes.c_double()
    _lib.call("tsm_probe_fp64", mode, iters, ctypes.byref(out), _stream(stream))
    return out.value


def bandwidth(buf, mode=0, ilp=16, blocks=0, threads=0, stream=None):
    """Measured GB/s over a device tensor (mode 0 read-only, 1 scale);
    blocks = CTAs in total (0: 8 per SM), threads per CTA (0: 256)."""
    out = ctypes.c_double()
    nbytes = buf.numel() * buf.element_size()
    nbytes -= nbytes % 16
    _lib.call("tsm_probe_bandwidth", ctypes.c_void_p(buf.data_ptr()), nbytes, mode, ilp, blocks, threads,
              ctypes.byref(out), _stream(stream))
    return out.value
