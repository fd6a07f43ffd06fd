"""Binding of the cost model's network (include/tsm_mlp.h): a 3-layer tanh
perceptron whose forward, backward and Adam steps run in the library's own
CUDA kernels.  Inputs, targets and outputs are float32 device tensors."""

import ctypes

import numpy as np

from . import _lib

_P = ctypes.c_void_p
_lib.extend_signatures({
    "tsm_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "tsm_mlp_destroy": (None, [_P]),
    "tsm_mlp_param_count": (ctypes.c_int, [_P]),
    "tsm_mlp_set_params": (ctypes.c_int, [_P, _P]),
    "tsm_mlp_get_params": (ctypes.c_int, [_P, _P]),
    "tsm_mlp_get_grads": (ctypes.c_int, [_P, _P]),
    "tsm_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
    "tsm_mlp_backward": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P]),
    "tsm_mlp_adam": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P]),
})


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Mlp:
    """Owns one tsm_mlp (device parameters, gradients, Adam state)."""

    def __init__(self, in_dim, hidden=64, max_batch=65536, seed=0):
        h = ctypes.c_void_p()
        _lib.call("tsm_mlp_create", in_dim, hidden, max_batch, ctypes.c_uint64(seed), ctypes.byref(h))
        self.h = h
        self.in_dim, self.hidden, self.max_batch = in_dim, hidden, max_batch
        self.n_params = _lib.load().tsm_mlp_param_count(h)

    def close(self):
        if self.h:
            _lib.load().tsm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _lib.call("tsm_mlp_get_params", self.h, out.ctypes.data_as(ctypes.c_void_p))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _lib.call("tsm_mlp_set_params", self.h, p.ctypes.data_as(ctypes.c_void_p))

    def grads(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _lib.call("tsm_mlp_get_grads", self.h, out.ctypes.data_as(ctypes.c_void_p))
        return out

    def forward(self, X, stream=None):
        import torch
        X = X.contiguous()
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _lib.call("tsm_mlp_forward", self.h, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                  ctypes.c_void_p(y.data_ptr()), _stream(stream))
        return y

    def backward(self, X, t, stream=None):
        """Loss (device scalar tensor); the gradient stays in the model."""
        import torch
        X = X.contiguous()
        t = t.contiguous()
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _lib.call("tsm_mlp_backward", self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                  X.shape[0], ctypes.c_void_p(loss.data_ptr()), _stream(stream))
        return loss

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _lib.call("tsm_mlp_adam", self.h, ctypes.c_float(lr), ctypes.c_float(beta1), ctypes.c_float(beta2),
                  ctypes.c_float(eps), _stream(stream))

    def fit(self, X, t, epochs=2000, lr=3e-3, stream=None):
        """Full-batch Adam; returns the loss history (host floats)."""
        import torch
        hist = []
        for e in range(epochs):
            loss = self.backward(X, t, stream)
            self.adam(lr, stream=stream)
            if e % 100 == 0 or e == epochs - 1:
                hist.append(float(loss.item()))
        torch.cuda.synchronize()
        return hist
