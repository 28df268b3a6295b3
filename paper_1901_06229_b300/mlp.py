"""Python binding of the learned-proposer ABI (include/geodock_mlp.h): marshalling only.

Device tensors come from PyTorch (memory and streams); every computation runs in
libgeodock.so's kernels.
"""
from __future__ import annotations

import ctypes as C

from . import geodock as _gd

_ready = False


def _lib():
    global _ready
    L = _gd.load()
    if not _ready:
        vp, i, f = C.c_void_p, C.c_int, C.c_float
        L.gd_mlp_gemm.argtypes = [vp, i, i, vp, i, i, vp, vp, i, i, i, i, vp, i, vp, f, vp, vp, vp]
        L.gd_mlp_gemm.restype = C.c_int
        _ready = True
    return L


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def gemm(A, B, M, N, K, transA=False, transB=False, C_out=None, Cb_out=None, ldc=None, bias=None, relu=False,
         dotw=None, dot_bias=0.0, dot_out=None, err=None):
    """gd_mlp_gemm on torch CUDA tensors: D = A B^T (BF16 in, FP32 accumulate) + epilogue."""
    lda = A.shape[1]
    ldb = B.shape[1]
    if ldc is None:
        ldc = (C_out if C_out is not None else Cb_out).shape[1] if (C_out is not None or Cb_out is not None) else N
    st = _lib().gd_mlp_gemm(_p(A), lda, int(transA), _p(B), ldb, int(transB), _p(C_out), _p(Cb_out), ldc, M, N, K,
                            _p(bias), int(relu), _p(dotw), float(dot_bias), _p(dot_out), _p(err), _stream())
    if st:
        raise _gd.GeoDockError(st, "gd_mlp_gemm rejected its arguments")


def _lib2():
    L = _lib()
    if not hasattr(L, "_model_ready"):
        vp, i, f = C.c_void_p, C.c_int, C.c_float
        L.gd_mlp_param_count.restype = C.c_int
        L.gd_mlp_create.argtypes = [i, C.c_uint64, i, C.POINTER(vp)]
        L.gd_mlp_destroy.argtypes = [vp]
        L.gd_mlp_set_params.argtypes = [vp, vp]
        L.gd_mlp_get_params.argtypes = [vp, vp]
        L.gd_mlp_predict.argtypes = [vp, vp, C.c_longlong, vp, vp]
        L.gd_mlp_gradients.argtypes = [vp, vp, vp, vp, i, vp, vp, vp]
        L.gd_mlp_train_step.argtypes = [vp, vp, vp, vp, i, f, vp, vp]
        L.gd_mlp_error.argtypes = [vp, C.POINTER(C.c_int)]
        L.gd_mlp_test_hold.argtypes = [vp, i]
        for n in ("gd_mlp_create", "gd_mlp_destroy", "gd_mlp_set_params", "gd_mlp_get_params", "gd_mlp_predict",
                  "gd_mlp_gradients", "gd_mlp_train_step", "gd_mlp_error", "gd_mlp_test_hold"):
            getattr(L, n).restype = C.c_int
        L._model_ready = True
    return L


def _check(st, what):
    if st:
        raise _gd.GeoDockError(st, what)


class MLP:
    """gd_mlp: the proposer network on one device."""

    def __init__(self, device=0, seed=1, max_batch=4096):
        L = _lib2()
        self.h = C.c_void_p()
        _check(L.gd_mlp_create(int(device), C.c_uint64(seed), int(max_batch), C.byref(self.h)), "gd_mlp_create")
        self.nparam = L.gd_mlp_param_count()

    def close(self):
        if self.h:
            _lib2().gd_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        import numpy as np
        out = np.zeros(self.nparam, np.float32)
        _check(_lib2().gd_mlp_get_params(self.h, C.c_void_p(out.ctypes.data)), "gd_mlp_get_params")
        return out

    def set_params(self, P):
        import numpy as np
        P = np.ascontiguousarray(P, np.float32)
        _check(_lib2().gd_mlp_set_params(self.h, C.c_void_p(P.ctypes.data)), "gd_mlp_set_params")

    def predict(self, X, y):
        """y[M] (float32 CUDA tensor) = network(X [M, 48] bfloat16 CUDA tensor)."""
        _check(_lib2().gd_mlp_predict(self.h, _p(X), X.shape[0], _p(y), _stream()), "gd_mlp_predict")

    def gradients(self, X, t, grad, loss, idx=None, B=None):
        B = B if B is not None else X.shape[0]
        _check(_lib2().gd_mlp_gradients(self.h, _p(X), _p(t), _p(idx), int(B), _p(grad), _p(loss), _stream()),
               "gd_mlp_gradients")

    def train_step(self, X, t, lr, loss=None, idx=None, B=None):
        B = B if B is not None else X.shape[0]
        _check(_lib2().gd_mlp_train_step(self.h, _p(X), _p(t), _p(idx), int(B), float(lr), _p(loss), _stream()),
               "gd_mlp_train_step")

    def error(self):
        e = C.c_int()
        _check(_lib2().gd_mlp_error(self.h, C.byref(e)), "gd_mlp_error")
        return e.value

    def test_hold(self, on):
        """Test only: the next tensor-core launch withholds its first MMA commit, so its
        bounded wait runs out (on=True); on=False clears the hold and the error flag."""
        _check(_lib2().gd_mlp_test_hold(self.h, int(bool(on))), "gd_mlp_test_hold")
