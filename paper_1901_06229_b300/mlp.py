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
