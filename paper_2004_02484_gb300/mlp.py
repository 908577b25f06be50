"""Thin ctypes binding of ``include/nmpc_mlp.h`` (argument marshalling only).

Device arrays are torch CUDA tensors (float32, or bfloat16 for GEMM
operands); every computation runs in the CUDA library.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from .nmpc import LIB, _stream

NMPC_MLP_OK = 0
NMPC_MLP_ERR_BAD_ARG = -1
NMPC_MLP_ERR_CUDA = -2

EXPORTED = ["nmpc_gemm_bf16", "nmpc_gemm_set_path", "nmpc_gemm_error", "nmpc_cast_f32_bf16", "nmpc_cast_f32_f64", "nmpc_cast_f64_f32",
            "nmpc_transpose_bf16", "nmpc_pool_avg",
            "nmpc_mlp_create", "nmpc_mlp_num_params",
            "nmpc_mlp_set_params", "nmpc_mlp_get_params", "nmpc_mlp_forward",
            "nmpc_mlp_backward", "nmpc_mlp_get_grads", "nmpc_mlp_set_grads", "nmpc_mlp_adam_step",
            "nmpc_mlp_train_step", "nmpc_mlp_launch_count", "nmpc_mlp_destroy"]

_P, _I, _F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
_SIG = {
    "nmpc_gemm_bf16": (_I, [_P, _P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _P]),
    "nmpc_gemm_set_path": (_I, [_I]),
    "nmpc_gemm_error": (_I, [_I]),
    "nmpc_cast_f32_bf16": (_I, [_P, _P, ctypes.c_int64, _P]),
    "nmpc_cast_f32_f64": (_I, [_P, _P, ctypes.c_int64, _P]),
    "nmpc_transpose_bf16": (_I, [_P, _P, _I, _I, _P]),
    "nmpc_cast_f64_f32": (_I, [_P, _P, ctypes.c_int64, _P]),
    "nmpc_pool_avg": (_I, [_P, _P, _I, _I, _I, _I, ctypes.c_int64, _P]),
    "nmpc_mlp_create": (_I, [_I, ctypes.POINTER(_I), _I, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "nmpc_mlp_num_params": (ctypes.c_int64, [_P]),
    "nmpc_mlp_set_params": (_I, [_P, _P]),
    "nmpc_mlp_get_params": (_I, [_P, _P]),
    "nmpc_mlp_forward": (_I, [_P, _P, _I, _P, _P]),
    "nmpc_mlp_backward": (_I, [_P, _P, _P, _I, ctypes.POINTER(_F), _P]),
    "nmpc_mlp_get_grads": (_I, [_P, _P]),
    "nmpc_mlp_set_grads": (_I, [_P, _P]),
    "nmpc_mlp_adam_step": (_I, [_P, _F, _P]),
    "nmpc_mlp_train_step": (_I, [_P, _P, _P, _I, _F, ctypes.POINTER(_F), _P]),
    "nmpc_mlp_launch_count": (ctypes.c_int64, [_P]),
    "nmpc_mlp_destroy": (None, [_P]),
}
for _name, (_res, _args) in _SIG.items():
    _fn = getattr(LIB, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def _check(rc: int, where: str):
    if rc != NMPC_MLP_OK:
        raise RuntimeError(f"{where} failed ({rc})")


def _dptr(t, dtype_name):
    import torch
    want = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype_name]
    if not (t.is_cuda and t.dtype == want and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA {dtype_name} tensor")
    return t.data_ptr()


def nmpc_gemm_bf16(A, B, C=None, Cb=None, bias=None, gelu=False, stream=None):
    """C = A @ B^T (+ bias) (GELU): A [M, K] bf16, B [N, K] bf16 -> C [M, N]."""
    M, K = A.shape
    N = B.shape[0]
    ldc = (C if C is not None else Cb).shape[1]
    rc = LIB.nmpc_gemm_bf16(_dptr(A, "bf16"), _dptr(B, "bf16"),
                            None if bias is None else _dptr(bias, "f32"),
                            None if C is None else _dptr(C, "f32"),
                            None if Cb is None else _dptr(Cb, "bf16"),
                            M, N, K, A.stride(0), B.stride(0), ldc, int(gelu), _stream(stream))
    _check(rc, "nmpc_gemm_bf16")


def nmpc_gemm_set_path(path: int) -> None:
    """0: tcgen05 tensor-core GEMM where the operands allow it (default);
    1: the mma.sync GEMM everywhere (comparisons)."""
    _check(LIB.nmpc_gemm_set_path(int(path)), "nmpc_gemm_set_path")


def nmpc_gemm_error(clear: bool = True) -> int:
    """1 if a tensor-core GEMM gave up on a bounded wait since the last clear."""
    rc = LIB.nmpc_gemm_error(1 if clear else 0)
    if rc < 0:
        raise RuntimeError(f"nmpc_gemm_error failed ({rc})")
    return rc


def nmpc_cast_f32_bf16(x, out, stream=None):
    _check(LIB.nmpc_cast_f32_bf16(_dptr(x, "f32"), _dptr(out, "bf16"), x.numel(), _stream(stream)),
           "nmpc_cast_f32_bf16")


def nmpc_transpose_bf16(x, out, stream=None):
    rows, cols = x.shape
    _check(LIB.nmpc_transpose_bf16(_dptr(x, "bf16"), _dptr(out, "bf16"), rows, cols,
                                   _stream(stream)), "nmpc_transpose_bf16")


def nmpc_cast_f32_f64(x, out, stream=None):
    import torch
    assert x.dtype == torch.float32 and out.dtype == torch.float64 and x.is_cuda and out.is_cuda
    _check(LIB.nmpc_cast_f32_f64(x.data_ptr(), out.data_ptr(), x.numel(), _stream(stream)),
           "nmpc_cast_f32_f64")


def nmpc_pool_avg(src, out, n_img: int, mx: int, my: int, factor: int, dst_stride: int = 0,
                  stream=None):
    """float64 fields [n_img, my, mx] -> float32 block means [n_img, my/f, mx/f]
    (image i's at out + i dst_stride; 0 = packed)."""
    import torch
    assert src.dtype == torch.float64 and out.dtype == torch.float32 and src.is_cuda and out.is_cuda
    per = (mx // factor) * (my // factor)
    stride = dst_stride or per
    assert src.numel() >= n_img * mx * my
    room = out.untyped_storage().nbytes() // 4 - out.storage_offset()
    assert n_img == 0 or room >= (n_img - 1) * stride + per
    _check(LIB.nmpc_pool_avg(src.data_ptr(), out.data_ptr(), n_img, mx, my, factor, dst_stride,
                             _stream(stream)), "nmpc_pool_avg")


def nmpc_cast_f64_f32(x, out, stream=None):
    import torch
    assert x.dtype == torch.float64 and out.dtype == torch.float32 and x.is_cuda and out.is_cuda
    _check(LIB.nmpc_cast_f64_f32(x.data_ptr(), out.data_ptr(), x.numel(), _stream(stream)),
           "nmpc_cast_f64_f32")


class MLP:
    """Handle over nmpc_mlp_*: widths [in, h1, ..., out]."""

    def __init__(self, widths: Sequence[int], max_batch: int, seed: int = 0):
        self.widths = list(widths)
        arr = (ctypes.c_int * len(widths))(*widths)
        h = ctypes.c_void_p()
        _check(LIB.nmpc_mlp_create(len(widths) - 1, arr, max_batch, seed, ctypes.byref(h)),
               "nmpc_mlp_create")
        self.h = h
        self.max_batch = max_batch
        self.n_params = int(LIB.nmpc_mlp_num_params(h))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(LIB.nmpc_mlp_get_params(self.h, out.ctypes.data), "nmpc_mlp_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _check(LIB.nmpc_mlp_set_params(self.h, p.ctypes.data), "nmpc_mlp_set_params")

    def get_grads(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(LIB.nmpc_mlp_get_grads(self.h, out.ctypes.data), "nmpc_mlp_get_grads")
        return out

    def set_grads(self, g: np.ndarray):
        g = np.ascontiguousarray(g, dtype=np.float32)
        assert g.size == self.n_params
        _check(LIB.nmpc_mlp_set_grads(self.h, g.ctypes.data), "nmpc_mlp_set_grads")

    def forward(self, x, y, stream=None):
        _check(LIB.nmpc_mlp_forward(self.h, _dptr(x, "f32"), x.shape[0], _dptr(y, "f32"),
                                    _stream(stream)), "nmpc_mlp_forward")

    def backward(self, x, t, stream=None) -> float:
        loss = ctypes.c_float()
        _check(LIB.nmpc_mlp_backward(self.h, _dptr(x, "f32"), _dptr(t, "f32"), x.shape[0],
                                     ctypes.byref(loss), _stream(stream)), "nmpc_mlp_backward")
        return float(loss.value)

    def adam_step(self, lr: float, stream=None):
        _check(LIB.nmpc_mlp_adam_step(self.h, lr, _stream(stream)), "nmpc_mlp_adam_step")

    def train_step(self, x, t, lr: float, want_loss: bool = True, stream=None):
        loss = ctypes.c_float()
        _check(LIB.nmpc_mlp_train_step(self.h, _dptr(x, "f32"), _dptr(t, "f32"), x.shape[0], lr,
                                       ctypes.byref(loss) if want_loss else None,
                                       _stream(stream)), "nmpc_mlp_train_step")
        return float(loss.value) if want_loss else None

    def launch_count(self) -> int:
        return int(LIB.nmpc_mlp_launch_count(self.h))

    def close(self):
        if self.h:
            LIB.nmpc_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
