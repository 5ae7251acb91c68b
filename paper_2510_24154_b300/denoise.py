"""Thin Python binding of the denoiser ABI (include/archer_denoise.h).

Argument marshalling only: the U-Net's forward, backward and optimiser steps
and the primitive operations run in the library's CUDA kernels; there is no
CPU fallback.  Device buffers come from PyTorch tensors (bf16 tensors are
passed as their raw 16-bit storage).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .binding import MCError, load as _load_lib

EXPORTED = ("dn_config_default", "dn_create", "dn_destroy", "dn_last_error", "dn_param_count", "dn_set_params",
            "dn_get_params", "dn_get_grads", "dn_forward", "dn_train_step", "dn_get_output", "dn_conv2d_forward",
            "dn_conv2d_backward_data", "dn_conv2d_backward_weights", "dn_maxpool2", "dn_maxpool2_backward",
            "dn_upsample2", "dn_upsample2_backward")


class DnConfig(C.Structure):
    _fields_ = [("height", C.c_int), ("width", C.c_int), ("batch", C.c_int), ("levels", C.c_int),
                ("base_channels", C.c_int), ("in_channels", C.c_int), ("seed", C.c_uint64)]


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = _load_lib()
    vp, i, f, sz = C.c_void_p, C.c_int, C.c_float, C.c_size_t
    L.dn_config_default.argtypes = [C.POINTER(DnConfig)]
    L.dn_config_default.restype = None
    L.dn_create.argtypes = [C.POINTER(DnConfig), i, C.POINTER(vp)]
    L.dn_destroy.argtypes = [vp]
    L.dn_last_error.argtypes = [vp]
    L.dn_last_error.restype = C.c_char_p
    L.dn_param_count.argtypes = [vp, C.POINTER(sz)]
    L.dn_set_params.argtypes = [vp, vp, sz]
    L.dn_get_params.argtypes = [vp, vp, sz]
    L.dn_get_grads.argtypes = [vp, vp, sz]
    L.dn_forward.argtypes = [vp, vp, f, vp, f, vp]
    L.dn_train_step.argtypes = [vp, vp, vp, f, f, C.POINTER(C.c_double), vp]
    L.dn_get_output.argtypes = [vp, vp, vp]
    L.dn_conv2d_forward.argtypes = [vp, i, vp, i, i, i, i, vp, vp, i, i, i, vp, i, vp]
    L.dn_conv2d_backward_data.argtypes = [vp, i, i, i, i, i, vp, i, vp, i, vp, vp, i, vp, vp]
    L.dn_conv2d_backward_weights.argtypes = [vp, i, i, vp, i, vp, i, i, i, i, i, vp, vp, vp]
    L.dn_maxpool2.argtypes = [vp, vp, i, i, i, i, vp]
    L.dn_maxpool2_backward.argtypes = [vp, vp, vp, vp, i, i, i, i, vp]
    L.dn_upsample2.argtypes = [vp, vp, i, i, i, i, vp]
    L.dn_upsample2_backward.argtypes = [vp, vp, i, i, i, i, vp]
    for n in EXPORTED:
        if n not in ("dn_config_default", "dn_last_error"):
            getattr(L, n).restype = C.c_int
    _lib = L
    return L


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _s(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check(st, what=""):
    if st != 0:
        raise MCError(st, f"{what} failed with status {st}")


class UNet:
    """The denoiser on one GPU: parameters, activations, gradients, Adam state."""

    def __init__(self, height=768, width=1024, batch=1, levels=4, base_channels=32, seed=1, device=0,
                 in_channels=1):
        self.lib = lib()
        cfg = DnConfig(height=height, width=width, batch=batch, levels=levels, base_channels=base_channels,
                       in_channels=in_channels, seed=seed)
        h = C.c_void_p()
        _check(self.lib.dn_create(C.byref(cfg), device, C.byref(h)), "dn_create")
        self.h = h
        self.shape = (batch, height, width)
        self.in_channels = in_channels
        n = C.c_size_t()
        self._ck(self.lib.dn_param_count(self.h, C.byref(n)))
        self.n_params = n.value

    def _ck(self, st):
        if st != 0:
            raise MCError(st, self.lib.dn_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.dn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        assert a.size == self.n_params
        self._ck(self.lib.dn_set_params(self.h, C.c_void_p(a.ctypes.data), a.size))

    def params(self):
        a = np.empty(self.n_params, dtype=np.float32)
        self._ck(self.lib.dn_get_params(self.h, C.c_void_p(a.ctypes.data), a.size))
        return a

    def grads(self):
        a = np.empty(self.n_params, dtype=np.float32)
        self._ck(self.lib.dn_get_grads(self.h, C.c_void_p(a.ctypes.data), a.size))
        return a

    def forward(self, x, out, in_scale=1.0, out_scale=1.0, stream=None):
        """x: CUDA float32 [batch][H][W] (one input plane) or [batch][in_channels][H][W];
        out: CUDA float32 [batch][H][W]."""
        self._ck(self.lib.dn_forward(self.h, _p(x), float(in_scale), _p(out), float(out_scale), _s(stream)))

    def train_step(self, x, target, lr, in_scale=1.0, stream=None, want_loss=True):
        loss = C.c_double()
        self._ck(self.lib.dn_train_step(self.h, _p(x), _p(target), float(in_scale), float(lr),
                                        C.byref(loss) if want_loss else None, _s(stream)))
        return loss.value if want_loss else None

    def output(self, out, stream=None):
        self._ck(self.lib.dn_get_output(self.h, _p(out), _s(stream)))


# ----------------------------------------------------------- primitives ----

def conv2d_forward(x0, weight, bias, k, co, relu, y, x1=None, stream=None):
    """x0 [N,H,W,c0] bf16 (x1 [N,H,W,c1] optional), weight float32 [co][k][k][c0+c1], y [N,H,W,ys] bf16."""
    N, H, W, c0 = x0.shape
    c1 = x1.shape[3] if x1 is not None else 0
    _check(lib().dn_conv2d_forward(_p(x0), c0, _p(x1), c1, N, H, W, _p(weight), _p(bias), k, co, int(relu), _p(y),
                                   y.shape[3], _s(stream)), "dn_conv2d_forward")


def conv2d_backward_data(dz, co, weight, k, dx0, mask0=None, dx1=None, mask1=None, stream=None):
    N, H, W, zs = dz.shape
    c0 = dx0.shape[3]
    c1 = dx1.shape[3] if dx1 is not None else 0
    _check(lib().dn_conv2d_backward_data(_p(dz), zs, co, N, H, W, _p(weight), k, _p(dx0), c0, _p(mask0), _p(dx1),
                                         c1, _p(mask1), _s(stream)), "dn_conv2d_backward_data")


def conv2d_backward_weights(dz, co, x0, k, dw, db=None, x1=None, stream=None):
    N, H, W, zs = dz.shape
    c0 = x0.shape[3]
    c1 = x1.shape[3] if x1 is not None else 0
    _check(lib().dn_conv2d_backward_weights(_p(dz), zs, co, _p(x0), c0, _p(x1), c1, N, H, W, k, _p(dw), _p(db),
                                            _s(stream)), "dn_conv2d_backward_weights")


def maxpool2(x, y, stream=None):
    N, H, W, c = x.shape
    _check(lib().dn_maxpool2(_p(x), _p(y), N, H, W, c, _s(stream)), "dn_maxpool2")


def maxpool2_backward(x, dy, dx, add=None, stream=None):
    N, H, W, c = x.shape
    _check(lib().dn_maxpool2_backward(_p(x), _p(dy), _p(add), _p(dx), N, H, W, c, _s(stream)),
           "dn_maxpool2_backward")


def upsample2(x, y, stream=None):
    N, h, w, c = x.shape
    _check(lib().dn_upsample2(_p(x), _p(y), N, h, w, c, _s(stream)), "dn_upsample2")


def upsample2_backward(dy, dx, stream=None):
    N, h, w, c = dx.shape
    _check(lib().dn_upsample2_backward(_p(dy), _p(dx), N, h, w, c, _s(stream)), "dn_upsample2_backward")
