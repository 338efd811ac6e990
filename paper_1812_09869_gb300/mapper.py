"""Thin ctypes binding of the learned mapper entry points (include/ptsne_mlp.h).

Argument marshalling only: training, gradients and inference run in the
library's CUDA kernels.  Tensors are torch CUDA tensors.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import ptsne

HIDDEN = 256
PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


class MlpParams(C.Structure):
    _fields_ = [
        ("d_in", C.c_int32),
        ("out_dim", C.c_int32),
        ("batch", C.c_int32),
        ("infer_rows", C.c_int64),
        ("lr", C.c_float),
        ("beta1", C.c_float),
        ("beta2", C.c_float),
        ("eps", C.c_float),
        ("weight_decay", C.c_float),
    ]


def shapes(d_in: int, out_dim: int) -> dict:
    return {"W1": (HIDDEN, d_in), "b1": (HIDDEN,), "W2": (HIDDEN, HIDDEN), "b2": (HIDDEN,),
            "W3": (out_dim, HIDDEN), "b3": (out_dim,)}


def n_params(d_in: int, out_dim: int) -> int:
    return sum(int(np.prod(s)) for s in shapes(d_in, out_dim).values())


def pack(W: dict) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([np.asarray(W[k], np.float32).ravel() for k in PARAM_ORDER]))


def unpack(flat, d_in: int, out_dim: int) -> dict:
    flat = np.asarray(flat)
    out, pos = {}, 0
    for k, shp in shapes(d_in, out_dim).items():
        size = int(np.prod(shp))
        out[k] = flat[pos:pos + size].reshape(shp)
        pos += size
    return out


_bound = False


def lib():
    global _bound
    L = ptsne.lib()
    if not _bound:
        vp = C.c_void_p
        L.ptsne_mlp_create.argtypes = [C.POINTER(vp), C.POINTER(MlpParams), vp]
        L.ptsne_mlp_destroy.argtypes = [vp]
        L.ptsne_mlp_destroy.restype = None
        L.ptsne_mlp_last_error.argtypes = [vp]
        L.ptsne_mlp_last_error.restype = C.c_char_p
        L.ptsne_mlp_get_params.argtypes = [vp, vp, vp]
        L.ptsne_mlp_fit_scaler.argtypes = [vp, vp, C.c_int64, vp]
        L.ptsne_mlp_grad.argtypes = [vp, vp, vp, C.c_int64, vp, vp, vp, vp]
        L.ptsne_mlp_train_step.argtypes = [vp, vp, vp, C.c_int64, vp, vp, vp]
        L.ptsne_mlp_train.argtypes = [vp, vp, vp, C.c_int64, vp, C.c_int32, C.POINTER(C.c_double), vp]
        L.ptsne_mlp_infer.argtypes = [vp, vp, C.c_int64, vp, vp]
        L.ptsne_mlp_autotune.argtypes = [vp, vp, vp, C.c_int64, vp, C.c_char_p, C.POINTER(C.c_int32), vp]
        L.ptsne_mlp_warm_start.argtypes = [vp, vp, vp, vp, vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_int32), vp]
        _bound = True
    return L


_ptr = ptsne._ptr
_stream = ptsne._stream


class Mapper:
    """Owns one ptsne_mlp handle (parameters, AdamW state, workspace)."""

    def __init__(self, d_in, init, out_dim=2, batch=4096, infer_rows=1 << 24, lr=1e-3, betas=(0.9, 0.999),
                 eps=1e-8, weight_decay=1e-4):
        self.d_in, self.out_dim, self.batch = int(d_in), int(out_dim), int(batch)
        flat = pack(init) if isinstance(init, dict) else np.ascontiguousarray(np.asarray(init, np.float32))
        if flat.size != n_params(self.d_in, self.out_dim):
            raise ValueError("init has the wrong number of parameters")
        p = MlpParams(self.d_in, self.out_dim, self.batch, int(infer_rows), lr, betas[0], betas[1], eps, weight_decay)
        h = C.c_void_p()
        rc = lib().ptsne_mlp_create(C.byref(h), C.byref(p), flat.ctypes.data_as(C.c_void_p))
        if rc != ptsne.OK:
            raise ptsne.PtsneError(rc, lib().ptsne_mlp_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().ptsne_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc != ptsne.OK:
            raise ptsne.PtsneError(rc, lib().ptsne_mlp_last_error(self.h).decode())
        return rc

    def params(self, stream=None) -> dict:
        flat = np.zeros(n_params(self.d_in, self.out_dim), np.float32)
        self._check(lib().ptsne_mlp_get_params(self.h, flat.ctypes.data_as(C.c_void_p), _stream(stream)))
        return unpack(flat, self.d_in, self.out_dim)

    def fit_scaler(self, T, stream=None):
        return self._check(lib().ptsne_mlp_fit_scaler(self.h, _ptr(T), int(T.shape[0]), _stream(stream)))

    def grad(self, X, T, rows, grad_out=None, loss_out=None, stream=None):
        return self._check(lib().ptsne_mlp_grad(self.h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(rows),
                                                _ptr(grad_out), _ptr(loss_out), _stream(stream)))

    def train_step(self, X, T, rows, loss_out=None, stream=None):
        return self._check(lib().ptsne_mlp_train_step(self.h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(rows),
                                                      _ptr(loss_out), _stream(stream)))

    def train(self, X, T, orders, epochs, stream=None) -> np.ndarray:
        loss = np.zeros(max(int(epochs), 1))
        self._check(lib().ptsne_mlp_train(self.h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(orders), int(epochs),
                                          loss.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))
        return loss[:int(epochs)]

    def autotune(self, X, T, rows, cache_path=None, stream=None) -> int:
        """Pick the split-K of the weight-gradient GEMMs by timing; returns it."""
        sp = C.c_int32(0)
        cp = None if cache_path is None else os.fsencode(cache_path)
        self._check(lib().ptsne_mlp_autotune(self.h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(rows), cp,
                                             C.byref(sp), _stream(stream)))
        return int(sp.value)

    def infer(self, X, Y_out, stream=None):
        return self._check(lib().ptsne_mlp_infer(self.h, _ptr(X), int(X.shape[0]), _ptr(Y_out), _stream(stream)))

    def warm_start(self, ctx, X, perm, Y_random, Y_out, stream=None):
        """ptsne_mlp_warm_start: the mapper's placement of X, one ptSNE epoch
        from it and one from Y_random on partition perm (context ctx), keeping
        the better map in Y_out.  Returns (used_mapper, warm KL, cold KL)."""
        kl = (C.c_double * 2)()
        used = C.c_int32(-1)
        self._check(lib().ptsne_mlp_warm_start(self.h, ctx.h, _ptr(X), _ptr(perm), _ptr(Y_random), _ptr(Y_out), kl,
                                               C.byref(used), _stream(stream)))
        return bool(used.value), float(kl[0]), float(kl[1])
