"""Learned warm start for the OS-TV loop (binding and training pipeline).

The network (``mvct_cnn_*`` in the C ABI) maps an FBP image to a start image for
``mvct_recon`` / ``mvct_batch``: 8 conv3x3 layers, 32 channels, ReLU, residual
output, BF16 weights and activations with FP32 accumulation, trained with Adam
on (FBP image, converged OS-TV image) pairs that the reconstruction itself
produces from seeded synthetic phantoms. The paper motivates the start image's
role (Sec. 3.3.2 and 4.2: mu^(0) changes the convergence speed); the network
itself is this project's addition.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional

import numpy as np

CH = 32
PARAM_COUNT = 9 * CH + CH + 6 * (9 * CH * CH + CH) + 9 * CH + 1
SCALE = 10.0   # images are multiplied by this inside the network (water ~ 0.7)


def param_count() -> int:
    return PARAM_COUNT


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases; the last layer starts small so that the
    residual network starts close to the identity (out ~ FBP)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.normal(0, np.sqrt(2.0 / 9), 9 * CH), np.zeros(CH)]
    for _ in range(6):
        parts += [rng.normal(0, np.sqrt(2.0 / (9 * CH)), 9 * CH * CH), np.zeros(CH)]
    parts += [rng.normal(0, 1e-3, 9 * CH), np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == PARAM_COUNT
    return p


class CNN:
    """The warm-start network on the current CUDA device (``mvct_cnn_*``)."""

    def __init__(self, batch_max: int, h: int, w: int, params: np.ndarray, scale: float = SCALE):
        from . import mvct

        self._m = mvct
        lib = mvct.lib()
        if lib.mvct_cnn_param_count() != PARAM_COUNT:
            raise RuntimeError("parameter layout of the library does not match the binding")
        p = np.ascontiguousarray(params, dtype=np.float32)
        h_ = ctypes.c_void_p()
        mvct._check(lib.mvct_cnn_create(batch_max, h, w, scale, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        ctypes.byref(h_)))
        self._h, self.h, self.w, self.batch_max = h_, h, w, batch_max

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._m.lib().mvct_cnn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptr(self, t, n, name):
        return self._m._dev_f32(t, n * self.h * self.w, name)

    def params(self) -> np.ndarray:
        out = np.zeros(PARAM_COUNT, dtype=np.float32)
        self._m._check(self._m.lib().mvct_cnn_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def forward(self, x, out=None, stream=None):
        import torch

        n = x.shape[0]
        if out is None:
            out = torch.empty_like(x)
        self._m._check(self._m.lib().mvct_cnn_forward(self._h, self._ptr(x, n, "x"), n, self._ptr(out, n, "out"),
                                                      ctypes.c_void_p(self._m._stream(stream))))
        return out

    def grad(self, x, y, stream=None):
        import torch

        n = x.shape[0]
        g = torch.empty(PARAM_COUNT, device=x.device, dtype=torch.float32)
        loss = ctypes.c_double()
        self._m._check(self._m.lib().mvct_cnn_grad(self._h, self._ptr(x, n, "x"), self._ptr(y, n, "y"), n,
                                                   ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss),
                                                   ctypes.c_void_p(self._m._stream(stream))))
        return loss.value, g

    def train_step(self, x, y, lr: float, stream=None) -> float:
        n = x.shape[0]
        loss = ctypes.c_double()
        self._m._check(self._m.lib().mvct_cnn_train_step(self._h, self._ptr(x, n, "x"), self._ptr(y, n, "y"), n,
                                                         lr, ctypes.byref(loss),
                                                         ctypes.c_void_p(self._m._stream(stream))))
        return loss.value
