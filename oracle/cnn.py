"""FP64 CPU reference of the warm-start network (TEST INFRASTRUCTURE ONLY).

Plain PyTorch CPU ops in float64. The GPU stores activations and gradients in
BF16 and uses BF16-rounded parameters; this reference rounds at exactly the
same points (the rounding is part of the definition of the BF16 network), so
the comparison isolates the kernels' arithmetic. Layer l: y = conv2d(x, W) + b,
zero padding 1, ReLU after layers 1-7; out = s x + f(s x), returned / s.
Parameter layout: see include/mvct.h (W[tap][in][out], tap = 3 ky + kx).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F
from torch.nn.grad import conv2d_input, conv2d_weight

CH = 32


_ROUND = True


def bf16(t):
    return t.to(torch.bfloat16).to(torch.float64) if _ROUND else t


def f32(t):
    return t.to(torch.float32).to(torch.float64) if _ROUND else t


class exact:
    """Context manager: no BF16/FP32 rounding (plain FP64 network), for pinning the
    hand-written backward against autograd."""

    def __enter__(self):
        global _ROUND
        self.prev, _ROUND = _ROUND, False

    def __exit__(self, *a):
        global _ROUND
        _ROUND = self.prev


def unpack(params):
    """FP64 tensors (W as [out][in][3][3], b), BF16-rounded like the GPU's copies."""
    dt = np.float32 if _ROUND else np.float64
    p = bf16(torch.as_tensor(np.asarray(params, dtype=dt)).to(torch.float64))
    layers = []
    off = 0
    shapes = [(1, CH)] + [(CH, CH)] * 6 + [(CH, 1)]
    for cin, cout in shapes:
        w = p[off:off + 9 * cin * cout].reshape(3, 3, cin, cout).permute(3, 2, 0, 1).contiguous()
        off += 9 * cin * cout
        b = p[off:off + cout]
        off += cout
        layers.append((w, b))
    assert off == len(p)
    return layers


def pack_grad(gs):
    """[(dW [out][in][3][3], db)] -> flat FP64 vector in the parameter layout."""
    out = []
    for dw, db in gs:
        out.append(dw.permute(2, 3, 1, 0).reshape(-1))
        out.append(db.reshape(-1))
    return torch.cat(out).numpy()


def forward(params, x, scale):
    """x: [N][H][W] float32 -> (output [N][H][W], activations)."""
    layers = unpack(params)
    dt = np.float32 if _ROUND else np.float64
    xs = f32(torch.as_tensor(np.asarray(x, dtype=dt)) * dt(scale)).to(torch.float64)[:, None]
    acts = [xs]
    h = xs
    for l, (w, b) in enumerate(layers[:-1]):
        h = bf16(torch.relu(F.conv2d(h, w, b, padding=1)))
        acts.append(h)
    w8, b8 = layers[-1]
    out = xs + F.conv2d(h, w8, b8, padding=1)
    return (out[:, 0] / scale).numpy(), acts, out


def loss_and_grad(params, x, y, scale):
    """Mean squared error in the scaled domain and its parameter gradient."""
    layers = unpack(params)
    _, acts, out = forward(params, x, scale)
    dt = np.float32 if _ROUND else np.float64
    ys = f32(torch.as_tensor(np.asarray(y, dtype=dt)) * dt(scale)).to(torch.float64)[:, None]
    r = out - ys
    count = r.numel()
    loss = float((r * r).sum() / count)
    dout = f32(2.0 * r / count)
    grads = [None] * len(layers)
    w8, _ = layers[-1]
    a7 = acts[-1]
    grads[-1] = (conv2d_weight(a7, w8.shape, dout, padding=1), dout.sum(dim=(0, 2, 3)))
    d = bf16(conv2d_input(a7.shape, w8, dout, padding=1) * (a7 > 0))
    for l in range(len(layers) - 2, 0, -1):       # the six 32 -> 32 layers
        w, _ = layers[l]
        a_in = acts[l]
        grads[l] = (conv2d_weight(a_in, w.shape, d, padding=1), d.sum(dim=(0, 2, 3)))
        d = bf16(conv2d_input(a_in.shape, w, d, padding=1) * (a_in > 0))
    w1, _ = layers[0]
    grads[0] = (conv2d_weight(acts[0], w1.shape, d, padding=1), d.sum(dim=(0, 2, 3)))
    return loss, pack_grad(grads)
