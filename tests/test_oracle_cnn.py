"""Pins of the FP64 CPU reference of the warm-start network (CPU only): without
the BF16 rounding its hand-written backward equals torch autograd, and its loss
equals the mean squared error written out directly."""
import numpy as np
import torch
import torch.nn.functional as F

from oracle import cnn as R
from paper_1903_10088_gb300 import warmstart as ws


def test_manual_backward_equals_autograd():
    rng = np.random.default_rng(0)
    params = ws.init_params(3).astype(np.float64)
    params += 0.05 * rng.normal(size=params.shape)        # non-trivial last layer
    x = rng.uniform(0, 0.1, (2, 9, 11))
    y = rng.uniform(0, 0.1, (2, 9, 11))
    with R.exact():
        loss, g = R.loss_and_grad(params, x, y, 10.0)
        # autograd on the same FP64 network
        p = torch.tensor(params, dtype=torch.float64, requires_grad=True)
        off, h = 0, None
        xs = torch.as_tensor(x)[:, None] * 10.0
        h = xs
        shapes = [(1, 32)] + [(32, 32)] * 6 + [(32, 1)]
        for k, (ci, co) in enumerate(shapes):
            w = p[off:off + 9 * ci * co].reshape(3, 3, ci, co).permute(3, 2, 0, 1)
            off += 9 * ci * co
            b = p[off:off + co]
            off += co
            h = F.conv2d(h, w, b, padding=1)
            if k < 7:
                h = torch.relu(h)
        out = xs + h
        ref_loss = ((out - torch.as_tensor(y)[:, None] * 10.0) ** 2).mean()
        ref_loss.backward()
    assert abs(loss - ref_loss.item()) <= 1e-12 * ref_loss.item()
    assert np.abs(g - p.grad.numpy()).max() <= 1e-10 * np.abs(p.grad.numpy()).max()


def test_parameter_layout_roundtrip():
    params = np.arange(R.CH * 0 + ws.param_count(), dtype=np.float32)
    layers = R.unpack(params * 0 + 1)
    assert len(layers) == 8
    assert layers[0][0].shape == (32, 1, 3, 3) and layers[1][0].shape == (32, 32, 3, 3)
    assert layers[7][0].shape == (1, 32, 3, 3) and layers[7][1].shape == (1,)
    back = R.pack_grad([(w, b) for w, b in layers])
    assert back.shape == (ws.param_count(),)
