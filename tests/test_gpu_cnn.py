"""The warm-start network's GPU kernels (BF16 tensor-core convolutions, FP32
accumulation) against the FP64 CPU reference that rounds at the same points:
forward output, loss, and the full parameter gradient (small ragged images, a
row width that leaves a partial 128-pixel tile, and a full-size 2 x 512^2
batch, so the weight-gradient reduction runs over whole images); determinism;
and that Adam steps lower the loss."""
import numpy as np
import pytest
import torch

from oracle import cnn as R
from paper_1903_10088_gb300 import warmstart as ws

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.ravel(np.asarray(a, dtype=np.float64)), np.ravel(np.asarray(b, dtype=np.float64))
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def mvct():
    from paper_1903_10088_gb300 import build, mvct

    build.build()
    mvct.lib()
    return mvct


def params_for_test(seed):
    rng = np.random.default_rng(seed)
    p = ws.init_params(seed)
    # give the last layer and the biases real weight so every layer matters
    p[-(9 * 32 + 1):] = rng.normal(0, 0.05, 9 * 32 + 1)
    return p.astype(np.float32)


def data(shape, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 0.1, shape).astype(np.float32)
    y = (x + rng.normal(0, 0.01, shape)).astype(np.float32)
    return x, y


@pytest.mark.parametrize("shape", [(2, 24, 32), (1, 19, 37), (3, 8, 16), (2, 512, 512), (1, 130, 257)])
def test_forward_matches_reference(mvct, shape):
    p = params_for_test(1)
    x, _ = data(shape, 2)
    net = ws.CNN(shape[0], shape[1], shape[2], p)
    out = net.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref, _, _ = R.forward(p, x, ws.SCALE)
    assert rel(out.cpu().numpy(), ref) < 1e-3
    # the residual part alone (output minus input) to the same relative accuracy
    assert rel(out.cpu().numpy() - x, ref - x) < 5e-3
    net.close()


@pytest.mark.parametrize("shape", [(2, 24, 32), (1, 19, 37), (2, 512, 512)])
def test_gradient_matches_reference(mvct, shape):
    p = params_for_test(3)
    x, y = data(shape, 4)
    net = ws.CNN(shape[0], shape[1], shape[2], p)
    loss, g = net.grad(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    g = g.cpu().numpy()
    ref_loss, ref_g = R.loss_and_grad(p, x, y, ws.SCALE)
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss
    assert rel(g, ref_g) < 1e-2
    # layer by layer (weights of the first, a middle and the last layer)
    sl = [(0, 288), (320 + 2 * 9248, 320 + 2 * 9248 + 9216), (ws.PARAM_COUNT - 289, ws.PARAM_COUNT - 1)]
    for a, b in sl:
        assert rel(g[a:b], ref_g[a:b]) < 2e-2
    net.close()


def test_gradient_is_deterministic(mvct):
    p = params_for_test(5)
    x, y = data((2, 24, 32), 6)
    net = ws.CNN(2, 24, 32, p)
    xs, ys = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    l1, g1 = net.grad(xs, ys)
    l2, g2 = net.grad(xs, ys)
    assert l1 == l2 and torch.equal(g1, g2)
    net.close()


def test_adam_steps_lower_the_loss(mvct):
    p = ws.init_params(7)
    x, _ = data((4, 32, 32), 8)
    y = (0.8 * x + 0.01).astype(np.float32)    # a map the network can represent
    net = ws.CNN(4, 32, 32, p)
    xs, ys = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    losses = [net.train_step(xs, ys, 1e-3) for _ in range(30)]
    assert losses[-1] < 0.7 * losses[0]
    net.close()


def test_convolution_wait_timeout_is_reported(mvct):
    """Failure path of the tensor-core convolutions without a GPU fault: with the
    stall knob their copy warps issue nothing, every block's first pipeline wait
    runs out after the 50 ms limit, the launch finishes, and the host reads
    MVCT_ETIMEOUT (forward: from the status call; training: from the step). The
    context stays usable: with the knob off the next forward matches a network
    that never stalled, bit for bit."""
    n, h, w = 2, 40, 150
    x = torch.from_numpy(data((n, h, w), 7)[0]).cuda()
    p = params_for_test(3)
    ref_net = ws.CNN(n, h, w, p)
    ref = ref_net.forward(x)
    ref_net.status()
    net = ws.CNN(n, h, w, p)
    try:
        net.set_wait(50.0, debug_stall=True)
        net.forward(x)
        with pytest.raises(mvct.MvctError) as ei:
            net.status()
        assert ei.value.code == -5
        with pytest.raises(mvct.MvctError) as ei:
            net.train_step(x, 0.9 * x, 1e-5)
        assert ei.value.code == -5
        net.set_wait(1000.0, debug_stall=False)
        out = net.forward(x)
        net.status()
        assert torch.equal(out, ref)
        with pytest.raises(mvct.MvctError):
            net.set_wait(0.0)
    finally:
        net.close()
        ref_net.close()
