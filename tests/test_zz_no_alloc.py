"""The allocation-free TV entry point (mvct_tv_grad_noalloc) agrees with the
plan-based mvct_tv_grad and with the FP64 oracle.

mvct_tv_grad_noalloc exists for callers that may not allocate device memory
(applications whose GPU memory is handed out by their own allocator, or
latency-critical paths where cudaMalloc, which can synchronise the device, is
off limits). It keeps its partial sums in a static device array shared by all
calls, so this test calls it twice in a row, with different images and sizes,
and checks each result against the existing entry point and against the FP64
oracle's TV within the tolerances the operator tests use (gradient 1e-5
relative L2, FP64-reduced value 1e-6), so a fault shared by both CUDA entry
points cannot pass unseen.

This file is collected last so that a run stopping at the first failure has
run every other test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle

from paper_1903_10088_gb300 import phantom as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mvct():
    from paper_1903_10088_gb300 import build, mvct

    build.build()
    mvct.lib()
    return mvct


def rel(a, b):
    a, b = np.ravel(a.astype(np.float64)), np.ravel(b.astype(np.float64))
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_tv_matches_plan_entry_point_twice(mvct):
    lib = mvct.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    eps = 1e-6
    for n, seed in ((300, 1), (97, 2)):
        img = torch.from_numpy(np.random.default_rng(seed).uniform(0, 0.1, (n, n)).astype(np.float32)).cuda()
        with mvct.Plan(ph.Geometry(n=n, n_views=4, n_channels=4), 1) as plan:
            ref_grad, ref_tv = plan.tv_grad(img, eps)
            torch.cuda.synchronize()
        grad = torch.full((n, n), float("nan"), device="cuda")
        tv = torch.full((1,), float("nan"), device="cuda", dtype=torch.float64)
        rc = lib.mvct_tv_grad_noalloc(ctypes.c_void_p(img.data_ptr()), n, eps,
                                      ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(tv.data_ptr()),
                                      stream)
        assert rc == 0, lib.mvct_last_error()
        torch.cuda.synchronize()
        assert rel(grad.cpu().numpy(), ref_grad.cpu().numpy()) < 1e-5
        assert abs(float(tv.cpu()) - float(ref_tv.cpu())) <= 1e-6 * float(ref_tv.cpu())
        o_tv, o_grad = oracle.tv(img.double().cpu().numpy(), eps)
        assert rel(grad.cpu().numpy(), o_grad) < 1e-5
        assert abs(float(tv.cpu()) - o_tv) <= 1e-6 * o_tv


def test_noalloc_rejects_sizes_beyond_the_maximum(mvct):
    lib = mvct.lib()
    dummy = torch.zeros(1, device="cuda")
    rc = lib.mvct_tv_grad_noalloc(ctypes.c_void_p(dummy.data_ptr()), 4097, 1e-6,
                                  ctypes.c_void_p(dummy.data_ptr()), None, None)
    assert rc == -1
    assert b"outside 1..4096" in lib.mvct_last_error()
