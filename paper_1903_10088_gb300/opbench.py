"""Per-operator timing of the C ABI on one GPU (CUDA events, warm caches).

    python -m paper_1903_10088_gb300.opbench [--n 512 --views 800 --channels 738 --subsets 20]
                                             [--ops forward,back,tv,objective,fbp,cnn] [--reps 20]
                                             [--cnn-batch 16]

Times mvct_forward / mvct_back on one subset (the per-sub-iteration work of the
reconstruction loop) and on all views, mvct_tv_grad, mvct_objective, mvct_fbp,
and the warm-start network (forward, and one Adam training step, on a batch of
--cnn-batch n x n images), on seeded random inputs, and prints one JSON object.
Also the driver for kernel-level profiler captures of the individual operators.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import mvct
from . import phantom as ph


def timed(fn, reps: int) -> float:
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--views", type=int, default=800)
    ap.add_argument("--channels", type=int, default=738)
    ap.add_argument("--subsets", type=int, default=20)
    ap.add_argument("--ops", default="forward,back,tv,objective,fbp,cnn")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--cnn-batch", type=int, default=16)
    args = ap.parse_args(argv)
    g = ph.Geometry(n=args.n, n_views=args.views, n_channels=args.channels)
    rng = np.random.default_rng(0)
    img = torch.from_numpy(rng.uniform(0, 0.1, (g.n, g.n)).astype(np.float32)).cuda()
    sino = torch.from_numpy(rng.uniform(0, 1, (g.n_views, g.n_channels)).astype(np.float32)).cuda()
    w = torch.from_numpy(rng.uniform(0.1, 1, (g.n_views, g.n_channels)).astype(np.float32)).cuda()
    Vs = g.n_views // args.subsets
    sub = sino[:Vs].contiguous()
    out = {"geometry": dict(n=g.n, views=g.n_views, channels=g.n_channels, subsets=args.subsets), "ms": {}}
    ops = args.ops.split(",")
    with mvct.Plan(g, args.subsets) as plan:
        q_sub = torch.empty((Vs, g.n_channels), device="cuda")
        q_all = torch.empty((g.n_views, g.n_channels), device="cuda")
        b = torch.empty((g.n, g.n), device="cuda")
        if "forward" in ops:
            out["ms"]["forward_subset"] = timed(lambda: plan.forward(img, 0, out=q_sub), args.reps)
            out["ms"]["forward_all"] = timed(lambda: plan.forward(img, -1, out=q_all), args.reps)
        if "back" in ops:
            out["ms"]["back_subset"] = timed(lambda: plan.back(sub, 0, out=b), args.reps)
            out["ms"]["back_all"] = timed(lambda: plan.back(sino, -1, out=b), args.reps)
        if "tv" in ops:
            out["ms"]["tv_grad"] = timed(lambda: plan.tv_grad(img, 1e-6), args.reps)
        if "objective" in ops:
            out["ms"]["objective"] = timed(lambda: plan.objective(img, sino, w, 1e-3, 1e-6), args.reps)
        if "fbp" in ops:
            out["ms"]["fbp"] = timed(lambda: plan.fbp(sino, out=b), args.reps)
    if "cnn" in ops:
        from . import warmstart as ws

        N = args.cnn_batch
        x = torch.from_numpy(rng.uniform(0, 0.1, (N, g.n, g.n)).astype(np.float32)).cuda()
        y = 0.9 * x
        xo = torch.empty_like(x)
        net = ws.CNN(N, g.n, g.n, ws.init_params(0))
        out["ms"]["cnn_forward"] = timed(lambda: net.forward(x, out=xo), args.reps)
        out["ms"]["cnn_train_step"] = timed(lambda: net.train_step(x, y, 1e-5), args.reps)
        net.close()
        flops = 2.0 * N * g.n * g.n * (6 * 9 * 32 * 32 + 2 * 9 * 32)
        out["cnn_batch"] = N
        out["cnn_forward_tflops"] = flops / out["ms"]["cnn_forward"] / 1e9
        out["cnn_train_tflops"] = 3 * flops / out["ms"]["cnn_train_step"] / 1e9
    print(json.dumps(out))


if __name__ == "__main__":
    main()
