"""What the learned warm start gains: on held-out seeded phantoms the network's
start image followed by K OS-TV sub-iterations reaches a lower objective than the
FBP start after the same K; every slice reaches the plain form's objective (FBP
start, 500 sub-iterations) within 1e-3 after fewer sub-iterations from the
network's start than from the FBP start; the GPU objective agrees with the FP64
oracle's. A second test trains a network from scratch on pairs the method
generates (small geometry) and checks the same gain."""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest
import torch

from paper_1903_10088_gb300 import warmstart as ws

pytestmark = pytest.mark.gpu

SEEDS = range(ws.HELDOUT_SEED0 + 100, ws.HELDOUT_SEED0 + 108)   # held out, not in the benchmark stack
KS = [25, 50, 100]


@pytest.fixture(scope="module")
def mvct():
    from paper_1903_10088_gb300 import build, mvct

    build.build()
    mvct.lib()
    return mvct


def test_trained_network_gains_over_fbp_start(mvct):
    import oracle_jobs

    pool = cf.ProcessPoolExecutor(4, mp_context=mp.get_context("spawn"))
    cases = list(pool.map(ws.case_for, SEEDS))
    dev = torch.device("cuda", torch.cuda.current_device())
    cnn = ws.CNN(8, 512, 512, ws.load_weights())
    res = ws.evaluate(cnn, cases, KS, dev, width=8, warm_opts={"lambda0": ws.FAST_LAMBDA0}, keep_images=2)
    for r in res:
        # the network's image is far closer to the converged one than FBP is (its
        # targets are the 2000-sub-iteration images, a little past the plain form)
        assert r["rel_plain_cnn_K0"] < 0.5 * r["rel_plain_fbp_K0"]
        for K in [0] + KS:
            assert r[f"psi_cnn_K{K}"] < r[f"psi_fbp_K{K}"], (r["seed"], K)
    # the per-slice bar: the smallest K of the grid at which every slice is within
    # 1e-3 of the plain form, from the network's start and from the FBP start
    k_cnn = ws.sub_iterations_to_bar(cnn, cases, dev, ws.K_GRID, width=8)
    k_fbp = ws.sub_iterations_to_bar(None, cases, dev, ws.K_GRID, width=8)
    cnn.close()
    print(f"\nsub-iterations until every slice is within {ws.BAR:g} of the plain form: network start {k_cnn}, "
          f"FBP start {k_fbp}")
    assert k_cnn is not None and k_fbp is not None and k_cnn < k_fbp
    # the FP64 oracle objective of two seeds' images: same values, same ordering
    jobs = [(r["seed"], key, r["images"][key]) for r in res[:2] for key in ("plain", "cnn_K100", "fbp_K100")]
    vals = list(pool.map(oracle_jobs.full_case_objective, [j[0] for j in jobs], [j[2] for j in jobs]))
    pool.shutdown()
    for (seed, key, _), v in zip(jobs, vals):
        r = next(x for x in res if x["seed"] == seed)
        gpu = r["psi_plain"] if key == "plain" else r[f"psi_{key}"]
        assert abs(gpu - v) <= 1e-6 * abs(v)
    for k in range(2):
        o = dict((key, v) for (seed, key, _), v in zip(jobs[3 * k:3 * k + 3], vals[3 * k:3 * k + 3]))
        assert o["cnn_K100"] < o["fbp_K100"]


def test_training_from_scratch_gains(mvct):
    """128^2, 200 views: 48 pairs (FBP, 100 sub-iterations), 15 epochs of Adam;
    on 8 held-out phantoms the trained start beats the FBP start after 10
    sub-iterations."""
    dev = torch.device("cuda", torch.cuda.current_device())
    X, Y, _ = ws.make_pairs(range(70_000, 70_048), dev, width=48, n_iter=100, workers=4, kind="small")
    cnn = ws.CNN(8, X.shape[1], X.shape[2], ws.init_params(0))
    hist = ws.train(cnn, X, Y, epochs=15, batch=8, lr=1e-3, seed=1)
    assert hist[-1] < 0.5 * hist[0]
    cases = ws.make_cases(range(71_000, 71_008), kind="small", workers=1)
    res = ws.evaluate(cnn, cases, [10], dev, width=8, n_plain=100)
    cnn.close()
    for r in res:
        assert r["psi_cnn_K10"] < r["psi_fbp_K10"], r["seed"]
        assert r["rel_plain_cnn_K0"] < r["rel_plain_fbp_K0"]


def test_warm_pipeline_graph_equals_direct_run(mvct):
    """WarmPipeline (FBP -> network -> batched loop): the CUDA-graph replay gives
    the same images as the direct chain, bit for bit, and they match running the
    three stages by hand."""
    cases = [ws.case_for(s) for s in range(ws.HELDOUT_SEED0 + 110, ws.HELDOUT_SEED0 + 113)]
    dev = torch.device("cuda", torch.cuda.current_device())
    pipe = ws.WarmPipeline(cases[0].geom, cases[0].n_subsets, len(cases), 20, dev)
    pipe.load(torch.stack([torch.from_numpy(c.p) for c in cases]),
              torch.stack([torch.from_numpy(c.w) for c in cases]), [c.beta for c in cases])
    pipe.run()
    torch.cuda.synchronize()
    pipe.check()
    direct = pipe.img.clone()
    fbp = pipe.fbp.clone()
    pipe.capture()
    pipe.img.zero_()
    pipe.run()
    torch.cuda.synchronize()
    pipe.check()
    assert torch.equal(direct, pipe.img)
    assert torch.isfinite(direct).all()
    # by hand: the network's start, then the batch from it
    start = ws.infer(pipe.cnn, fbp)
    pipe.close()
    plans = [mvct.Plan(c.geom, c.n_subsets) for c in cases]
    imgs = [start[k].clone() for k in range(len(cases))]
    with mvct.Batch(plans) as b:
        b.bind([torch.from_numpy(c.p).to(dev) for c in cases], [torch.from_numpy(c.w).to(dev) for c in cases],
               [c.beta for c in cases], imgs, 20, init_from_input=True, lambda0=ws.FAST_LAMBDA0)
        b.run(20)
        b.stats(0)
    for k in range(len(cases)):
        assert torch.equal(imgs[k], direct[k])
    for pl in plans:
        pl.close()
