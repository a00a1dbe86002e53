"""Batched reconstruction of uneven slices in one persistent launch (mvct_batch_*),
checked slice by slice against the FP64 oracle and against mvct_recon, plus
CUDA-graph capture of the enqueue-only run."""
import numpy as np
import pytest
import torch

import oracle
from paper_1903_10088_gb300 import phantom as ph

pytestmark = pytest.mark.gpu

RTOL_IMG = 1e-4


def rel(a, b):
    a, b = np.ravel(np.asarray(a, dtype=np.float64)), np.ravel(np.asarray(b, dtype=np.float64))
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def mvct():
    from paper_1903_10088_gb300 import build, mvct

    build.build()
    mvct.lib()
    return mvct


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


UNEVEN = [
    (ph.Geometry(n=64, n_views=60, n_channels=70), 6),
    (ph.Geometry(n=48, n_views=40, n_channels=52, view0_rad=0.3), 4),
    (ph.Geometry(n=80, n_views=72, n_channels=90, channel_offset=0.25), 8),
    (ph.Geometry(n=33, n_views=30, n_channels=41), 3),
]


def make_cases(n_iter, seed0=200):
    return [ph.make_case("small", seed0 + k, geom=g, n_subsets=S, n_iter=n_iter, I0=3e3 * (k + 1))
            for k, (g, S) in enumerate(UNEVEN)]


def run_batch(mvct, cases, n_iter):
    plans = [mvct.Plan(c.geom, c.n_subsets) for c in cases]
    p = [cuda(c.p) for c in cases]
    w = [cuda(c.w) for c in cases]
    imgs = [torch.zeros((c.geom.n, c.geom.n), device="cuda") for c in cases]
    with mvct.Batch(plans) as b:
        b.bind(p, w, [c.beta for c in cases], imgs, n_iter)
        b.run(n_iter)
        stats = [b.stats(i, n_iter) for i in range(len(cases))]
    out = [im.double().cpu().numpy() for im in imgs]
    for pl in plans:
        pl.close()
    return out, stats


def test_batch_matches_oracle_per_slice(mvct):
    n_iter = 14
    cases = make_cases(n_iter)
    imgs, stats = run_batch(mvct, cases, n_iter)
    for c, img, st in zip(cases, imgs, stats):
        ref = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, n_iter)
        assert np.array_equal(st.lam, ref["lam"])
        assert np.allclose(st.phi, ref["phi"], rtol=1e-5)
        assert rel(img, ref["image"]) < RTOL_IMG


def test_batch_agrees_with_single_slice_calls(mvct):
    n_iter = 9
    cases = make_cases(n_iter, seed0=300)
    imgs, _ = run_batch(mvct, cases, n_iter)
    for c, img in zip(cases, imgs):
        with mvct.Plan(c.geom, c.n_subsets) as plan:
            single, _ = plan.recon(cuda(c.p), cuda(c.w), c.beta, n_iter)
            single = single.double().cpu().numpy()
        assert rel(img, single) < 1e-5


def test_batch_is_deterministic_and_graph_capturable(mvct):
    n_iter = 8
    cases = make_cases(n_iter, seed0=400)
    plans = [mvct.Plan(c.geom, c.n_subsets) for c in cases]
    p = [cuda(c.p) for c in cases]
    w = [cuda(c.w) for c in cases]
    imgs = [torch.zeros((c.geom.n, c.geom.n), device="cuda") for c in cases]
    with mvct.Batch(plans) as b:
        b.bind(p, w, [c.beta for c in cases], imgs, n_iter)
        b.run(n_iter)
        b.stats(0, n_iter)
        first = [im.clone() for im in imgs]
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(graph, stream=s):
                b.run(n_iter, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        for im in imgs:
            im.zero_()
        graph.replay()
        torch.cuda.synchronize()
        b.stats(0, n_iter)
        for a, c in zip(first, imgs):
            assert torch.equal(a, c)
    for pl in plans:
        pl.close()


def test_batch_argument_errors(mvct):
    c = make_cases(3)[0]
    plan = mvct.Plan(c.geom, c.n_subsets)
    with mvct.Batch([plan]) as b:
        with pytest.raises(mvct.MvctError):
            b.run(3)                       # not bound
        with pytest.raises(mvct.MvctError):
            plan.recon(cuda(c.p), cuda(c.w), c.beta, 2)   # plan reserved by the batch
        img = torch.zeros((c.geom.n, c.geom.n), device="cuda")
        with pytest.raises(mvct.MvctError):
            b.bind([cuda(c.p)], [cuda(c.w)], [c.beta], [img], 3, lambda_schedule=None, mu0=float("nan"))
        b.bind([cuda(c.p)], [cuda(c.w)], [c.beta], [img], 3)
        with pytest.raises(mvct.MvctError):
            b.run(4)                       # beyond max_iter
    with pytest.raises(mvct.MvctError):
        mvct.Batch([plan, plan])           # a plan twice
    plan.close()


def test_batch_barrier_timeout_reports_and_recovers(mvct):
    """A group barrier that can never complete (host-side test knob, 50 ms limit)
    ends the batch run with MVCT_ETIMEOUT read by the host; the context stays
    usable and the next bound run matches the reference."""
    cases = make_cases(4, seed0=430)
    plans = [mvct.Plan(c.geom, c.n_subsets) for c in cases]
    p = [cuda(c.p) for c in cases]
    w = [cuda(c.w) for c in cases]
    imgs = [torch.zeros((c.geom.n, c.geom.n), device="cuda") for c in cases]
    with mvct.Batch(plans) as b:
        b.bind(p, w, [c.beta for c in cases], imgs, 4, debug_unreachable_barrier=1, barrier_timeout_ms=50.0)
        b.run(4)
        with pytest.raises(mvct.MvctError) as ei:
            b.stats(0)
        assert ei.value.code == -5          # MVCT_ETIMEOUT
        b.bind(p, w, [c.beta for c in cases], imgs, 4)
        b.run(4)
        b.stats(0)
        ok = [im.clone() for im in imgs]
    for i, c in enumerate(cases):
        ref = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, 4)
        assert rel(ok[i].cpu().numpy(), ref["image"]) < RTOL_IMG
    for pl in plans:
        pl.close()


def test_large_batch_descriptor_array_path(mvct):
    """Batches of more than 96 slices keep their descriptors in global memory
    (the other kernel variant): 100 small slices of two geometries against the
    one-slice runs of the same data."""
    geoms = [ph.Geometry(n=24, n_views=40, n_channels=36), ph.Geometry(n=16, n_views=30, n_channels=28)]
    cases = [ph.make_case("small", 600 + k, geom=geoms[k % 2], n_subsets=5 if k % 2 == 0 else 3, n_iter=6)
             for k in range(100)]
    plans = [mvct.Plan(c.geom, c.n_subsets) for c in cases]
    p = [cuda(c.p) for c in cases]
    w = [cuda(c.w) for c in cases]
    imgs = [torch.zeros((c.geom.n, c.geom.n), device="cuda") for c in cases]
    with mvct.Batch(plans) as b:
        b.bind(p, w, [c.beta for c in cases], imgs, 6)
        b.run(6)
        b.stats(0)
        got = [im.clone() for im in imgs]
    for pl in plans:
        pl.close()
    for k in (0, 1, 57, 98, 99):
        c = cases[k]
        with mvct.Plan(c.geom, c.n_subsets) as plan:
            single, _ = plan.recon(cuda(c.p), cuda(c.w), c.beta, 6)
        assert rel(got[k].cpu().numpy(), single.cpu().numpy()) < 1e-5


def highest_averages(work, G):
    """Blocks per slice: one each, then each further block to the slice with the
    largest work per block (ties to the lower index)."""
    blocks = [1] * len(work)
    for _ in range(G - len(work)):
        k = max(range(len(work)), key=lambda i: (work[i] / blocks[i], -i))
        blocks[k] += 1
    return blocks


def test_blocks_dealt_by_work_per_block(mvct):
    """The grid is split among the slices of an uneven batch so that the largest
    work per block (views/S x channels x n per block) is as small as it can be:
    the launch lasts as long as its slowest group. Checked against the
    highest-averages split computed here, and the two properties that define it."""
    cases = make_cases(2)
    _, stats = run_batch(mvct, cases, 2)
    blocks = [s.grid_blocks for s in stats]
    G = sum(blocks)
    work = [c.geom.n_views // c.n_subsets * c.geom.n_channels * c.geom.n for c in cases]
    assert blocks == highest_averages(work, G)
    worst = max(w / b for w, b in zip(work, blocks))
    # taking a block from any slice and giving it to another never lowers the worst ratio
    for i in range(len(work)):
        for j in range(len(work)):
            if i != j and blocks[i] > 1:
                alt = list(blocks)
                alt[i] -= 1
                alt[j] += 1
                assert max(w / b for w, b in zip(work, alt)) >= worst
