"""Launch-shape autotuner of the loop (mvct_plan_tune / mvct_plan_set_shape /
mvct_batch_tune): every shape the tuner may pick gives the oracle's result, the
tuner keeps a shape no slower than the default, and batch tuning leaves the
bound images as they were."""
import numpy as np
import pytest
import torch

import oracle
from paper_1903_10088_gb300 import phantom as ph

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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("groups,bps", [(1, 0), (3, 0), (8, 0), (2, 2), (8, 2), (4, 3)])
def test_every_shape_matches_oracle(mvct, groups, bps):
    """256^2, 400 views x 368 channels, S = 20 (64 tiles): with 2 blocks per SM
    and 8 groups each block takes several (tile, group) items."""
    g = ph.GEOM_256
    c = ph.make_case("full", 7, geom=g, n_iter=12, n_subsets=20)
    ref = oracle.recon(g, c.n_subsets, c.p, c.w, c.beta, c.n_iter)
    with mvct.Plan(g, c.n_subsets) as plan:
        plan.set_shape(groups, bps * sms())
        img, res = plan.recon(cuda(c.p), cuda(c.w), c.beta, c.n_iter)
        torch.cuda.synchronize()
        assert res.grid_blocks == (bps * sms() if bps else res.grid_blocks)
        assert np.array_equal(res.lam, ref["lam"])
        assert rel(img.cpu().numpy(), ref["image"]) < 1e-4


def test_full_size_shapes_agree(mvct):
    """512^2, 800 x 738: 8 groups on 2 blocks per SM (about 7 items per block),
    one group per tile on 3 blocks per SM, and two groups per tile on every
    block against the default shape (the balanced plan of items), 6
    sub-iterations."""
    c = ph.make_case("full", 100)
    out = {}
    for shape in [(0, 0), (8, 2 * sms()), (1, 3 * sms()), (2, 0)]:
        with mvct.Plan(c.geom, c.n_subsets) as plan:
            plan.set_shape(*shape)
            img, res = plan.recon(cuda(c.p), cuda(c.w), c.beta, 6)
            out[shape] = (img.cpu().numpy(), res.lam)
    base_img, base_lam = out[(0, 0)]
    for shape, (img, lam) in out.items():
        assert np.array_equal(lam, base_lam)
        assert rel(img, base_img) < 1e-5


def test_plan_tune_keeps_fastest_and_stays_correct(mvct):
    c = ph.make_case("small", 3)
    with mvct.Plan(c.geom, c.n_subsets) as plan:
        rep = plan.tune(cuda(c.p), cuda(c.w), c.beta, 20)
        assert rep["ms_per_iter"] <= rep["default_ms_per_iter"]
        assert len(rep["candidates"]) >= 2
        assert (rep["groups"], rep["grid_blocks"]) in [(x["groups"], x["grid_blocks"]) for x in rep["candidates"]]
        img, res = plan.recon(cuda(c.p), cuda(c.w), c.beta, c.n_iter)
        assert res.grid_blocks == rep["grid_blocks"]
    ref = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, c.n_iter)
    assert np.array_equal(res.lam, ref["lam"])
    assert rel(img.cpu().numpy(), ref["image"]) < 1e-4


def test_batch_tune_restores_images_and_keeps_results(mvct):
    geoms = [ph.GEOM_128, ph.Geometry(n=96, n_views=160, n_channels=140), ph.GEOM_128]
    cases = [ph.make_case("small", 40 + k, geom=g, n_subsets=10, n_iter=10) for k, g in enumerate(geoms)]
    plans = [mvct.Plan(c.geom, c.n_subsets) for c in cases]
    p = [cuda(c.p) for c in cases]
    w = [cuda(c.w) for c in cases]
    starts = [torch.full((c.geom.n, c.geom.n), 0.03, device="cuda") for c in cases]
    imgs = [s.clone() for s in starts]
    with mvct.Batch(plans) as b:
        b.bind(p, w, [c.beta for c in cases], imgs, 10, init_from_input=True)
        b.run(10)
        b.stats(0)
        untuned = [im.clone() for im in imgs]
        for im, s in zip(imgs, starts):
            im.copy_(s)
        rep = b.tune(10)
        torch.cuda.synchronize()
        for im, s in zip(imgs, starts):
            assert torch.equal(im, s)              # bound start images restored
        assert rep["ms_per_iter"] <= rep["default_ms_per_iter"]
        b.run(10)
        b.stats(0)
        for a, u in zip(imgs, untuned):
            assert rel(a.cpu().numpy(), u.cpu().numpy()) < 1e-5
    for pl in plans:
        pl.close()


def test_shape_arguments_rejected(mvct):
    with mvct.Plan(ph.GEOM_128, 10) as plan:
        with pytest.raises(mvct.MvctError):
            plan.set_shape(99, 0)
        with pytest.raises(mvct.MvctError):
            plan.set_shape(0, 10 ** 6)
