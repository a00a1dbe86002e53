"""Method variants (the paper's comparisons, reproduced as trends on synthetic
data) and the Poisson data term, GPU vs oracle."""
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


def test_poisson_data_term_matches_oracle(mvct):
    c = ph.make_case("small", 21)
    with mvct.Plan(c.geom, c.n_subsets) as plan:
        img, res = plan.recon(cuda(c.p), cuda(c.w), c.beta, c.n_iter, data_term=1)
        img = img.double().cpu().numpy()
    ref = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, c.n_iter, data_term=1)
    assert np.array_equal(res.lam, ref["lam"])
    assert rel(img, ref["image"]) < 1e-4


def test_constant_lambda_baseline_and_adaptive_gain(mvct):
    """Sec. 4.2: the adaptive parameter converges faster than a constant one
    started from the zero image; with dlambda = 0 the parameter stays lambda0."""
    c = ph.make_case("small", 22, n_subsets=10)
    n_iter = 120
    with mvct.Plan(c.geom, c.n_subsets) as plan:
        _, const = plan.recon(cuda(c.p), cuda(c.w), c.beta, n_iter, dlambda_up=0.0, dlambda_down=0.0, mu0=0.0)
        _, adapt = plan.recon(cuda(c.p), cuda(c.w), c.beta, n_iter)
    assert np.all(const.lam == 0.01)
    S = c.n_subsets
    last_pass = lambda r: r.phi[-S:].sum()
    assert last_pass(adapt) < last_pass(const)


def test_ordered_subsets_accelerate_per_pass(mvct):
    """Sec. 3.4 / 4.3: for the same number of passes over the data, more subsets
    reach a lower objective (up to the point where subsets become too thin)."""
    g = ph.Geometry(n=64, n_views=80, n_channels=92)
    psis = {}
    for S in (1, 2, 5, 10):
        c = ph.make_case("small", 23, geom=g, n_subsets=S)
        with mvct.Plan(g, S) as plan:
            img, _ = plan.recon(cuda(c.p), cuda(c.w), c.beta, 3 * S)   # three passes
            psis[S] = float(plan.objective(img, cuda(c.p), cuda(c.w), c.beta, 1e-6).cpu())
    assert psis[10] < psis[5] < psis[2] < psis[1]


def test_subset_order_matches_oracle(mvct):
    """A spread visiting order of the equal-interval subsets (mvct.spread_order):
    GPU and oracle agree (lambda sequence identical, image 1e-4); an order that is
    not a permutation is rejected."""
    c = ph.make_case("small", 24)
    order = mvct.spread_order(c.n_subsets)
    with mvct.Plan(c.geom, c.n_subsets) as plan:
        img, res = plan.recon(cuda(c.p), cuda(c.w), c.beta, c.n_iter, subset_order=order)
        img = img.double().cpu().numpy()
        with pytest.raises(mvct.MvctError):
            plan.recon(cuda(c.p), cuda(c.w), c.beta, 2, subset_order=[0] * c.n_subsets)
    ref = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, c.n_iter, subset_order=order)
    assert np.array_equal(res.lam, ref["lam"])
    assert rel(img, ref["image"]) < 1e-4


@pytest.mark.parametrize("rule", ["subset", "pass", "pass_sliding"])
def test_lambda_rules_match_oracle(mvct, rule):
    """Each reading of Eq. 4-5 under ordered subsets (mvct.h MVCT_LAMBDA_*): 128^2,
    S = 10, 60 sub-iterations (six passes, so the once-per-pass rule decides four
    times), from the homogeneous start: lambda sequence identical, Phi 1e-5,
    image 1e-4, on the default launch shape (a block reduces and publishes Phi)
    and on a shape where every block reduces Phi itself."""
    c = ph.make_case("small", 25)
    ref = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, 60, lambda_rule=rule)
    for shape in ((0, 0), (1, 16)):   # 16 blocks for 16 tiles: no block is free to reduce
        with mvct.Plan(c.geom, c.n_subsets) as plan:
            plan.set_shape(*shape)
            img, res = plan.recon(cuda(c.p), cuda(c.w), c.beta, 60, lambda_rule=rule)
            img = img.double().cpu().numpy()
        assert np.array_equal(res.lam, ref["lam"]), shape
        assert np.allclose(res.phi, ref["phi"], rtol=1e-5)
        assert rel(img, ref["image"]) < 1e-4


@pytest.mark.parametrize("rule", ["pass", "pass_sliding"])
def test_lambda_rules_resume_bitwise(mvct, rule):
    """A run of 27 sub-iterations resumed after 13 (the pass sums straddle the cut,
    S = 10) equals one run of 40 bit for bit."""
    c = ph.make_case("small", 26)
    p, w = cuda(c.p), cuda(c.w)
    with mvct.Plan(c.geom, c.n_subsets) as plan:
        full, rf = plan.recon(p, w, c.beta, 40, lambda_rule=rule)
        full = full.double().cpu().numpy()
        st = mvct.fresh_state()
        img = torch.zeros((c.geom.n, c.geom.n), device="cuda")
        img, r1 = plan.recon(p, w, c.beta, 13, img=img, state=st, lambda_rule=rule)
        img, r2 = plan.recon(p, w, c.beta, 27, img=img, init_from_input=True, state=st, lambda_rule=rule)
        part = img.double().cpu().numpy()
    assert np.array_equal(np.concatenate([r1.lam, r2.lam]), rf.lam)
    assert np.array_equal(part, full)


def test_lambda_rules_in_a_batch(mvct):
    """The batch loop takes the rule from the bound options: two slices of different
    geometry, pass_sliding, against the oracle."""
    cases = [ph.make_case("small", 27), ph.make_case("small", 28, geom=ph.Geometry(n=80, n_views=60, n_channels=90),
                                                    n_subsets=6)]
    plans = [mvct.Plan(c.geom, c.n_subsets) for c in cases]
    imgs = [torch.zeros((c.geom.n, c.geom.n), device="cuda") for c in cases]
    with mvct.Batch(plans) as b:
        b.bind([cuda(c.p) for c in cases], [cuda(c.w) for c in cases], [c.beta for c in cases], imgs, 40,
               lambda_rule="pass_sliding")
        b.run(40)
        stats = [b.stats(i, 40) for i in range(2)]
    for pl in plans:
        pl.close()
    for c, im, s in zip(cases, imgs, stats):
        ref = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, 40, lambda_rule="pass_sliding")
        assert np.array_equal(s.lam, ref["lam"])
        assert rel(im.double().cpu().numpy(), ref["image"]) < 1e-4
