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
