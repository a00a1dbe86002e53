"""The paper's convergence comparisons, measured as trends on the full-size
synthetic case (512^2, 800 x 738, beta = 1e-3; the paper's phantoms and patient
data are not available, so the numbers are compared in kind, not in value):
* Sec. 4.2: the adaptive parameter started from the homogeneous 0.05 /cm image
  against a constant parameter (lambda = 0.01) started from the zero image: how
  many constant-parameter sub-iterations reach the objective the adaptive run has
  after N. The paper reports about three times as many at N = 500. Measured here
  (GB300): 1.5x at N = 50, 1.25x at 100, 1.125x at 200 and 0.8x at 500 -- the
  adaptive run is ahead early, but with lambda driven by the subset's square
  difference (each sub-iteration compares a different subset with the previous
  one) lambda drifts down to its floor within a few hundred sub-iterations, and the
  constant parameter then overtakes it;
* Sec. 4.3: with 40 subsets 500 sub-iterations are not enough to reach what 20
  subsets reach in 500."""
import numpy as np
import pytest
import torch

from paper_1903_10088_gb300 import phantom as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mvct():
    from paper_1903_10088_gb300 import build, mvct

    build.build()
    mvct.lib()
    return mvct


@pytest.fixture(scope="module")
def case():
    return ph.make_case("full", 100)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def psi_curve(mvct, c, S, checkpoints, chunk=25, **opts):
    """Psi after each checkpoint (multiples of `chunk`), one resumed run."""
    p, w = cuda(c.p), cuda(c.w)
    out = {}
    with mvct.Plan(c.geom, S) as plan:
        st = mvct.fresh_state()
        img = torch.zeros((c.geom.n, c.geom.n), device="cuda")
        done = 0
        for n in sorted(checkpoints):
            if n > done:
                first = done == 0
                plan.recon(p, w, c.beta, n - done, img=img, init_from_input=not first or opts.get("mu0") == 0.0,
                           state=st, **opts)
                done = n
            out[n] = float(plan.objective(img, p, w, c.beta, c.tv_eps).cpu())
    return out


def test_adaptive_against_constant_parameter(mvct, case, capsys):
    grid = list(range(25, 3001, 25))
    const = psi_curve(mvct, case, 20, grid, dlambda_up=0.0, dlambda_down=0.0, mu0=0.0)
    adapt = psi_curve(mvct, case, 20, [50, 100, 200, 500])
    ratios = {}
    for n, target in adapt.items():
        hit = next((m for m in grid if const[m] <= target), None)
        ratios[n] = None if hit is None else hit / n
    with capsys.disabled():
        print("\nconstant-parameter sub-iterations / adaptive sub-iterations for the same objective:",
              {n: r for n, r in ratios.items()})
        print("Psi adaptive:", adapt, " constant @500/1000/1500:", const[500], const[1000], const[1500])
    # early on the adaptive run (homogeneous start) is ahead of the constant one from zero
    assert ratios[50] is None or ratios[50] >= 1.25
    assert ratios[100] is None or ratios[100] >= 1.1


def test_forty_subsets_need_more_than_500(mvct, case, capsys):
    psi20 = psi_curve(mvct, case, 20, [500])[500]
    psi40 = psi_curve(mvct, case, 40, [500, 1000])
    with capsys.disabled():
        print(f"\nPsi: S=20 @500 {psi20:.4f}; S=40 @500 {psi40[500]:.4f}, @1000 {psi40[1000]:.4f}")
    assert psi40[500] > psi20
    assert psi40[1000] < psi40[500]


def test_spread_subset_order(mvct, case, capsys):
    """The paper visits its equal-interval subsets in an unstated order (read as
    0, 1, ..., S-1); a spread order (consecutive subsets far apart in angle) is
    measured beside it."""
    order = mvct.spread_order(20)
    seq = psi_curve(mvct, case, 20, [50, 100, 200, 500])
    spr = psi_curve(mvct, case, 20, [50, 100, 200, 500], subset_order=order)
    with capsys.disabled():
        print("\nPsi sequential:", {k: round(v, 4) for k, v in seq.items()},
              "\nPsi spread:    ", {k: round(v, 4) for k, v in spr.items()})
    assert all(np.isfinite(v) for v in spr.values())
