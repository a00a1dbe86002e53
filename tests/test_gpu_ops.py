"""GPU parity of the stand-alone operators against the FP64 oracle, through the C ABI.

Tolerances (relative L2, FP32 kernels vs FP64 oracle on identical FP32 inputs):
projections and backprojections 1e-5, TV gradient 1e-5, FP64-reduced scalars
(TV value, objective) 1e-6; the adjoint identity with FP64 dot products of the
FP32 results 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1903_10088_gb300 import phantom as ph

pytestmark = pytest.mark.gpu

RTOL_PROJ = 1e-5


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


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


GEOMS = {
    "small": ph.GEOM_128,
    "ragged": ph.Geometry(n=37, n_views=30, n_channels=29, view0_rad=0.4, channel_offset=0.3),
    "offset": ph.Geometry(n=64, n_views=96, n_channels=77, view0_rad=-1.1, channel_offset=-0.6,
                          fan_angle_rad=0.6),
}


def phantom_image(g, seed):
    ell = ph.phantom_random_ellipses(seed)
    return ph.rasterize(ell, g.n, g.fov_cm, 2).astype(np.float32)


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("subset_S", [(-1, 1), (0, 2), (1, 2)])
def test_forward_parity(mvct, name, subset_S):
    g = GEOMS[name]
    subset, S = subset_S
    if g.n_views % S:
        pytest.skip("views not divisible")
    img = phantom_image(g, 11)
    with mvct.Plan(g, S) as plan:
        q = host(plan.forward(cuda(img), subset))
    ref = oracle.forward(g, img.astype(np.float64), subset, S)
    assert q.shape == ref.shape
    assert rel(q, ref) < RTOL_PROJ


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("subset_S", [(-1, 1), (1, 2)])
def test_back_parity(mvct, name, subset_S):
    g = GEOMS[name]
    subset, S = subset_S
    rows = g.n_views if subset < 0 else g.n_views // S
    y = np.random.default_rng(12).uniform(-1, 1, (rows, g.n_channels)).astype(np.float32)
    with mvct.Plan(g, S) as plan:
        b = host(plan.back(cuda(y), subset))
    ref = oracle.back(g, y.astype(np.float64), subset, S)
    assert rel(b, ref) < RTOL_PROJ


def test_back_of_ones_has_no_gaps(mvct):
    """A^T 1 is positive exactly where the oracle's is: the gather's channel window
    never misses a ray with a non-zero weight."""
    g = ph.GEOM_128
    with mvct.Plan(g, 1) as plan:
        b = host(plan.back(torch.ones((g.n_views, g.n_channels), device="cuda")))
    ref = oracle.back(g, np.ones((g.n_views, g.n_channels)))
    assert np.array_equal(b > 0, ref > 0)
    assert rel(b, ref) < RTOL_PROJ


def test_adjoint_identity(mvct):
    g = ph.GEOM_128
    rng = np.random.default_rng(13)
    x = rng.uniform(0, 1, (g.n, g.n)).astype(np.float32)
    y = rng.uniform(-1, 1, (g.n_views, g.n_channels)).astype(np.float32)
    with mvct.Plan(g, 1) as plan:
        ax = host(plan.forward(cuda(x)))
        aty = host(plan.back(cuda(y)))
    lhs = np.vdot(ax, y.astype(np.float64))
    rhs = np.vdot(x.astype(np.float64), aty)
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


@pytest.mark.parametrize("n", [1, 2, 3, 37, 128])
def test_tv_parity(mvct, n):
    g = ph.Geometry(n=n, n_views=8, n_channels=8)
    img = np.random.default_rng(14).uniform(0, 0.1, (n, n)).astype(np.float32)
    eps = 1e-6
    with mvct.Plan(g, 1) as plan:
        grad, val = plan.tv_grad(cuda(img), eps)
        grad = host(grad)
        val = float(val.cpu())
    rv, rg = oracle.tv(img.astype(np.float64), eps)
    assert abs(val - rv) <= 1e-6 * rv
    if n > 1:
        assert rel(grad, rg) < RTOL_PROJ
    else:
        assert np.abs(grad).max() == 0.0


def test_objective_parity(mvct):
    c = ph.make_case("small", 15)
    img = phantom_image(c.geom, 15)
    with mvct.Plan(c.geom, c.n_subsets) as plan:
        psi = float(plan.objective(cuda(img), cuda(c.p), cuda(c.w), c.beta, c.tv_eps).cpu())
    ref = oracle.objective(c.geom, img.astype(np.float64), c.p, c.w, c.beta, c.tv_eps)
    assert abs(psi - ref) <= 1e-6 * abs(ref)


@pytest.mark.parametrize("geom", [
    ph.Geometry(n=1, n_views=4, n_channels=3),
    ph.Geometry(n=2, n_views=2, n_channels=1),
    ph.Geometry(n=33, n_views=1, n_channels=65),
    ph.Geometry(n=16, n_views=7, n_channels=2, sad_cm=30.0),
])
def test_degenerate_geometries(mvct, geom):
    img = np.random.default_rng(16).uniform(0, 1, (geom.n, geom.n)).astype(np.float32)
    y = np.random.default_rng(17).uniform(-1, 1, (geom.n_views, geom.n_channels)).astype(np.float32)
    with mvct.Plan(geom, 1) as plan:
        q = host(plan.forward(cuda(img)))
        b = host(plan.back(cuda(y)))
    assert rel(q, oracle.forward(geom, img.astype(np.float64))) < RTOL_PROJ
    assert rel(b, oracle.back(geom, y.astype(np.float64))) < RTOL_PROJ


def test_full_size_projector_sampled(mvct):
    """512^2, 800 views, 738 channels: the rows of one subset of the full-sinogram
    projection and of the subset projection, and the subset backprojection, against
    the oracle (one subset keeps the oracle to seconds)."""
    g = ph.GEOM_512
    img = phantom_image(g, 18)
    y = np.random.default_rng(19).uniform(0, 1, (g.n_views, g.n_channels)).astype(np.float32)
    with mvct.Plan(g, 20) as plan:
        q = host(plan.forward(cuda(img)))
        qs = host(plan.forward(cuda(img), 7))
        b = host(plan.back(cuda(y)))
    # full-sinogram oracle for one subset (40 views) is cheap; compare its rows
    ref7 = oracle.forward(g, img.astype(np.float64), 7, 20)
    assert rel(qs, ref7) < RTOL_PROJ
    assert rel(q[7::20], ref7) < RTOL_PROJ
    # back: oracle over the 40 views of subset 7 against the GPU back of the same rows
    with mvct.Plan(g, 20) as plan:
        bs = host(plan.back(cuda(y[7::20].copy()), 7))
    refb = oracle.back(g, y[7::20].astype(np.float64), 7, 20)
    assert rel(bs, refb) < RTOL_PROJ
    assert np.all(np.isfinite(b))
    # the all-view backprojection path: by linearity, a full sinogram that is zero
    # except on the rows of subset 7 backprojects to the oracle's subset-7 image
    y7 = np.zeros_like(y)
    y7[7::20] = y[7::20]
    with mvct.Plan(g, 20) as plan:
        b7 = host(plan.back(cuda(y7)))
    assert rel(b7, refb) < RTOL_PROJ


def test_invalid_subset_rejected(mvct):
    g = ph.GEOM_128
    with mvct.Plan(g, 10) as plan:
        with pytest.raises(mvct.MvctError):
            plan.forward(torch.zeros((g.n, g.n), device="cuda"), 10,
                         out=torch.zeros((20, g.n_channels), device="cuda"))


@pytest.mark.parametrize("name", ["small", "offset"])
def test_fbp_parity(mvct, name):
    from oracle import fbp as F

    g = GEOMS[name]
    ell = ph.phantom_random_ellipses(31)
    sino = ph.analytic_sinogram(g, ell).astype(np.float32)
    with mvct.Plan(g, 1) as plan:
        img = host(plan.fbp(cuda(sino)))
    ref = F.fbp(g, sino.astype(np.float64))
    assert rel(img, ref) < 1e-4


def test_fbp_full_size_sampled(mvct):
    """512^2, 800 x 738: the GPU FBP of a noisy full-size case against the oracle."""
    from oracle import fbp as F

    c = ph.make_case("full", 32)
    with mvct.Plan(c.geom, 20) as plan:
        img = host(plan.fbp(cuda(c.p)))
    ref = F.fbp(c.geom, c.p.astype(np.float64))
    assert rel(img, ref) < 1e-4


def test_host_pointer_rejected_before_launch(mvct):
    """The C ABI checks that every pointer is device memory of the plan's device
    before it launches anything: a host buffer gives MVCT_EINVAL."""
    import ctypes

    g = ph.GEOM_128
    host = torch.zeros((g.n, g.n), dtype=torch.float32).pin_memory()
    dev = torch.zeros((g.n_views, g.n_channels), device="cuda")
    with mvct.Plan(g, 1) as plan:
        rc = mvct.lib().mvct_forward(plan._h, ctypes.c_void_p(host.data_ptr()), ctypes.c_void_p(dev.data_ptr()),
                                     -1, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == -1
        assert b"not device memory" in mvct.lib().mvct_last_error()
        rc = mvct.lib().mvct_fbp(plan._h, ctypes.c_void_p(dev.data_ptr()), ctypes.c_void_p(host.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == -1
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", ["small", "offset"])
def test_objective_gradient_matches_oracle(mvct, name):
    """mvct_objective_grad: A^T (w (A img - p)) + beta grad TV_eps against the same
    expression built from the oracle's projector, transpose and TV (1e-5), and
    the value against the oracle's objective (1e-6)."""
    g = GEOMS[name]
    img = phantom_image(g, 41)
    rng = np.random.default_rng(42)
    p = rng.uniform(0, 2, (g.n_views, g.n_channels)).astype(np.float32)
    w = rng.uniform(0.1, 1, (g.n_views, g.n_channels)).astype(np.float32)
    beta, eps = 2e-3, 1e-6
    with mvct.Plan(g, 1) as plan:
        grad, val = plan.objective_grad(cuda(img), cuda(p), cuda(w), beta, eps, with_value=True)
        grad, val = host(grad), float(val.cpu())
    i64 = img.astype(np.float64)
    r = oracle.forward(g, i64) - p.astype(np.float64)
    ref = oracle.back(g, w.astype(np.float64) * r) + beta * oracle.tv(i64, eps)[1]
    assert rel(grad, ref) < RTOL_PROJ
    refv = oracle.objective(g, i64, p, w, beta, eps)
    assert abs(val - refv) <= 1e-6 * abs(refv)
