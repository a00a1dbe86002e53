"""Pins of the FP64 oracle against what the paper and mathematics fix (CPU only).

Each test checks the oracle against something other than itself: analytic line
integrals, closed forms, a textbook linear-algebra routine, a brute-force system
matrix built from an independent per-(ray, pixel) formula, or the constants the
paper prints (Eq. 4-5, Sec. 3.3.2, Sec. 3.4).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1903_10088_gb300 import phantom as ph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Independent system matrix: entry (ray, pixel) from the Joseph model written
# per pixel as a triangle ("hat") weight, geometry from the direction angle
# theta = beta + gamma + pi (not the oracle's rotation-matrix route).
# ---------------------------------------------------------------------------
def brute_system_matrix(g: ph.Geometry, views=None) -> np.ndarray:
    n, d = g.n, g.fov_cm / g.n
    cen = (np.arange(n) - (n - 1) / 2.0) * d
    V, C = g.n_views, g.n_channels
    views = range(V) if views is None else views
    rows = []
    for v in views:
        beta = g.view0_rad + 2 * math.pi * v / V
        sx, sy = g.sad_cm * math.cos(beta), g.sad_cm * math.sin(beta)
        for c in range(C):
            th = beta + (c - (C - 1) / 2.0 + g.channel_offset) * g.fan / C + math.pi
            dx, dy = math.cos(th), math.sin(th)
            row = np.zeros((n, n))
            for i in range(n):
                for j in range(n):
                    if abs(dx) >= abs(dy):
                        y = sy + (cen[j] - sx) * dy / dx
                        row[i, j] = d / abs(dx) * max(0.0, 1.0 - abs(y - cen[i]) / d)
                    else:
                        x = sx + (cen[i] - sy) * dx / dy
                        row[i, j] = d / abs(dy) * max(0.0, 1.0 - abs(x - cen[j]) / d)
            rows.append(row.ravel())
    return np.array(rows)


G8 = ph.Geometry(n=8, n_views=32, n_channels=16, view0_rad=0.3, channel_offset=0.25)


@pytest.fixture(scope="module")
def A8():
    return brute_system_matrix(G8)


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


# ------------------------------- projector ---------------------------------
def test_forward_matches_brute_force_matrix(A8):
    rng = np.random.default_rng(1)
    x = rng.uniform(0.0, 0.1, (8, 8))
    q = oracle.forward(G8, x)
    assert np.abs(q.ravel() - A8 @ x.ravel()).max() < 1e-12


def test_back_matches_brute_force_transpose(A8):
    rng = np.random.default_rng(2)
    y = rng.normal(size=(G8.n_views, G8.n_channels))
    b = oracle.back(G8, y)
    ref = A8.T @ y.ravel()
    assert np.abs(b.ravel() - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("s", [0, 3, 7])
def test_subset_rows_are_thinned_views(A8, s):
    """Sec. 3.4: subset s holds views s, s+S, s+2S, ... (equal-interval thinning)."""
    S = 8
    rng = np.random.default_rng(3)
    x = rng.uniform(0.0, 0.1, (8, 8))
    q = oracle.forward(G8, x, subset=s, n_subsets=S)
    Asub = A8.reshape(G8.n_views, G8.n_channels, 64)[s::S].reshape(-1, 64)
    assert q.shape == (G8.n_views // S, G8.n_channels)
    assert np.abs(q.ravel() - Asub @ x.ravel()).max() < 1e-12
    y = rng.normal(size=q.shape)
    ref = Asub.T @ y.ravel()
    assert np.abs(oracle.back(G8, y, s, S).ravel() - ref).max() < 1e-13 * np.abs(ref).max()


def test_adjoint_identity_small_case():
    g = ph.GEOM_128
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (g.n, g.n))
    y = rng.uniform(-1, 1, (g.n_views, g.n_channels))
    lhs = np.vdot(oracle.forward(g, x), y)
    rhs = np.vdot(x, oracle.back(g, y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_forward_converges_to_analytic_line_integrals():
    """Ellipse phantom, pixel-averaged 4x4: the discrete integrals approach the
    exact chord integrals as the grid is refined."""
    ell = ph.phantom_random_ellipses(3)
    errs = []
    for n in (128, 256, 512):
        g = ph.Geometry(n=n, n_views=90, n_channels=184)
        img = ph.rasterize(ell, n, g.fov_cm, 4)
        errs.append(rel(oracle.forward(g, img), ph.analytic_sinogram(g, ell)))
    assert errs[-1] <= 0.02
    assert errs[0] / errs[1] >= 1.5 and errs[1] / errs[2] >= 1.5


def test_forward_exact_on_affine_image():
    """For f = a + b x + c y, linear interpolation and the midpoint rule are exact, so
    every ray whose samples all have both taps inside the image integrates f exactly
    over the image's slab: (fov/|d_major|) f(midpoint)."""
    g = ph.Geometry(n=64, n_views=36, n_channels=61, view0_rad=0.1)
    n, d = g.n, g.delta
    cen = (np.arange(n) - (n - 1) / 2.0) * d
    a, b, c = 0.3, 0.02, -0.015
    img = a + b * cen[None, :] + c * cen[:, None]
    q = oracle.forward(g, img)
    sx, sy, dx, dy = ph.rays(g)
    checked = 0
    for v in range(g.n_views):
        for ch in range(g.n_channels):
            if abs(dx[v, ch]) >= abs(dy[v, ch]):
                u = (sy[v, ch] + (cen - sx[v, ch]) * dy[v, ch] / dx[v, ch] - cen[0]) / d
                y0 = sy[v, ch] + (0.0 - sx[v, ch]) * dy[v, ch] / dx[v, ch]
                expect = g.fov_cm / abs(dx[v, ch]) * (a + c * y0)
            else:
                u = (sx[v, ch] + (cen - sy[v, ch]) * dx[v, ch] / dy[v, ch] - cen[0]) / d
                x0 = sx[v, ch] + (0.0 - sy[v, ch]) * dx[v, ch] / dy[v, ch]
                expect = g.fov_cm / abs(dy[v, ch]) * (a + b * x0)
            if u.min() >= 1e-9 and u.max() <= n - 1 - 1e-9:
                assert abs(q[v, ch] - expect) <= 1e-12 * abs(expect)
                checked += 1
    assert checked > 500


def test_axis_aligned_ray_sums_a_row():
    """A horizontal ray through the centre of row i integrates to delta * sum of row i."""
    n, i = 16, 11
    fov, sad = 40.0, 85.0
    d = fov / n
    yi = (i - (n - 1) / 2.0) * d
    beta = math.asin(yi / sad)           # source height equal to the row centre
    C = 9
    fan = 2.0 * math.asin((fov / 2.0) / sad)
    # the middle channel (gamma = offset * fan/C) must cancel beta: direction angle pi
    g = ph.Geometry(n=n, n_views=4, n_channels=C, fov_cm=fov, sad_cm=sad, view0_rad=beta,
                    channel_offset=-beta / (fan / C))
    rng = np.random.default_rng(5)
    img = rng.uniform(0, 1, (n, n))
    q = oracle.forward(g, img)
    assert abs(q[0, (C - 1) // 2] - d * img[i].sum()) <= 1e-12 * d * img[i].sum()


# ---------------------------------- TV --------------------------------------
def test_tv_constant_image():
    n, eps = 24, 1e-6
    val, grad = oracle.tv(np.full((n, n), 0.37), eps)
    assert abs(val - n * n * math.sqrt(eps)) <= 1e-12 * val
    assert np.abs(grad).max() == 0.0


def test_tv_vertical_step_closed_form():
    n, eps, h = 20, 1e-6, 0.013
    img = np.full((n, n), 0.05)
    img[:, 7:] += h
    val, _ = oracle.tv(img, eps)
    expect = n * math.sqrt(h * h + eps) + (n * n - n) * math.sqrt(eps)
    assert abs(val - expect) <= 1e-12 * expect


def test_tv_gradient_finite_differences():
    n, eps = 12, 1e-4
    rng = np.random.default_rng(6)
    img = rng.uniform(0, 0.1, (n, n))
    _, grad = oracle.tv(img, eps)
    h = 1e-6
    fd = np.zeros_like(img)
    for i in range(n):
        for j in range(n):
            e = np.zeros_like(img)
            e[i, j] = h
            fd[i, j] = (oracle.tv(img + e, eps, False)[0] - oracle.tv(img - e, eps, False)[0]) / (2 * h)
    assert rel(grad, fd) < 1e-6


def test_objective_is_half_weighted_residual_plus_beta_tv(A8):
    """Psi = 1/2 sum w (A mu - p)^2 + beta TV_eps(mu) (Eq. 1-2 with R1, R3, R12):
    the data term through the brute-force matrix, the TV term on a vertical step
    whose TV has the closed form of test_tv_vertical_step_closed_form."""
    n, eps, beta, h = G8.n, 1e-6, 3e-3, 0.013
    img = np.full((n, n), 0.05)
    img[:, 3:] += h
    rng = np.random.default_rng(12)
    p = A8 @ img.ravel() + rng.normal(0, 0.02, A8.shape[0])
    w = rng.uniform(0.2, 1.0, A8.shape[0])
    data = 0.5 * float(np.sum(w * (A8 @ img.ravel() - p) ** 2))
    tv = n * math.sqrt(h * h + eps) + (n * n - n) * math.sqrt(eps)
    got = oracle.objective(G8, img, p.reshape(G8.n_views, G8.n_channels), w.reshape(G8.n_views, G8.n_channels),
                           beta, eps)
    assert abs(got - (data + beta * tv)) <= 1e-11 * (data + beta * tv)


# --------------------------------- set-up -----------------------------------
def test_setup_diagonal_and_mask(A8):
    rng = np.random.default_rng(7)
    w = rng.uniform(0.1, 1.0, (G8.n_views, G8.n_channels))
    beta, eps = 1e-3, 1e-6
    D, M = oracle.setup(G8, w, beta, eps)
    a1t = A8.T @ np.ones(A8.shape[0])
    awa = A8.T @ (w.ravel() * (A8 @ np.ones(64)))
    M_ref = a1t > 0
    D_ref = np.where(M_ref, 1.0 / (awa + beta * 8.0 / math.sqrt(eps)), 0.0)
    assert np.array_equal(M.ravel(), M_ref)
    assert rel(D, D_ref) < 1e-13


def test_surrogate_majorises_hessian(A8):
    """diag(1/D) - (A^T W A + beta * TV Hessian bound) must be positive semidefinite."""
    rng = np.random.default_rng(8)
    w = rng.uniform(0.1, 1.0, (G8.n_views, G8.n_channels))
    D, M = oracle.setup(G8, w, 0.0, 1e-6)
    H = A8.T @ (w.ravel()[:, None] * A8)
    m = M.ravel()
    Dm = np.diag(1.0 / D.ravel()[m]) - H[np.ix_(m, m)]
    assert np.linalg.eigvalsh(Dm).min() > -1e-10


# ---------------------------------- loop ------------------------------------
def test_paper_constants_are_the_defaults():
    gold = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    assert oracle.DEFAULTS["lambda0"] == gold["lambda0"]["value"]
    assert oracle.DEFAULTS["dlambda_up"] == gold["dlambda_up"]["value"]
    assert oracle.DEFAULTS["dlambda_down"] == gold["dlambda_down"]["value"]
    assert oracle.DEFAULTS["mu0"] in gold["mu0_tested"]["value"]
    for S, height in zip(gold["thinning"]["value"], gold["subset_height"]["value"]):
        g = ph.Geometry(n=4, n_views=gold["views_per_rotation"]["value"], n_channels=1)
        assert oracle.forward(g, np.zeros((4, 4)), 0, S).shape[0] == height


def test_lambda_rule_and_best_iterate_follow_eq4_eq5():
    c = ph.make_case("small", 1)
    r = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, 40, want_best=True, lambda_rule="subset")
    phi, lam = r["phi"], r["lam"]
    assert lam[0] == 0.01
    for k in range(1, len(phi)):
        if phi[k] < phi[k - 1]:
            expect = lam[k - 1] + 1e-4
        elif phi[k] > phi[k - 1]:
            expect = lam[k - 1] - 2e-4
        else:
            expect = lam[k - 1]
        assert lam[k] == max(expect, 1e-4)
    S = c.n_subsets
    passes = [phi[k - S + 1:k + 1].sum() for k in range(S - 1, len(phi))]
    assert r["best_n"] == S - 1 + int(np.argmin(passes))


def test_lambda_replay_reproduces_the_adaptive_run():
    """Replaying an adaptive run's own lambda sequence (the mode the GPU parity
    tests use to separate arithmetic from a flipped Eq. 4-5 decision) gives the
    same iterates bit for bit; another schedule gives other iterates and is
    taken verbatim."""
    c = ph.make_case("small", 2)
    n_iter = 12
    r = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, n_iter)
    rr = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, n_iter, lambda_schedule=r["lam"])
    assert np.array_equal(rr["image"], r["image"]) and np.array_equal(rr["lam"], r["lam"])
    r2 = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, n_iter, lambda_schedule=np.full(n_iter, 0.005))
    assert np.all(r2["lam"] == 0.005)
    assert rel(r2["image"], r["image"]) > 1e-3


def _eq45(lam_prev, now, before):
    """Eq. 4-5 with the paper's constants and the floor: one decision."""
    if now < before:
        lam = lam_prev + 1e-4
    elif now > before:
        lam = lam_prev - 2e-4
    else:
        lam = lam_prev
    return max(lam, 1e-4)


def test_pass_rules_follow_their_comparisons():
    """The two pass readings of Sec. 3.3.2 under ordered subsets, checked on the
    run's own square differences: "pass_sliding" compares Phi_n with Phi_{n-S}
    (the pass sums P_n and P_{n-1}) from n = S on and keeps lambda0 during the
    first pass; "pass" decides once per pass, at n = kS (k >= 2), on the sums of
    the last two complete passes, and keeps lambda between decisions."""
    c = ph.make_case("small", 2)
    S, N = 4, 36
    r = oracle.recon(c.geom, S, c.p, c.w, c.beta, N, lambda_rule="pass_sliding")
    phi, lam = r["phi"], r["lam"]
    assert np.all(lam[:S] == 0.01)
    for n in range(S, N):
        assert lam[n] == _eq45(lam[n - 1], phi[n], phi[n - S])
    assert np.any(lam != 0.01)
    r = oracle.recon(c.geom, S, c.p, c.w, c.beta, N, lambda_rule="pass")
    phi, lam = r["phi"], r["lam"]
    assert np.all(lam[:2 * S] == 0.01)
    for n in range(2 * S, N):
        if n % S:
            assert lam[n] == lam[n - 1]
        else:
            now = sum(phi[k] for k in range(n - S, n))
            before = sum(phi[k] for k in range(n - 2 * S, n - S))
            assert lam[n] == _eq45(lam[n - 1], now, before)
    assert np.any(lam != 0.01)


def test_pass_readings_coincide_with_the_subset_reading_without_subsets():
    """With one subset (S = 1) the pass of the sliding reading is one sub-iteration,
    so it compares Phi_n with Phi_{n-1} exactly like the subset reading: the runs
    are identical bit for bit; and every reading gives the same first pass."""
    c = ph.make_case("small", 3, geom=ph.Geometry(n=48, n_views=40, n_channels=60))
    a = oracle.recon(c.geom, 1, c.p, c.w, c.beta, 12, lambda_rule="subset")
    b = oracle.recon(c.geom, 1, c.p, c.w, c.beta, 12, lambda_rule="pass_sliding")
    assert np.array_equal(a["image"], b["image"]) and np.array_equal(a["lam"], b["lam"])
    S = 4
    runs = [oracle.recon(c.geom, S, c.p, c.w, c.beta, S, lambda_rule=rule)
            for rule in ("subset", "pass", "pass_sliding")]
    # during the first pass the pass readings hold lambda0; with lambda replayed the
    # subset reading's run is the same arithmetic
    for r in runs[1:]:
        assert np.array_equal(r["image"], runs[1]["image"])
    rep = oracle.recon(c.geom, S, c.p, c.w, c.beta, S, lambda_schedule=np.full(S, 0.01), lambda_rule="subset")
    assert np.array_equal(rep["image"], runs[1]["image"])


@pytest.mark.parametrize("rule", ["pass", "pass_sliding"])
def test_lambda_replay_reproduces_each_pass_rule(rule):
    c = ph.make_case("small", 4)
    r = oracle.recon(c.geom, 5, c.p, c.w, c.beta, 30, lambda_rule=rule)
    rep = oracle.recon(c.geom, 5, c.p, c.w, c.beta, 30, lambda_schedule=r["lam"], lambda_rule=rule)
    assert np.array_equal(r["image"], rep["image"])


def test_first_step_is_preconditioned_gradient_step(A8):
    """One sub-iteration with S subsets equals mu0 - tau D (S A_s^T W_s (A_s mu0 - p_s)
    + beta grad TV), clamped at 0, with A_s taken from the brute-force matrix."""
    rng = np.random.default_rng(9)
    S, beta = 4, 2e-3
    w = rng.uniform(0.2, 1.0, (G8.n_views, G8.n_channels))
    p = rng.uniform(0.0, 0.5, (G8.n_views, G8.n_channels))
    mu0 = rng.uniform(0.02, 0.1, (8, 8))
    lam = 0.013
    r = oracle.recon(G8, S, p, w, beta, 1, init=mu0, lambda_schedule=[lam])
    D, M = oracle.setup(G8, w, beta, 1e-6)
    As = A8.reshape(G8.n_views, G8.n_channels, 64)[0::S].reshape(-1, 64)
    ws, ps = w[0::S].ravel(), p[0::S].ravel()
    g = As.T @ (ws * (As @ mu0.ravel() - ps))
    _, tvg = oracle.tv(mu0, 1e-6)
    kappa = oracle.DEFAULTS["kappa"]
    expect = np.maximum(0.0, mu0.ravel() - kappa * lam * D.ravel() * (S * g + beta * tvg.ravel()))
    assert np.abs(r["image"].ravel() - expect).max() < 1e-13
    assert abs(r["phi"][0] - np.sum((As @ mu0.ravel() - ps) ** 2)) < 1e-12 * r["phi"][0]


def test_objective_decreases_monotonically_at_small_step():
    """S = 1 and a fixed step kappa*lambda = 0.5 on the surrogate-preconditioned
    gradient: Psi must fall at every iteration."""
    g = ph.Geometry(n=32, n_views=48, n_channels=44)
    c = ph.make_case("small", 2, geom=g)
    prev = None
    img = None
    for k in range(12):
        r = oracle.recon(g, 1, c.p, c.w, c.beta, 1, init=img, lambda_schedule=[0.5 / oracle.DEFAULTS["kappa"]])
        img = r["image"]
        psi = oracle.objective(g, img, c.p, c.w, c.beta, 1e-6)
        if prev is not None:
            assert psi < prev
        prev = psi


def test_wls_limit_matches_cholesky_solution(A8):
    """beta = 0, S = 1, noise-free data: the loop converges to the weighted-least-
    squares solution obtained with a dense Cholesky factorisation."""
    rng = np.random.default_rng(10)
    x = rng.uniform(0.02, 0.1, (8, 8))
    w = rng.uniform(0.2, 1.0, (G8.n_views, G8.n_channels))
    p = (A8 @ x.ravel()).reshape(G8.n_views, G8.n_channels)
    H = A8.T @ (w.ravel()[:, None] * A8)
    L = np.linalg.cholesky(H)
    sol = np.linalg.solve(L.T, np.linalg.solve(L, A8.T @ (w.ravel() * p.ravel())))
    r = oracle.recon(G8, 1, p, w, 0.0, 1500, lambda_schedule=np.full(1500, 0.019))
    assert rel(r["image"], sol) < 1e-6


def test_noise_free_generator_gives_analytic_projection():
    c = ph.make_case("small", 4, noise=False)
    li = ph.analytic_sinogram(c.geom, c.ellipses)
    assert np.allclose(c.p, li, rtol=1e-6, atol=1e-6)
    assert np.allclose(c.w, np.exp(-li), rtol=1e-6)


def test_poisson_gradient_matches_finite_differences(A8):
    """The Poisson data term's first step uses e = w - exp(-q): compare the step
    with one built from a central finite-difference gradient of the negative
    Poisson log-likelihood (divided by I0)."""
    rng = np.random.default_rng(11)
    w = rng.uniform(0.2, 1.0, (G8.n_views, G8.n_channels))
    p = -np.log(w)
    mu0 = rng.uniform(0.02, 0.1, (8, 8))
    lam, S = 0.011, 1
    r = oracle.recon(G8, S, p, w, 0.0, 1, init=mu0, lambda_schedule=[lam], data_term=1)
    D, _ = oracle.setup(G8, w, 0.0, 1e-6)

    def nll(x):
        q = A8 @ x
        return np.sum(w.ravel() * q + np.exp(-q))

    h = 1e-6
    grad = np.array([(nll(mu0.ravel() + h * e) - nll(mu0.ravel() - h * e)) / (2 * h) for e in np.eye(64)])
    expect = np.maximum(0.0, mu0.ravel() - oracle.DEFAULTS["kappa"] * lam * D.ravel() * grad)
    assert np.abs(r["image"].ravel() - expect).max() < 1e-8


def test_poisson_term_reduces_to_wls_near_the_data(A8):
    """With p = ln(1/w) exactly, w - exp(-q) = w (q - p) + O((q - p)^2): the two data
    terms give the same first step to second order."""
    rng = np.random.default_rng(12)
    x = rng.uniform(0.02, 0.1, (8, 8))
    q = (A8 @ x.ravel()).reshape(G8.n_views, G8.n_channels)
    w = np.exp(-q)
    p = q.copy()
    mu0 = x + 2e-5 * rng.normal(size=x.shape)
    a = oracle.recon(G8, 1, p, w, 0.0, 1, init=mu0, lambda_schedule=[0.01], data_term=0)["image"]
    b = oracle.recon(G8, 1, p, w, 0.0, 1, init=mu0, lambda_schedule=[0.01], data_term=1)["image"]
    # the difference is second order in q - p (here |q - p| < 1e-3): relative 1e-3 of the step
    dq = np.abs(A8 @ (mu0 - x).ravel()).max()
    assert dq < 1e-3
    assert np.abs(a - b).max() < dq * np.abs(a - mu0).max()


def test_subset_order_first_steps_use_the_listed_subsets(A8):
    """With subset_order = (2, 0, 3, 1), sub-iteration n uses subset order[n mod 4]:
    the first sub-iteration is the preconditioned gradient step with A_2 (brute
    force), the second Phi is the square difference on subset 0, and the identity
    order reproduces the default run bit for bit."""
    rng = np.random.default_rng(10)
    S, beta, lam = 4, 2e-3, 0.011
    w = rng.uniform(0.2, 1.0, (G8.n_views, G8.n_channels))
    p = rng.uniform(0.0, 0.5, (G8.n_views, G8.n_channels))
    mu0 = rng.uniform(0.02, 0.1, (8, 8))
    order = [2, 0, 3, 1]
    r1 = oracle.recon(G8, S, p, w, beta, 1, init=mu0, lambda_schedule=[lam], subset_order=order)
    D, M = oracle.setup(G8, w, beta, 1e-6)
    A3 = A8.reshape(G8.n_views, G8.n_channels, 64)
    As = A3[2::S].reshape(-1, 64)
    g = As.T @ (w[2::S].ravel() * (As @ mu0.ravel() - p[2::S].ravel()))
    _, tvg = oracle.tv(mu0, 1e-6)
    kappa = oracle.DEFAULTS["kappa"]
    expect = np.maximum(0.0, mu0.ravel() - kappa * lam * D.ravel() * (S * g + beta * tvg.ravel()))
    assert np.abs(r1["image"].ravel() - expect).max() < 1e-13
    r2 = oracle.recon(G8, S, p, w, beta, 2, init=mu0, lambda_schedule=[lam, lam], subset_order=order)
    A0 = A3[0::S].reshape(-1, 64)
    assert abs(r2["phi"][1] - np.sum((A0 @ r1["image"].ravel() - p[0::S].ravel()) ** 2)) < 1e-12 * r2["phi"][1]
    ident = oracle.recon(G8, S, p, w, beta, 9, init=mu0, subset_order=[0, 1, 2, 3])
    base = oracle.recon(G8, S, p, w, beta, 9, init=mu0)
    assert np.array_equal(ident["image"], base["image"]) and np.array_equal(ident["lam"], base["lam"])
