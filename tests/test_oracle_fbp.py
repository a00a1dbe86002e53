"""Pins of the FP64 fan-beam FBP oracle against exact projections of analytic
phantoms (CPU only)."""
import numpy as np

from oracle import fbp as F
from paper_1903_10088_gb300 import phantom as ph


def grid(g):
    cen = (np.arange(g.n) - (g.n - 1) / 2.0) * g.delta
    return np.meshgrid(cen, cen)


def test_uniform_disk_value_and_background():
    g = ph.Geometry(n=128, n_views=360, n_channels=256)
    img = F.fbp(g, ph.analytic_sinogram(g, [ph.Ellipse(0, 0, 10, 10, 0, 0.07)]))
    X, Y = grid(g)
    r2 = X ** 2 + Y ** 2
    assert abs(img[r2 < 25].mean() - 0.07) < 1e-4            # 0.15 % of the disk value
    assert abs(img[(r2 > 144) & (r2 < 324)].mean()) < 1e-4   # empty ring outside the disk


def test_off_centre_ellipse_and_refinement():
    """An ellipse phantom: the error inside the object falls as the grid is refined."""
    ell = ph.phantom_random_ellipses(5)
    errs = []
    for n, V, C in ((128, 200, 184), (256, 400, 368)):
        g = ph.Geometry(n=n, n_views=V, n_channels=C)
        img = F.fbp(g, ph.analytic_sinogram(g, ell))
        tr = ph.rasterize(ell, n, g.fov_cm, 4)
        X, Y = grid(g)
        inner = X ** 2 + Y ** 2 < 13 ** 2
        errs.append(np.linalg.norm((img - tr)[inner]) / np.linalg.norm(tr[inner]))
    assert errs[1] < 0.015 and errs[1] < errs[0]


def test_fan_filter_is_the_equiangular_ramp():
    """g(0) = 1/(8 a^2), zero at even offsets, -1/(2 pi^2 sin^2(k a)) at odd k;
    for small angles it tends to half the parallel-beam ramp -1/(2 pi^2 (k a)^2)."""
    C, a = 9, 0.01
    g = F.fan_filter(C, a)
    k = np.arange(-(C - 1), C)
    assert np.isclose(g[C - 1], 1 / (8 * a * a), rtol=1e-15)
    assert np.all(g[(k % 2 == 0) & (k != 0)] == 0)
    odd = k % 2 == 1
    assert np.allclose(g[odd] * 2 * np.pi ** 2 * np.sin(k[odd] * a) ** 2, -1.0, rtol=1e-13)
    # small-angle limit: (k a)^2 / sin^2(k a) - 1 ~ (k a)^2 / 3 <= 2.2e-3 here
    assert np.allclose(g[odd], -1 / (2 * np.pi ** 2 * (k[odd] * a) ** 2), rtol=3e-3)


def test_start_angle_places_the_object():
    """A small disk 11.7 cm off centre scanned from a start angle of 0.4 rad: the
    reconstruction has the disk's value at its true place (dropping the start
    angle, or flipping its sign, moves the disk about 4.7 cm away)."""
    g = ph.Geometry(n=128, n_views=360, n_channels=256, view0_rad=0.4)
    img = F.fbp(g, ph.analytic_sinogram(g, [ph.Ellipse(10.0, -6.0, 2.0, 2.0, 0, 0.07)]))
    X, Y = grid(g)
    assert abs(img[(X - 10.0) ** 2 + (Y + 6.0) ** 2 < 1.0].mean() - 0.07) < 2e-4


def test_detector_offset_is_inverted_consistently():
    """A whole-channel detector offset relabels the channels (channel c of the
    offset detector is channel c + 1 of the centred one); reconstructing each
    sinogram with its own geometry gives the same image (a wrong offset sign
    leaves a 25 % error)."""
    ell = [ph.Ellipse(3.0, 2.0, 5.0, 3.0, 0.3, 0.07)]
    g0 = ph.Geometry(n=128, n_views=360, n_channels=256)
    g1 = ph.Geometry(n=128, n_views=360, n_channels=256, channel_offset=1.0)
    s0, s1 = ph.analytic_sinogram(g0, ell), ph.analytic_sinogram(g1, ell)
    assert np.array_equal(s1[:, :-1], s0[:, 1:])
    a, b = F.fbp(g1, s1), F.fbp(g0, s0)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-3
