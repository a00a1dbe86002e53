"""The oracle's multi-threaded mode (used only to time the CPU baseline over all
host cores) gives the same numbers as its single-threaded mode: bit for bit for
the C oracle (rays and views are shared out without changing any rounding), and
within 1e-12 for the FBP, whose threads add their view runs' images in run order.
"""
import numpy as np
import pytest

import oracle
from oracle import fbp as F
from paper_1903_10088_gb300 import phantom as ph


@pytest.fixture
def threads4():
    got = oracle.set_threads(4)
    yield got
    oracle.set_threads(1)


def test_forward_and_back_are_bit_identical_across_thread_counts(threads4):
    c = ph.make_case("small", 5)
    g = c.geom
    img = np.random.default_rng(1).uniform(0, 0.1, (g.n, g.n))
    y = np.random.default_rng(2).uniform(-1, 1, (g.n_views, g.n_channels))
    many = (oracle.forward(g, img), oracle.forward(g, img, 3, 10), oracle.back(g, y),
            oracle.back(g, y[3::10], 3, 10))
    oracle.set_threads(1)
    one = (oracle.forward(g, img), oracle.forward(g, img, 3, 10), oracle.back(g, y),
           oracle.back(g, y[3::10], 3, 10))
    for a, b in zip(many, one):
        assert np.array_equal(a, b)


def test_recon_is_bit_identical_across_thread_counts(threads4):
    c = ph.make_case("small", 6)
    many = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, c.n_iter)
    oracle.set_threads(1)
    one = oracle.recon(c.geom, c.n_subsets, c.p, c.w, c.beta, c.n_iter)
    assert np.array_equal(many["image"], one["image"])
    assert np.array_equal(many["lam"], one["lam"]) and np.array_equal(many["phi"], one["phi"])


def test_threaded_fbp_equals_serial_fbp():
    c = ph.make_case("small", 7)
    a = F.fbp(c.geom, c.p)
    b = F.fbp(c.geom, c.p, threads=5)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
