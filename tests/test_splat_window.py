"""Geometry of the splat's channel windows (host arithmetic, no GPU).

The backprojection walks, for each 32x32 pixel tile and view, only the channels
inside a window: the angular extent, seen from the source, of the tile's box of
pixel centres grown by one pixel, widened by 0.01 channel (mvct_device.cuh,
tile_window). This checks in FP64, over every tile and (a stride of) the views
of the benchmarked geometries, that each ray with a non-zero Joseph weight on a
pixel of the tile (Sec. 2: linear interpolation between the two rows or columns
that bracket the ray at each sample) lies inside that window, and that the
nearest such ray sits inside the unwidened extent, so the 0.01-channel margin is
left entirely for rounding."""
import math

import numpy as np
import pytest

from paper_1903_10088_gb300 import phantom as ph

TILE = 32
MARGIN = 0.01


def ray_lines(g):
    """(x-driven flag, slope m, centre-line coordinate u_c) of every ray, index units."""
    sx, sy, dx, dy = ph.rays(g)
    pc = (g.n - 1) / 2.0
    xd = np.abs(dx) >= np.abs(dy)
    with np.errstate(divide="ignore", invalid="ignore"):
        m = np.where(xd, dy / dx, dx / dy)
        uc = np.where(xd, (sy - sx * dy / dx) / g.delta + pc, (sx - sy * dx / dy) / g.delta + pc)
    return xd, m, uc


def window_bounds(g, v, ti, tj):
    """Unrounded angular extent (in channels) of the tile's grown box, as tile_window computes it."""
    pc = (g.n - 1) / 2.0
    beta = g.view0_rad + 2.0 * math.pi * v / g.n_views
    Sx, Sy = g.sad_cm * math.cos(beta), g.sad_cm * math.sin(beta)
    ex, ey = -math.cos(beta), -math.sin(beta)
    inv_dg = g.n_channels / g.fan
    c_mid = (g.n_channels - 1) / 2.0 - g.channel_offset
    cs = []
    for jj in (tj - 1, tj + TILE):
        for ii in (ti - 1, ti + TILE):
            px, py = (jj - pc) * g.delta - Sx, (ii - pc) * g.delta - Sy
            dot, crs = px * ex + py * ey, ex * py - ey * px
            assert dot > 0
            cs.append(math.atan(crs / dot) * inv_dg + c_mid)
    return min(cs), max(cs)


@pytest.mark.parametrize("g, view_step", [
    (ph.GEOM_128, 1),
    (ph.GEOM_256, 3),
    (ph.GEOM_512, 16),
    (ph.Geometry(n=130, n_views=90, n_channels=120, channel_offset=0.25, view0_rad=0.3), 1),
])
def test_every_weighted_ray_is_in_its_window(g, view_step):
    xd, m, uc = ray_lines(g)
    pc = (g.n - 1) / 2.0
    cc = np.arange(g.n_channels)
    closest = np.inf
    for v in range(0, g.n_views, view_step):
        for ti in range(0, g.n, TILE):
            for tj in range(0, g.n, TILE):
                lo, hi = window_bounds(g, v, ti, tj)
                c0 = max(0, math.ceil(lo - MARGIN))
                c1 = min(g.n_channels - 1, math.floor(hi + MARGIN))
                # sample positions along the driving axis that lie in the tile, and the
                # minor-axis range whose two taps reach the tile
                p_lo = np.where(xd[v], tj, ti)
                minor = np.where(xd[v], ti, tj)
                p_hi = np.minimum(p_lo + TILE - 1, g.n - 1)
                ua, ub = m[v] * (p_lo - pc) + uc[v], m[v] * (p_hi - pc) + uc[v]
                lo_u, hi_u = np.minimum(ua, ub), np.maximum(ua, ub)
                last = np.minimum(minor + TILE - 1, g.n - 1)
                hit = (np.floor(hi_u) >= minor - 1) & (np.floor(lo_u) <= last)
                assert not np.any(hit & ((cc < c0) | (cc > c1))), (v, ti, tj)
                if hit.any():
                    closest = min(closest, cc[hit].min() - lo, hi - cc[hit].max())
    assert closest >= 0.0
