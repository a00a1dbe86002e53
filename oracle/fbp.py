"""FP64 fan-beam filtered backprojection (TEST INFRASTRUCTURE ONLY).

The paper's clinical comparison and the reconstruction loop's plain start image
(Sec. 1, Sec. 4.5: FBP). The paper does not define its filter; this is the
textbook equiangular fan-beam FBP written out step by step:

  1. cosine pre-weighting  R'(beta, gamma) = R(beta, gamma) * D cos(gamma), D = SAD
  2. filtering along gamma with the fan-beam ramp
         g(n a) = 1/2 (n a / sin(n a))^2 h(n a),  a = channel pitch (rad),
     h the band-limited ramp sampled at pitch a: h(0) = 1/(4 a^2), h(n a) = 0 for
     even n != 0, -1/(n^2 pi^2 a^2) for odd n; so g(0) = 1/(8 a^2) and
     g(n a) = -1/(2 pi^2 sin^2(n a)) for odd n;
         Q(beta, gamma_n) = a sum_k R'(beta, gamma_k) g(gamma_n - gamma_k)
  3. weighted backprojection over the full rotation
         f(x, y) = dbeta sum_v Q(beta_v, gamma'(x, y)) / L^2(x, y, beta_v),
     L the source-pixel distance, gamma' the angle of the ray through the pixel,
     Q interpolated linearly in gamma (0 outside the detector), dbeta = 2 pi / V.

Pinned in tests/test_oracle_fbp.py against exact (analytic) projections of
ellipse phantoms: the reconstruction approaches the pixelised phantom.
"""
from __future__ import annotations

import math

import numpy as np


def fan_filter(C: int, a: float) -> np.ndarray:
    """g(k a) for k = -(C-1) .. C-1 (index k + C - 1)."""
    k = np.arange(-(C - 1), C, dtype=np.float64)
    g = np.zeros_like(k)
    g[k == 0] = 1.0 / (8.0 * a * a)
    odd = (np.abs(k) % 2) == 1
    g[odd] = -1.0 / (2.0 * math.pi ** 2 * np.sin(k[odd] * a) ** 2)
    return g


def fbp(geom, sino, threads: int = 1) -> np.ndarray:
    """FBP image [n][n] (1/cm) from log projections [V][C] of `geom`.

    threads > 1 (a timed CPU baseline over the host cores) backprojects
    contiguous runs of views in worker threads, each into its own image (views in
    order), and adds the run images in run order: the same sum as threads = 1 up
    to the grouping of the additions (pinned to 1e-12 relative)."""
    n, V, C = geom.n, geom.n_views, geom.n_channels
    a = geom.fan / C
    D = geom.sad_cm
    sino = np.asarray(sino, dtype=np.float64).reshape(V, C)
    gam = (np.arange(C) - (C - 1) / 2.0 + geom.channel_offset) * a
    pre = sino * (D * np.cos(gam))[None, :]
    g = fan_filter(C, a)
    q = np.zeros((V, C))
    for v in range(V):
        # q[n] = a sum_k pre[k] g[n - k]
        q[v] = a * np.convolve(pre[v], g, mode="full")[C - 1:2 * C - 1]
    delta = geom.fov_cm / n
    cen = (np.arange(n) - (n - 1) / 2.0) * delta
    X, Y = np.meshgrid(cen, cen)            # X[i, j] = x_j, Y[i, j] = y_i
    dbeta = 2.0 * math.pi / V
    c_mid = (C - 1) / 2.0 - geom.channel_offset

    def back_views(v0, v1):
        img = np.zeros((n, n))
        for v in range(v0, v1):
            b = geom.view0_rad + 2.0 * math.pi * v / V
            sx, sy = D * math.cos(b), D * math.sin(b)
            ex, ey = -math.cos(b), -math.sin(b)            # central ray direction
            px, py = X - sx, Y - sy
            dot = px * ex + py * ey
            crs = ex * py - ey * px
            gp = np.arctan2(crs, dot)                       # angle of the pixel's ray
            L2 = px * px + py * py
            u = gp / a + c_mid                              # fractional channel index
            k0 = np.floor(u).astype(np.int64)
            f = u - k0
            val = np.zeros_like(u)
            for kk, wt in ((k0, 1.0 - f), (k0 + 1, f)):
                ok = (kk >= 0) & (kk < C)
                val[ok] += wt[ok] * q[v, kk[ok]]
            img += dbeta * val / L2
        return img

    threads = max(1, min(int(threads), V))
    if threads == 1:
        return back_views(0, V)
    import concurrent.futures as cf

    cuts = [V * t // threads for t in range(threads + 1)]
    with cf.ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(back_views, cuts[:-1], cuts[1:]))
    img = parts[0]
    for part in parts[1:]:
        img = img + part
    return img
