"""Seeded synthetic inputs for the fan-beam MVCT OS-TV reconstruction.

This module is the one input generator that both the FP64 CPU oracle (``oracle/``)
and the CUDA path consume. It simulates the *measurement*, not the reconstruction:
analytic line integrals of ellipse phantoms along the scanner's fan-beam rays,
Poisson photon counts, and their log transform into projections ``p`` and
per-ray statistical weights ``w``. It holds none of the reconstruction's
arithmetic (no Joseph projector, no backprojector, no TV, no update rule).

The scanner model is the one the paper reconstructs (Sec. 3.1 and 3.4: one
512x512 slice, 800 views per rotation): a point source on a circle of radius
``sad_cm`` around the isocentre, an equiangular (arc) detector, views uniform
over 2*pi. The paper's Gammex, Cheese-phantom and patient data are not
available; these seeded ellipse phantoms with Poisson noise stand in for them.

Geometry conventions (shared by definition, implemented independently by each
consumer):

* pixel centre x_j = (j - (n-1)/2) * delta, y_i = (i - (n-1)/2) * delta,
  delta = fov_cm / n; image arrays are row-major ``[i][j]`` (row = y).
* view v: beta_v = view0_rad + 2*pi*v/V, source S_v = sad*(cos beta_v, sin beta_v).
* channel c: gamma_c = (c - (C-1)/2 + channel_offset) * fan/C.
* ray direction d = Rot(gamma_c) (-cos beta_v, -sin beta_v).
* sinograms are view-major ``[V][C]``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np

WATER_MU = 0.07      # /cm, attenuation of the water disk (Sec. 4.2 quotes ~0.07 /cm for water)
WATER_RADIUS = 15.0  # cm


@dataclass(frozen=True)
class Geometry:
    """Fan-beam scanner and image grid (all lengths in cm, angles in rad)."""

    n: int
    n_views: int
    n_channels: int
    fov_cm: float = 40.0
    sad_cm: float = 85.0
    sdd_cm: float = 145.0
    view0_rad: float = 0.0
    fan_angle_rad: float = 0.0   # <= 0 selects 2*asin((fov/2)/sad)
    channel_offset: float = 0.0  # in channels

    @property
    def delta(self) -> float:
        return self.fov_cm / self.n

    @property
    def fan(self) -> float:
        if self.fan_angle_rad > 0:
            return self.fan_angle_rad
        return 2.0 * math.asin((self.fov_cm / 2.0) / self.sad_cm)


def rays(geom: Geometry):
    """Source points and unit directions of every ray, arrays of shape [V][C]."""
    v = np.arange(geom.n_views, dtype=np.float64)
    c = np.arange(geom.n_channels, dtype=np.float64)
    beta = geom.view0_rad + 2.0 * math.pi * v / geom.n_views
    gamma = (c - (geom.n_channels - 1) / 2.0 + geom.channel_offset) * (geom.fan / geom.n_channels)
    bx, by = -np.cos(beta)[:, None], -np.sin(beta)[:, None]
    cg, sg = np.cos(gamma)[None, :], np.sin(gamma)[None, :]
    dx = cg * bx - sg * by
    dy = sg * bx + cg * by
    sx = np.broadcast_to(geom.sad_cm * np.cos(beta)[:, None], dx.shape)
    sy = np.broadcast_to(geom.sad_cm * np.sin(beta)[:, None], dx.shape)
    return sx, sy, dx, dy


@dataclass(frozen=True)
class Ellipse:
    """An ellipse that ADDS ``delta`` (1/cm) to the attenuation inside it."""

    cx: float
    cy: float
    a: float
    b: float
    phi: float
    delta: float


def chord_lengths(e: Ellipse, sx, sy, dx, dy) -> np.ndarray:
    """Exact length of each ray's intersection with ellipse ``e`` (rays are lines)."""
    c, s = math.cos(e.phi), math.sin(e.phi)
    px, py = sx - e.cx, sy - e.cy
    # rotate into the ellipse frame, then scale to the unit circle
    qx, qy = (c * px + s * py) / e.a, (-s * px + c * py) / e.b
    ux, uy = (c * dx + s * dy) / e.a, (-s * dx + c * dy) / e.b
    A = ux * ux + uy * uy
    B = qx * ux + qy * uy
    C0 = qx * qx + qy * qy - 1.0
    disc = B * B - A * C0
    return np.where(disc > 0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / A, 0.0)


def analytic_sinogram(geom: Geometry, ellipses: Sequence[Ellipse]) -> np.ndarray:
    """Line integrals of the phantom along every ray, FP64 ``[V][C]``."""
    sx, sy, dx, dy = rays(geom)
    out = np.zeros(dx.shape, dtype=np.float64)
    for e in ellipses:
        out += e.delta * chord_lengths(e, sx, sy, dx, dy)
    return out


def rasterize(ellipses: Sequence[Ellipse], n: int, fov_cm: float, supersample: int = 4) -> np.ndarray:
    """Pixel-average image ``[n][n]`` (FP64) by ``supersample``^2 sub-samples per pixel."""
    delta = fov_cm / n
    centres = (np.arange(n) - (n - 1) / 2.0) * delta
    offs = ((np.arange(supersample) + 0.5) / supersample - 0.5) * delta
    img = np.zeros((n, n), dtype=np.float64)
    for oy in offs:
        y = (centres + oy)[:, None]
        for ox in offs:
            x = (centres + ox)[None, :]
            for e in ellipses:
                c, s = math.cos(e.phi), math.sin(e.phi)
                xr, yr = x - e.cx, y - e.cy
                u = (c * xr + s * yr) / e.a
                v = (-s * xr + c * yr) / e.b
                img += e.delta * (u * u + v * v <= 1.0)
    return img / (supersample * supersample)


def _place(rng, radii_fn, values, max_centre_r, existing: List[tuple], tries=10000):
    """Rejection-sample non-overlapping ellipses fully inside the water disk."""
    out = []
    for val in values:
        for _ in range(tries):
            a, b = radii_fn()
            rmax = max(a, b)
            r = max_centre_r * math.sqrt(rng.uniform())
            t = rng.uniform(0, 2 * math.pi)
            cx, cy = r * math.cos(t), r * math.sin(t)
            if math.hypot(cx, cy) + rmax > WATER_RADIUS - 0.2:
                continue
            if any(math.hypot(cx - ox, cy - oy) <= rmax + orr + 0.1 for ox, oy, orr in existing):
                continue
            existing.append((cx, cy, rmax))
            out.append(Ellipse(cx, cy, a, b, rng.uniform(0, math.pi), val - WATER_MU))
            break
    return out


def water_disk() -> Ellipse:
    return Ellipse(0.0, 0.0, WATER_RADIUS, WATER_RADIUS, 0.0, WATER_MU)


def phantom_random_ellipses(seed: int) -> List[Ellipse]:
    """Water disk with 2-8 random ellipses of attenuation U[0, 0.10] /cm replacing water."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = int(rng.integers(2, 9))
    vals = rng.uniform(0.0, 0.10, size=k)
    ell = _place(rng, lambda: (rng.uniform(0.5, 4.0), rng.uniform(0.5, 4.0)), vals, 12.0, [])
    return [water_disk()] + ell


def phantom_inserts_and_rods(seed: int) -> List[Ellipse]:
    """Water disk with 7 low-contrast inserts (0.5-3 % of water, radius 2-15 mm)
    and 4 high-contrast rods (0.10-0.20 /cm, radius 3-10 mm)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    existing: List[tuple] = []
    low = [WATER_MU * (1.0 + rng.choice([-1.0, 1.0]) * rng.uniform(0.005, 0.03)) for _ in range(7)]
    def circ(lo, hi):
        def f():
            r = rng.uniform(lo, hi)
            return r, r
        return f
    ell = _place(rng, circ(0.2, 1.5), low, 12.0, existing)
    rods = list(rng.uniform(0.10, 0.20, size=4))
    ell += _place(rng, circ(0.3, 1.0), rods, 12.0, existing)
    return [water_disk()] + ell


def poisson_data(line_integrals: np.ndarray, I0: float, rng) -> tuple:
    """Poisson counts y ~ P(I0 exp(-l)); p = ln(I0/max(y,1)), w = max(y,1)/I0 (FP32)."""
    y = rng.poisson(I0 * np.exp(-line_integrals)).astype(np.float64)
    y1 = np.maximum(y, 1.0)
    p = np.log(I0 / y1)
    w = y1 / I0
    return p.astype(np.float32), w.astype(np.float32)


@dataclass
class Case:
    """One slice's reconstruction problem: geometry, data and method settings."""

    name: str
    geom: Geometry
    n_subsets: int
    n_iter: int
    beta: float
    tv_eps: float
    I0: float
    p: np.ndarray            # float32 [V][C] log projections
    w: np.ndarray            # float32 [V][C] statistical weights
    ellipses: List[Ellipse] = field(default_factory=list)
    seed: int = 0

    def truth(self, supersample: int = 4) -> np.ndarray:
        return rasterize(self.ellipses, self.geom.n, self.geom.fov_cm, supersample)


GEOM_128 = Geometry(n=128, n_views=200, n_channels=184)
GEOM_512 = Geometry(n=512, n_views=800, n_channels=738)
GEOM_384 = Geometry(n=384, n_views=600, n_channels=552)
GEOM_256 = Geometry(n=256, n_views=400, n_channels=368)


def make_case(kind: str, seed: int, geom: Optional[Geometry] = None, I0: Optional[float] = None,
              beta: Optional[float] = None, n_iter: Optional[int] = None,
              n_subsets: Optional[int] = None, noise: bool = True) -> Case:
    """Build a seeded case.

    kind ``"small"``: 128^2 over 40 cm, 200 views, 184 channels, 2-8 random
    ellipses, I0 = 1e4, 10 subsets, 20 sub-iterations, beta = 1e-3, eps = 1e-6.
    kind ``"full"``: 512^2, 800 views, 738 channels, 7 low-contrast inserts and
    4 rods, I0 = 5e3, 20 subsets, 500 sub-iterations, beta = 1e-3, eps = 1e-6.
    """
    if kind == "small":
        g, ell = GEOM_128, phantom_random_ellipses(seed)
        d = dict(I0=1e4, beta=1e-3, n_iter=20, n_subsets=10)
    elif kind == "full":
        g, ell = GEOM_512, phantom_inserts_and_rods(seed)
        d = dict(I0=5e3, beta=1e-3, n_iter=500, n_subsets=20)
    else:
        raise ValueError(kind)
    if geom is not None:
        g = geom
    I0 = d["I0"] if I0 is None else I0
    beta = d["beta"] if beta is None else beta
    n_iter = d["n_iter"] if n_iter is None else n_iter
    n_subsets = d["n_subsets"] if n_subsets is None else n_subsets
    li = analytic_sinogram(g, ell)
    rng = np.random.Generator(np.random.PCG64(10_000 + seed))
    if noise:
        p, w = poisson_data(li, I0, rng)
    else:
        p = li.astype(np.float32)
        w = np.exp(-li).astype(np.float32)
    return Case(kind, g, n_subsets, n_iter, beta, 1e-6, I0, p, w, ell, seed)


# Uneven helical-stack batch: 48 x (512^2, 800 views, 738 ch), 32 x (384^2, 600, 552),
# 16 x (256^2, 400, 368), each with its own phantom seed and I0 log-uniform in [2e3, 2e4].
BATCH_GROUPS = ((48, GEOM_512), (32, GEOM_384), (16, GEOM_256))


def make_batch(seed0: int = 1000, groups=BATCH_GROUPS, n_iter: int = 500, n_subsets: int = 20,
               beta: float = 1e-3) -> List[Case]:
    cases = []
    k = 0
    for count, g in groups:
        for _ in range(count):
            rng = np.random.Generator(np.random.PCG64(seed0 + k))
            I0 = float(math.exp(rng.uniform(math.log(2e3), math.log(2e4))))
            cases.append(make_case("full", seed0 + k, geom=g, I0=I0, beta=beta, n_iter=n_iter,
                                   n_subsets=n_subsets))
            k += 1
    return cases
