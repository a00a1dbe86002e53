"""Oracle runs executed in spawned worker processes by the full-size GPU tests.

Each job regenerates its seeded input (so nothing large is pickled in) and runs
the FP64 oracle; workers are started with the "spawn" method, never forked
from a process that already initialised CUDA.
"""
import numpy as np

import oracle
from paper_1903_10088_gb300 import phantom as ph


def full_case_recon(seed: int, beta: float, n_iter: int):
    c = ph.make_case("full", seed, beta=beta, n_iter=n_iter)
    r = oracle.recon(c.geom, c.n_subsets, c.p, c.w, beta, n_iter)
    return r["image"].astype(np.float64), r["phi"], r["lam"]


def full_case_objective(seed: int, img):
    """FP64 oracle objective of an image for the seeded full-size case."""
    c = ph.make_case("full", seed)
    return oracle.objective(c.geom, np.asarray(img, dtype=np.float64), c.p, c.w, c.beta, c.tv_eps)


def case_and_truth(seed: int, kind: str = "full"):
    c = ph.make_case(kind, seed)
    return c, c.truth(2)


def full_case_recon_checkpoints(seed: int, beta: float, checkpoints):
    """Oracle images and lambda sequences after each of `checkpoints` sub-iterations
    (separate runs from the same start)."""
    c = ph.make_case("full", seed, beta=beta)
    out = {}
    for n in checkpoints:
        r = oracle.recon(c.geom, c.n_subsets, c.p, c.w, beta, n)
        out[n] = (r["image"].astype(np.float64), r["lam"])
    return out


def fbp_start(c):
    """The plain form's start image: the oracle's FBP of the case, rounded to FP32
    (the same host array is handed to the oracle and to the GPU)."""
    from oracle import fbp as F

    return F.fbp(c.geom, c.p.astype(np.float64)).astype(np.float32)


def full_case_recon_from(seed: int, beta: float, n_iter: int, start):
    """Oracle reconstruction of the seeded full-size case from a given start image."""
    c = ph.make_case("full", seed, beta=beta, n_iter=n_iter)
    r = oracle.recon(c.geom, c.n_subsets, c.p, c.w, beta, n_iter, init=np.asarray(start, dtype=np.float64))
    return r["image"].astype(np.float64), r["phi"], r["lam"]


def case_recon_from(seed: int, geom, beta: float, n_iter: int, start, lambda0: float):
    """Oracle reconstruction of a seeded full-kind case on `geom` from a start image
    with the given lambda0."""
    c = ph.make_case("full", seed, geom=geom, beta=beta, n_iter=n_iter)
    r = oracle.recon(c.geom, c.n_subsets, c.p, c.w, beta, n_iter, init=np.asarray(start, dtype=np.float64),
                     lambda0=lambda0)
    return r["image"].astype(np.float64), r["phi"], r["lam"]
