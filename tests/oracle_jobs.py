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
