"""FP64 CPU oracle for the OS-TV MVCT reconstruction (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package. It compiles ``mvct_oracle.c`` (plain C, gcc) into a
shared library and exposes it through ctypes with numpy FP64 arrays. It shares
no code with the CUDA library in ``paper_1903_10088_gb300``.

What pins each function is listed in ``mvct_oracle.c``; parity of the adaptive
lambda dynamics against the paper's own data is unpinned (the paper prints no
worked example), and so is the absolute scale of the paper's alpha.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mvct_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OracleGeometry(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("fov_cm", ctypes.c_double),
        ("sad_cm", ctypes.c_double),
        ("sdd_cm", ctypes.c_double),
        ("n_views", ctypes.c_int32),
        ("n_channels", ctypes.c_int32),
        ("view0_rad", ctypes.c_double),
        ("fan_angle_rad", ctypes.c_double),
        ("channel_offset", ctypes.c_double),
    ]


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("lambda0", ctypes.c_double),
        ("dlambda_up", ctypes.c_double),
        ("dlambda_down", ctypes.c_double),
        ("lambda_min", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("tv_eps", ctypes.c_double),
        ("mu0", ctypes.c_double),
        ("init_from_input", ctypes.c_int32),
        ("data_term", ctypes.c_int32),
        ("subset_order", ctypes.POINTER(ctypes.c_int32)),
        ("lambda_rule", ctypes.c_int32),
    ]


# which square difference drives Eq. 4-5 (see oracle_recon in mvct_oracle.c)
LAMBDA_RULES = {"subset": 0, "pass": 1, "pass_sliding": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C99, no arch-specific flags), with
    OpenMP if the compiler has it (used only when set_threads() asks for it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base + ["-fopenmp"], capture_output=True)
        if r.returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            G = ctypes.POINTER(OracleGeometry)
            lib.oracle_forward.argtypes = [G, dp, ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_back.argtypes = [G, dp, ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_tv.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp]
            lib.oracle_tv.restype = ctypes.c_double
            lib.oracle_objective.argtypes = [G, dp, dp, dp, ctypes.c_double, ctypes.c_double]
            lib.oracle_objective.restype = ctypes.c_double
            lib.oracle_setup.argtypes = [G, dp, ctypes.c_double, ctypes.c_double, dp,
                                         ctypes.POINTER(ctypes.c_ubyte)]
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = ctypes.c_int
            lib.oracle_recon.argtypes = [G, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(OracleParams), dp, dp, dp, dp, dp,
                                         ctypes.POINTER(ctypes.c_int), dp]
            _lib = lib
    return _lib


def set_threads(threads: int) -> int:
    """Threads for the reprojection (rays) and the transpose (views); results are
    bit-identical for any count. Returns the count in effect (1 without OpenMP)."""
    return _load().oracle_set_threads(int(threads))


def _geom(g) -> OracleGeometry:
    return OracleGeometry(g.n, g.fov_cm, g.sad_cm, g.sdd_cm, g.n_views, g.n_channels,
                          g.view0_rad, g.fan_angle_rad, g.channel_offset)


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _rows(g, subset, n_subsets):
    return g.n_views if subset < 0 else g.n_views // n_subsets


def forward(g, img, subset: int = -1, n_subsets: int = 1) -> np.ndarray:
    """A img for all views (subset=-1) or the rows v = subset + k*S."""
    img = _f64(img).reshape(g.n, g.n)
    out = np.zeros((_rows(g, subset, n_subsets), g.n_channels), dtype=np.float64)
    if _load().oracle_forward(ctypes.byref(_geom(g)), _dp(img), subset, n_subsets, _dp(out)):
        raise ValueError("oracle_forward: invalid arguments")
    return out


def back(g, sino, subset: int = -1, n_subsets: int = 1) -> np.ndarray:
    """A^T sino over the same rays as :func:`forward`."""
    sino = _f64(sino).reshape(_rows(g, subset, n_subsets), g.n_channels)
    out = np.zeros((g.n, g.n), dtype=np.float64)
    if _load().oracle_back(ctypes.byref(_geom(g)), _dp(sino), subset, n_subsets, _dp(out)):
        raise ValueError("oracle_back: invalid arguments")
    return out


def tv(img, eps: float, with_grad: bool = True):
    """(TV_eps(img), grad TV_eps(img) or None)."""
    img = _f64(img)
    n = img.shape[0]
    grad = np.zeros_like(img) if with_grad else None
    val = _load().oracle_tv(n, _dp(img), eps, _dp(grad))
    return val, grad


def objective(g, img, p, w, beta: float, eps: float) -> float:
    """Weighted-least-squares objective Psi (see oracle_objective)."""
    return _load().oracle_objective(ctypes.byref(_geom(g)), _dp(_f64(img)), _dp(_f64(p)),
                                    _dp(_f64(w)), beta, eps)


def poisson_objective(g, img, w, beta: float, eps: float) -> float:
    """sum_i (w_i q_i + exp(-q_i)) + beta TV_eps: the negative Poisson log-likelihood
    divided by I0 (counts y = I0 w, up to a constant), q = A img, plus the prior."""
    q = forward(g, img)
    wv = _f64(w).reshape(q.shape)
    return float(np.sum(wv * q + np.exp(-q)) + beta * tv(img, eps, False)[0])


def setup(g, w, beta: float, eps: float):
    """(D, M): surrogate diagonal and support mask of the loop's set-up step."""
    D = np.zeros((g.n, g.n), dtype=np.float64)
    M = np.zeros((g.n, g.n), dtype=np.uint8)
    rc = _load().oracle_setup(ctypes.byref(_geom(g)), _dp(_f64(w)), beta, eps, _dp(D),
                              M.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    if rc:
        raise ValueError("oracle_setup failed")
    return D, M.astype(bool)


DEFAULTS = dict(lambda0=0.01, dlambda_up=1e-4, dlambda_down=2e-4, lambda_min=1e-4, kappa=50.0,
                tv_eps=1e-6, mu0=0.05, data_term=0, lambda_rule="pass_sliding")


def recon(g, n_subsets: int, p, w, beta: float, n_iter: int, init=None, lambda_schedule=None,
          want_best: bool = False, subset_order=None, **params):
    """Run the OS-TV loop; returns dict(image, phi, lam, best_n, best_pass, best_image).
    subset_order: a permutation of 0..S-1 visited cyclically (default 0, 1, ..., S-1).
    lambda_rule: "subset", "pass" or "pass_sliding" (which square differences Eq. 4-5
    compare; see oracle_recon in mvct_oracle.c)."""
    prm = dict(DEFAULTS)
    prm.update(params)
    order = None
    if subset_order is not None:
        order = np.ascontiguousarray(subset_order, dtype=np.int32)
        if sorted(order.tolist()) != list(range(n_subsets)):
            raise ValueError("subset_order must be a permutation of 0..S-1")
    op = OracleParams(prm["lambda0"], prm["dlambda_up"], prm["dlambda_down"], prm["lambda_min"],
                      prm["kappa"], prm["tv_eps"], prm["mu0"], 1 if init is not None else 0, prm["data_term"],
                      order.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if order is not None else None,
                      LAMBDA_RULES[prm["lambda_rule"]])
    img = np.zeros((g.n, g.n)) if init is None else _f64(init).reshape(g.n, g.n).copy()
    phi = np.zeros(max(n_iter, 1))
    lam = np.zeros(max(n_iter, 1))
    best = np.zeros((g.n, g.n)) if want_best else None
    sched = None if lambda_schedule is None else _f64(lambda_schedule)
    bn = ctypes.c_int(-1)
    bp = ctypes.c_double(0.0)
    rc = _load().oracle_recon(ctypes.byref(_geom(g)), n_subsets, _dp(_f64(p)), _dp(_f64(w)), beta,
                              n_iter, ctypes.byref(op), _dp(sched), _dp(img), _dp(best), _dp(phi),
                              _dp(lam), ctypes.byref(bn), ctypes.byref(bp))
    if rc:
        raise ValueError(f"oracle_recon failed ({rc})")
    return dict(image=img, phi=phi[:n_iter], lam=lam[:n_iter], best_n=bn.value,
                best_pass=bp.value, best_image=best)
