"""Python binding of the C-ABI library ``libmvct.so`` (argument marshalling only).

Every operator runs in the library's CUDA kernels; this module only checks
tensor shapes/dtypes/devices, passes raw device pointers and the current torch
CUDA stream through ctypes, and raises on a non-zero return code. There is no
CPU fallback: if the library is missing, importing this module raises.

Entry points mirror ``include/mvct.h``: :class:`Plan` wraps ``mvct_plan_create``
/ ``mvct_plan_destroy`` and exposes ``forward``, ``back``, ``tv_grad``,
``objective`` and ``recon``.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import torch

from .build import LIB as _LIB_PATH

MVCT_MAX_SUBSETS = 1024
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ELAUNCH", -5: "ETIMEOUT", -6: "EDATA"}


class MvctError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Geometry(ctypes.Structure):
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


class ReconState(ctypes.Structure):
    _fields_ = [
        ("n_done", ctypes.c_int64),
        ("lambda_", ctypes.c_double),
        ("phi_prev", ctypes.c_double),
        ("best_pass", ctypes.c_double),
        ("best_n", ctypes.c_int64),
        ("phi_ring", ctypes.c_double * MVCT_MAX_SUBSETS),
        ("pass_prev", ctypes.c_double),
    ]


class ReconOpts(ctypes.Structure):
    _fields_ = [
        ("lambda0", ctypes.c_double),
        ("dlambda_up", ctypes.c_double),
        ("dlambda_down", ctypes.c_double),
        ("lambda_min", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("tv_eps", ctypes.c_double),
        ("mu0", ctypes.c_double),
        ("init_from_input", ctypes.c_int32),
        ("d_best_out", ctypes.c_void_p),
        ("lambda_schedule", ctypes.POINTER(ctypes.c_double)),
        ("state", ctypes.POINTER(ReconState)),
        ("barrier_timeout_ms", ctypes.c_double),
        ("debug_unreachable_barrier", ctypes.c_int32),
        ("data_term", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("subset_order", ctypes.POINTER(ctypes.c_int32)),
        ("lambda_rule", ctypes.c_int32),
        ("psi_record", ctypes.POINTER(ctypes.c_double)),
    ]


# which square differences drive Eq. 4-5 under ordered subsets (mvct.h MVCT_LAMBDA_*)
LAMBDA_RULES = {"subset": 0, "pass": 1, "pass_sliding": 2}


class ReconStats(ctypes.Structure):
    _fields_ = [
        ("phi", ctypes.POINTER(ctypes.c_double)),
        ("lambda_", ctypes.POINTER(ctypes.c_double)),
        ("best_n", ctypes.c_int64),
        ("best_pass", ctypes.c_double),
        ("loop_ms", ctypes.c_double),
        ("setup_ms", ctypes.c_double),
        ("forward_ms", ctypes.c_double),
        ("back_ms", ctypes.c_double),
        ("grid_blocks", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
    ]


TUNE_MAX = 32


class TuneReport(ctypes.Structure):
    _fields_ = [
        ("groups", ctypes.c_int32),
        ("grid_blocks", ctypes.c_int32),
        ("ms_per_iter", ctypes.c_double),
        ("default_ms_per_iter", ctypes.c_double),
        ("n_candidates", ctypes.c_int32),
        ("cand_groups", ctypes.c_int32 * TUNE_MAX),
        ("cand_grid", ctypes.c_int32 * TUNE_MAX),
        ("cand_ms_per_iter", ctypes.c_double * TUNE_MAX),
    ]

    def to_dict(self) -> dict:
        k = self.n_candidates
        return dict(groups=self.groups, grid_blocks=self.grid_blocks, ms_per_iter=self.ms_per_iter,
                    default_ms_per_iter=self.default_ms_per_iter,
                    candidates=[dict(groups=self.cand_groups[i], grid_blocks=self.cand_grid[i],
                                     ms_per_iter=self.cand_ms_per_iter[i]) for i in range(k)])


EXPORTS = ["mvct_recon_opts_init", "mvct_plan_create", "mvct_plan_destroy", "mvct_forward",
           "mvct_back", "mvct_tv_grad", "mvct_objective", "mvct_objective_grad", "mvct_recon", "mvct_last_error",
           "mvct_tv_grad_noalloc", "mvct_batch_create", "mvct_batch_destroy", "mvct_batch_bind",
           "mvct_batch_run", "mvct_batch_stats", "mvct_fbp", "mvct_cnn_param_count", "mvct_cnn_create",
           "mvct_cnn_destroy", "mvct_cnn_get_params", "mvct_cnn_set_wait", "mvct_cnn_status", "mvct_cnn_forward", "mvct_cnn_grad", "mvct_cnn_train_step", "mvct_plan_tune", "mvct_batch_tune",
           "mvct_plan_set_shape", "mvct_phase_b_plan"]


def load_library(path: str = _LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libmvct.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.mvct_recon_opts_init.argtypes = [ctypes.POINTER(ReconOpts)]
    lib.mvct_recon_opts_init.restype = None
    lib.mvct_plan_create.argtypes = [ctypes.POINTER(Geometry), i32, ctypes.POINTER(vp)]
    lib.mvct_plan_destroy.argtypes = [vp]
    lib.mvct_plan_destroy.restype = None
    lib.mvct_forward.argtypes = [vp, vp, vp, i32, vp]
    lib.mvct_back.argtypes = [vp, vp, vp, i32, vp]
    lib.mvct_tv_grad.argtypes = [vp, vp, ctypes.c_double, vp, vp, vp]
    lib.mvct_objective.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, vp, vp]
    lib.mvct_objective_grad.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, vp, vp, vp]
    lib.mvct_recon.argtypes = [vp, vp, vp, ctypes.c_double, i32, ctypes.POINTER(ReconOpts), vp,
                               ctypes.POINTER(ReconStats), vp]
    lib.mvct_tv_grad_noalloc.argtypes = [vp, i32, ctypes.c_double, vp, vp, vp]
    lib.mvct_fbp.argtypes = [vp, vp, vp, vp]
    fp = ctypes.POINTER(ctypes.c_float)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.mvct_cnn_param_count.argtypes = []
    lib.mvct_cnn_param_count.restype = i32
    lib.mvct_cnn_create.argtypes = [i32, i32, i32, ctypes.c_double, fp, ctypes.POINTER(vp)]
    lib.mvct_cnn_destroy.argtypes = [vp]
    lib.mvct_cnn_destroy.restype = None
    lib.mvct_cnn_get_params.argtypes = [vp, fp]
    lib.mvct_cnn_set_wait.argtypes = [vp, ctypes.c_double, i32]
    lib.mvct_cnn_status.argtypes = [vp, vp]
    lib.mvct_cnn_forward.argtypes = [vp, vp, i32, vp, vp]
    lib.mvct_cnn_grad.argtypes = [vp, vp, vp, i32, vp, dp, vp]
    lib.mvct_cnn_train_step.argtypes = [vp, vp, vp, i32, ctypes.c_double, dp, vp]
    lib.mvct_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]
    lib.mvct_batch_destroy.argtypes = [vp]
    lib.mvct_batch_destroy.restype = None
    lib.mvct_batch_bind.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(vp), i32, ctypes.POINTER(ReconOpts)]
    lib.mvct_batch_run.argtypes = [vp, i32, vp]
    lib.mvct_batch_stats.argtypes = [vp, i32, ctypes.POINTER(ReconStats)]
    lib.mvct_plan_tune.argtypes = [vp, vp, vp, ctypes.c_double, i32, ctypes.POINTER(TuneReport), vp]
    lib.mvct_batch_tune.argtypes = [vp, i32, ctypes.POINTER(TuneReport), vp]
    lib.mvct_plan_set_shape.argtypes = [vp, i32, i32]
    lib.mvct_phase_b_plan.argtypes = [i32, i32, i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.mvct_last_error.restype = ctypes.c_char_p
    lib.mvct_last_error.argtypes = []
    return lib


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(rc: int):
    if rc != 0:
        raise MvctError(rc, lib().mvct_last_error().decode())


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _dev_f32(t: torch.Tensor, numel: int, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    if not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be contiguous with {numel} elements (got {tuple(t.shape)})")
    return ctypes.c_void_p(t.data_ptr())


def geometry(g) -> Geometry:
    """Accepts any object with the geometry fields (e.g. ``phantom.Geometry``)."""
    return Geometry(g.n, g.fov_cm, g.sad_cm, g.sdd_cm, g.n_views, g.n_channels, g.view0_rad,
                    g.fan_angle_rad, g.channel_offset)


STORAGE = {"f32": 0, "bf16": 1, "f16": 2}   # mvct_recon_opts.storage (MVCT_STORAGE_*)


def phase_b_plan(n_tiles: int, views_per_subset: int, groups_cap: int, grid: int, num_sms: int):
    """``mvct_phase_b_plan``: the balanced phase-B plan of the default one-slice
    launch shape, as an int32 array [grid][4] (tile, view group, view groups of
    the tile, first partial slot; tile -1: no item) and the reducer block, or
    None when the sizes do not allow it. Host arithmetic only (no GPU needed)."""
    items = np.zeros((grid, 4), dtype=np.int32)
    idle = ctypes.c_int32(-1)
    rc = lib().mvct_phase_b_plan(n_tiles, views_per_subset, groups_cap, grid, num_sms,
                                 items.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(idle))
    if rc < 0:
        raise MvctError(rc, lib().mvct_last_error().decode())
    return (items, idle.value) if rc == 1 else None


def spread_order(S: int) -> List[int]:
    """A subset visiting order for mvct_recon_opts.subset_order that keeps
    consecutive subsets far apart in angle: starting at 0, the next subset is the
    unused one farthest (circularly, in units of the view step) from the last two
    picks, then from all picks so far, then the smallest index. For S = 20:
    0, 10, 5, 17, 11, 4, 18, ... (consecutive subsets 6-10 view steps apart). The
    paper's order is 0, 1, ..., S-1."""
    order, used = [0], {0}
    cd = lambda a, b: min(abs(a - b), S - abs(a - b))
    while len(order) < S:
        key, best = None, None
        for s in range(S):
            if s in used:
                continue
            k = (min(cd(s, u) for u in order[-2:]), min(cd(s, u) for u in used), -s)
            if key is None or k > key:
                key, best = k, s
        order.append(best)
        used.add(best)
    return order


@dataclass
class ReconResult:
    phi: np.ndarray
    lam: np.ndarray
    best_n: int
    best_pass: float
    loop_ms: float
    setup_ms: float
    grid_blocks: int
    forward_ms: float = 0.0
    back_ms: float = 0.0
    psi: Optional[np.ndarray] = None   # Psi after every pass (psi_record=True)


class Plan:
    """A reconstruction plan for one geometry and subset count (``mvct_plan_create``)."""

    def __init__(self, geom, n_subsets: int):
        self.geom = geom
        self.n = geom.n
        self.V, self.C, self.S = geom.n_views, geom.n_channels, n_subsets
        self._g = geometry(geom)
        h = ctypes.c_void_p()
        _check(lib().mvct_plan_create(ctypes.byref(self._g), n_subsets, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mvct_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def rows(self, subset: int) -> int:
        return self.V if subset < 0 else self.V // self.S

    def forward(self, img: torch.Tensor, subset: int = -1, out: Optional[torch.Tensor] = None,
                stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.rows(subset), self.C), device=img.device, dtype=torch.float32)
        _check(lib().mvct_forward(self._h, _dev_f32(img, self.n * self.n, "img"),
                                  _dev_f32(out, self.rows(subset) * self.C, "out"), subset,
                                  ctypes.c_void_p(_stream(stream))))
        return out

    def back(self, sino: torch.Tensor, subset: int = -1, out: Optional[torch.Tensor] = None,
             stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.n, self.n), device=sino.device, dtype=torch.float32)
        _check(lib().mvct_back(self._h, _dev_f32(sino, self.rows(subset) * self.C, "sino"),
                               _dev_f32(out, self.n * self.n, "out"), subset,
                               ctypes.c_void_p(_stream(stream))))
        return out

    def fbp(self, sino: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """``mvct_fbp``: fan-beam filtered backprojection of all views."""
        if out is None:
            out = torch.empty((self.n, self.n), device=sino.device, dtype=torch.float32)
        _check(lib().mvct_fbp(self._h, _dev_f32(sino, self.V * self.C, "sino"), _dev_f32(out, self.n * self.n, "out"),
                              ctypes.c_void_p(_stream(stream))))
        return out

    def tv_grad(self, img: torch.Tensor, eps: float, with_value: bool = True, stream=None):
        grad = torch.empty((self.n, self.n), device=img.device, dtype=torch.float32)
        val = torch.zeros(1, device=img.device, dtype=torch.float64) if with_value else None
        _check(lib().mvct_tv_grad(self._h, _dev_f32(img, self.n * self.n, "img"), eps,
                                  _dev_f32(grad, self.n * self.n, "grad"),
                                  ctypes.c_void_p(val.data_ptr()) if val is not None else None,
                                  ctypes.c_void_p(_stream(stream))))
        return grad, val

    def objective(self, img, p, w, beta: float, eps: float, stream=None) -> torch.Tensor:
        out = torch.zeros(1, device=img.device, dtype=torch.float64)
        R = self.V * self.C
        _check(lib().mvct_objective(self._h, _dev_f32(img, self.n * self.n, "img"), _dev_f32(p, R, "p"),
                                    _dev_f32(w, R, "w"), beta, eps, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(_stream(stream))))
        return out

    def objective_grad(self, img, p, w, beta: float, eps: float, out: Optional[torch.Tensor] = None,
                       with_value: bool = False, stream=None):
        """``mvct_objective_grad``: the gradient of Psi at img (and Psi if with_value)."""
        out = torch.empty((self.n, self.n), device=img.device, dtype=torch.float32) if out is None else out
        val = torch.zeros(1, device=img.device, dtype=torch.float64) if with_value else None
        R = self.V * self.C
        _check(lib().mvct_objective_grad(self._h, _dev_f32(img, self.n * self.n, "img"), _dev_f32(p, R, "p"),
                                         _dev_f32(w, R, "w"), beta, eps, _dev_f32(out, self.n * self.n, "out"),
                                         ctypes.c_void_p(val.data_ptr()) if val is not None else None,
                                         ctypes.c_void_p(_stream(stream))))
        return (out, val) if with_value else out

    def recon(self, p: torch.Tensor, w: torch.Tensor, beta: float, n_iter: int,
              img: Optional[torch.Tensor] = None, init_from_input: bool = False,
              best_out: Optional[torch.Tensor] = None, lambda_schedule=None,
              state: Optional[ReconState] = None, stream=None, psi_record: bool = False, **opts):
        """Run ``mvct_recon``; returns (image tensor, ReconResult). psi_record: also
        return Psi of the iterate after every pass (ReconResult.psi)."""
        R = self.V * self.C
        if img is None:
            img = torch.zeros((self.n, self.n), device=p.device, dtype=torch.float32)
        o = ReconOpts()
        lib().mvct_recon_opts_init(ctypes.byref(o))
        if isinstance(opts.get("storage"), str):
            opts = dict(opts, storage=STORAGE[opts["storage"]])
        if isinstance(opts.get("lambda_rule"), str):
            opts = dict(opts, lambda_rule=LAMBDA_RULES[opts["lambda_rule"]])
        order = None
        if opts.get("subset_order") is not None:
            order = np.ascontiguousarray(opts["subset_order"], dtype=np.int32)
            opts = dict(opts, subset_order=order.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        o.init_from_input = 1 if init_from_input else 0
        if best_out is not None:
            o.d_best_out = ctypes.c_void_p(_dev_f32(best_out, self.n * self.n, "best_out").value)
        sched = None
        if lambda_schedule is not None:
            sched = np.ascontiguousarray(lambda_schedule, dtype=np.float64)
            if sched.size < n_iter:
                raise ValueError("lambda_schedule shorter than n_iter")
            o.lambda_schedule = sched.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if state is not None:
            o.state = ctypes.pointer(state)
        psi = None
        if psi_record:
            psi = np.full(n_iter // self.S + 1, np.nan)
            o.psi_record = psi.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        phi = np.zeros(max(n_iter, 1))
        lam = np.zeros(max(n_iter, 1))
        st = ReconStats()
        st.phi = phi.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        st.lambda_ = lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib().mvct_recon(self._h, _dev_f32(p, R, "p"), _dev_f32(w, R, "w"), beta, n_iter,
                                ctypes.byref(o), _dev_f32(img, self.n * self.n, "img"),
                                ctypes.byref(st), ctypes.c_void_p(_stream(stream))))
        return img, ReconResult(phi[:n_iter], lam[:n_iter], st.best_n, st.best_pass, st.loop_ms,
                                st.setup_ms, st.grid_blocks, st.forward_ms, st.back_ms, psi)


def _plan_tune(self, p: torch.Tensor, w: torch.Tensor, beta: float, n_iter_probe: int = 40, stream=None) -> dict:
    """``mvct_plan_tune``: time the loop's launch-shape candidates on (p, w) and
    keep the fastest for this plan; returns the report as a dict (groups 0 = the
    default rule, i.e. the balanced phase-B plan where the sizes allow it)."""
    R = self.V * self.C
    rep = TuneReport()
    _check(lib().mvct_plan_tune(self._h, _dev_f32(p, R, "p"), _dev_f32(w, R, "w"), beta, n_iter_probe,
                                ctypes.byref(rep), ctypes.c_void_p(_stream(stream))))
    return rep.to_dict()


def _plan_set_shape(self, groups: int = 0, grid_blocks: int = 0) -> None:
    """``mvct_plan_set_shape``: fix the loop's launch shape. groups = view groups
    per tile (0: the default rule, the balanced plan where the sizes allow it;
    > 0: every tile split into that many groups), grid_blocks = blocks of the
    launch (0: every co-resident block)."""
    _check(lib().mvct_plan_set_shape(self._h, groups, grid_blocks))


Plan.tune = _plan_tune
Plan.set_shape = _plan_set_shape


def tv_grad_noalloc(img: torch.Tensor, eps: float, grad: torch.Tensor, tv: Optional[torch.Tensor] = None,
                    stream=None) -> None:
    """``mvct_tv_grad_noalloc``: TV gradient (and value) into caller-provided
    tensors; the library allocates nothing."""
    n = img.shape[-1]
    if tv is not None and (not tv.is_cuda or tv.dtype != torch.float64 or tv.numel() < 1):
        raise TypeError("tv must be a CUDA float64 tensor")
    _check(lib().mvct_tv_grad_noalloc(_dev_f32(img, n * n, "img"), n, eps, _dev_f32(grad, n * n, "grad"),
                                      ctypes.c_void_p(tv.data_ptr()) if tv is not None else None,
                                      ctypes.c_void_p(_stream(stream))))


class Batch:
    """Many slices in one persistent launch (``mvct_batch_*``).

    ``plans``: distinct :class:`Plan` objects (one per slice). ``bind`` keeps the
    tensors alive; ``run`` only enqueues work on the stream (CUDA-graph
    capturable); ``stats`` waits for it.
    """

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib().mvct_batch_create(arr, len(self.plans), ctypes.byref(h)))
        self._h = h
        self._keep = None
        self.max_iter = 0
        self.last_n_iter = 0

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mvct_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def bind(self, sinos, weights, betas, imgs, max_iter: int, init_from_input: bool = False, **opts):
        m = len(self.plans)
        assert len(sinos) == len(weights) == len(betas) == len(imgs) == m
        ptr = lambda ts, nm, sizes: (ctypes.c_void_p * m)(*[_dev_f32(t, k, nm).value for t, k in zip(ts, sizes)])
        R = [p.V * p.C for p in self.plans]
        N = [p.n * p.n for p in self.plans]
        o = ReconOpts()
        lib().mvct_recon_opts_init(ctypes.byref(o))
        if isinstance(opts.get("lambda_rule"), str):
            opts = dict(opts, lambda_rule=LAMBDA_RULES[opts["lambda_rule"]])
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        o.init_from_input = 1 if init_from_input else 0
        b = (ctypes.c_double * m)(*[float(x) for x in betas])
        _check(lib().mvct_batch_bind(self._h, ptr(sinos, "p", R), ptr(weights, "w", R), b, ptr(imgs, "img", N),
                                     max_iter, ctypes.byref(o)))
        self._keep = (list(sinos), list(weights), list(imgs))
        self.max_iter = max_iter

    def run(self, n_iter: int, stream=None):
        _check(lib().mvct_batch_run(self._h, n_iter, ctypes.c_void_p(_stream(stream))))
        self.last_n_iter = n_iter

    def tune(self, n_iter_probe: int = 40, stream=None) -> dict:
        """``mvct_batch_tune``: time the view-group candidates on the bound data
        (bound images restored afterwards) and keep the fastest."""
        rep = TuneReport()
        _check(lib().mvct_batch_tune(self._h, n_iter_probe, ctypes.byref(rep), ctypes.c_void_p(_stream(stream))))
        return rep.to_dict()

    def stats(self, i: int, n_iter: Optional[int] = None) -> ReconResult:
        """Statistics of slice i of the last run (its n_iter sub-iterations)."""
        if n_iter is not None and n_iter != self.last_n_iter:
            raise ValueError(f"the last run had {self.last_n_iter} sub-iterations, not {n_iter}")
        n_iter = self.last_n_iter
        phi = np.zeros(max(n_iter, 1))
        lam = np.zeros(max(n_iter, 1))
        st = ReconStats()
        st.phi = phi.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        st.lambda_ = lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib().mvct_batch_stats(self._h, i, ctypes.byref(st)))
        return ReconResult(phi[:n_iter], lam[:n_iter], st.best_n, st.best_pass, st.loop_ms, st.setup_ms,
                           st.grid_blocks)


def fresh_state() -> ReconState:
    s = ReconState()
    s.n_done = 0
    s.best_pass = math.inf
    s.best_n = -1
    return s
