"""Learned warm start for the OS-TV loop (binding and training pipeline).

The network (``mvct_cnn_*`` in the C ABI) maps an FBP image to a start image for
``mvct_recon`` / ``mvct_batch``: 8 conv3x3 layers, 32 channels, ReLU, residual
output, BF16 weights and activations with FP32 accumulation, trained with Adam
on (FBP image, converged OS-TV image) pairs that the reconstruction itself
produces from seeded synthetic phantoms. The paper motivates the start image's
role (Sec. 3.3.2 and 4.2: mu^(0) changes the convergence speed); the network
itself is this project's addition.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional

import numpy as np

CH = 32
PARAM_COUNT = 9 * CH + CH + 6 * (9 * CH * CH + CH) + 9 * CH + 1
SCALE = 10.0   # images are multiplied by this inside the network (water ~ 0.7)


def param_count() -> int:
    return PARAM_COUNT


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases; the last layer starts small so that the
    residual network starts close to the identity (out ~ FBP)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.normal(0, np.sqrt(2.0 / 9), 9 * CH), np.zeros(CH)]
    for _ in range(6):
        parts += [rng.normal(0, np.sqrt(2.0 / (9 * CH)), 9 * CH * CH), np.zeros(CH)]
    parts += [rng.normal(0, 1e-3, 9 * CH), np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == PARAM_COUNT
    return p


class CNN:
    """The warm-start network on the current CUDA device (``mvct_cnn_*``)."""

    def __init__(self, batch_max: int, h: int, w: int, params: np.ndarray, scale: float = SCALE):
        from . import mvct

        self._m = mvct
        lib = mvct.lib()
        if lib.mvct_cnn_param_count() != PARAM_COUNT:
            raise RuntimeError("parameter layout of the library does not match the binding")
        p = np.ascontiguousarray(params, dtype=np.float32)
        h_ = ctypes.c_void_p()
        mvct._check(lib.mvct_cnn_create(batch_max, h, w, scale, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        ctypes.byref(h_)))
        self._h, self.h, self.w, self.batch_max = h_, h, w, batch_max

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._m.lib().mvct_cnn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptr(self, t, n, name):
        return self._m._dev_f32(t, n * self.h * self.w, name)

    def params(self) -> np.ndarray:
        out = np.zeros(PARAM_COUNT, dtype=np.float32)
        self._m._check(self._m.lib().mvct_cnn_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def set_wait(self, timeout_ms: float = 1000.0, debug_stall: bool = False):
        """``mvct_cnn_set_wait``: wait limit of the tensor-core convolutions (and the
        stall test knob)."""
        self._m._check(self._m.lib().mvct_cnn_set_wait(self._h, float(timeout_ms), int(bool(debug_stall))))

    def status(self, stream=None):
        """``mvct_cnn_status``: raises MvctError (MVCT_ETIMEOUT) if a convolution gave
        up waiting since the last check."""
        self._m._check(self._m.lib().mvct_cnn_status(self._h, ctypes.c_void_p(self._m._stream(stream))))

    def forward(self, x, out=None, stream=None):
        import torch

        n = x.shape[0]
        if out is None:
            out = torch.empty_like(x)
        self._m._check(self._m.lib().mvct_cnn_forward(self._h, self._ptr(x, n, "x"), n, self._ptr(out, n, "out"),
                                                      ctypes.c_void_p(self._m._stream(stream))))
        return out

    def grad(self, x, y, stream=None):
        import torch

        n = x.shape[0]
        g = torch.empty(PARAM_COUNT, device=x.device, dtype=torch.float32)
        loss = ctypes.c_double()
        self._m._check(self._m.lib().mvct_cnn_grad(self._h, self._ptr(x, n, "x"), self._ptr(y, n, "y"), n,
                                                   ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss),
                                                   ctypes.c_void_p(self._m._stream(stream))))
        return loss.value, g

    def train_step(self, x, y, lr: float, stream=None) -> float:
        n = x.shape[0]
        loss = ctypes.c_double()
        self._m._check(self._m.lib().mvct_cnn_train_step(self._h, self._ptr(x, n, "x"), self._ptr(y, n, "y"), n,
                                                         lr, ctypes.byref(loss),
                                                         ctypes.c_void_p(self._m._stream(stream))))
        return loss.value


# ---------------------------------------------------------------------------
# Training pairs generated by the method, training, inference
# ---------------------------------------------------------------------------
TRAIN_SEED0 = 30_000     # training phantoms: seeds TRAIN_SEED0 ..
HELDOUT_SEED0 = 50_000   # held-out phantoms: seeds HELDOUT_SEED0 ..
N_ITER_TARGET = 500
# Warm-started loop settings (measured on 48 held-out slices against the plain
# form): FAST_K sub-iterations from lambda0 = FAST_LAMBDA0 is the operating point
# near 5x the plain form's slices/s; the smallest K on the grid K_GRID at which
# every slice of a stack reaches the plain form's objective within BAR is found
# per stack (lambda0 = BAR_LAMBDA0).
FAST_K, FAST_LAMBDA0 = 100, 0.04
K_GRID, BAR_LAMBDA0, BAR = (100, 150, 200, 250, 300, 350, 400, 450, 500), 0.02, 1e-3


def case_for(seed, kind: str = "full"):
    """The seeded case of `kind` ("full": 512^2, 800 views x 738 channels,
    inserts and rods, I0 = 5e3; "small": 128^2, 200 x 184, random ellipses)."""
    from . import phantom as ph

    return ph.make_case(kind, seed)


def make_cases(seeds, kind: str = "full", workers: int = 8):
    """Seeded cases generated on the host in spawned worker processes."""
    import concurrent.futures as cf
    import functools
    import multiprocessing as mp

    seeds = list(seeds)
    if workers <= 1 or len(seeds) < 4:
        return [case_for(s, kind) for s in seeds]
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(functools.partial(case_for, kind=kind), seeds, chunksize=4))


class StackReconstructor:
    """FBP and batched OS-TV reconstructions of stacks of same-geometry slices:
    `width` plans in one :class:`mvct.Batch`, re-bound for every chunk."""

    def __init__(self, geom, n_subsets: int, width: int, device):
        import torch

        from . import mvct

        self.geom, self.width, self.device = geom, width, device
        self.plans = [mvct.Plan(geom, n_subsets) for _ in range(width)]
        self.batch = mvct.Batch(self.plans)
        R = (geom.n_views, geom.n_channels)
        self.p = [torch.empty(R, device=device) for _ in range(width)]
        self.w = [torch.empty(R, device=device) for _ in range(width)]
        self.img = [torch.empty((geom.n, geom.n), device=device) for _ in range(width)]

    def close(self):
        self.batch.close()
        for p in self.plans:
            p.close()

    def load(self, cases):
        """Copy the sinograms and weights of up to `width` cases to the device."""
        for k, c in enumerate(cases):
            self.p[k].copy_(_torch().from_numpy(c.p))
            self.w[k].copy_(_torch().from_numpy(c.w))

    def fbp(self, k: int, out):
        return self.plans[0].fbp(self.p[k], out=out)

    def run(self, count: int, betas, starts, n_iter: int, stream=None, **opts):
        """OS-TV of the first `count` loaded slices from `starts` (list of
        images; None = the loop's homogeneous start). Results in self.img."""
        torch = _torch()
        for k in range(self.width):
            if k < count and starts is not None:
                self.img[k].copy_(starts[k])
            elif k >= count:
                # unused lanes reconstruct a copy of slice 0 (results ignored)
                self.p[k].copy_(self.p[0])
                self.w[k].copy_(self.w[0])
                if starts is not None:
                    self.img[k].copy_(starts[0])
        b = list(betas) + [betas[0]] * (self.width - count)
        self.batch.bind(self.p, self.w, b, self.img, n_iter, init_from_input=starts is not None, **opts)
        self.batch.run(n_iter, stream=stream)
        self.batch.stats(0)             # waits; raises on a data or barrier error
        torch.cuda.synchronize()
        return self.img[:count]


def _torch():
    import torch

    return torch


def make_pairs(seeds, device, width: int = 96, n_iter: int = N_ITER_TARGET, workers: int = 8, log=None,
               kind: str = "full", target_opts=None):
    """(FBP images, n_iter-iteration OS-TV images from the FBP start) for the
    seeded cases, both [N][n][n] FP32 on `device`: the pairs the network learns.
    `target_opts`: loop options of the target reconstructions (default: the
    library's). The host generates the next chunk of cases while the GPU
    reconstructs one."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import time

    torch = _torch()
    seeds = list(seeds)
    ex = cf.ProcessPoolExecutor(max(1, workers), mp_context=mp.get_context("spawn"))
    chunks = [seeds[c0:c0 + width] for c0 in range(0, len(seeds), width)]
    submit = lambda ch: [ex.submit(case_for, s, kind) for s in ch]
    t_wait = t_gpu = 0.0
    rec = X = Y = None
    try:
        pending = submit(chunks[0])
        done = 0
        for ci, ch in enumerate(chunks):
            t0 = time.perf_counter()
            cases = [f.result() for f in pending]
            t_wait += time.perf_counter() - t0
            pending = submit(chunks[ci + 1]) if ci + 1 < len(chunks) else []
            if rec is None:
                g = cases[0].geom
                X = torch.empty((len(seeds), g.n, g.n), device=device)
                Y = torch.empty_like(X)
                rec = StackReconstructor(g, cases[0].n_subsets, min(width, len(seeds)), device)
            t0 = time.perf_counter()
            rec.load(cases)
            for k in range(len(cases)):
                rec.fbp(k, X[done + k])
            out = rec.run(len(cases), [c.beta for c in cases], [X[done + k] for k in range(len(cases))], n_iter,
                          **dict(target_opts or {}))
            for k in range(len(cases)):
                Y[done + k].copy_(out[k])
            torch.cuda.synchronize()
            t_gpu += time.perf_counter() - t0
            done += len(cases)
            if log:
                log(f"pairs {done}/{len(seeds)}  waiting for host cases {t_wait:.1f} s  gpu {t_gpu:.1f} s")
    finally:
        ex.shutdown(cancel_futures=True)
        if rec is not None:
            rec.close()
    return X, Y, dict(host_wait_s=t_wait, gpu_s=t_gpu)


def train(cnn: CNN, X, Y, epochs: int, batch: int, lr: float, seed: int = 0, log=None,
          lr_final: Optional[float] = None):
    """Adam on minibatches of the pairs (X, Y: [N][n][n] device tensors),
    shuffled per epoch by a seeded generator; the step size is `lr`, or, with
    `lr_final`, decays from `lr` to `lr_final` on a cosine over all steps.
    Returns the mean loss per epoch."""
    import math

    torch = _torch()
    rng = np.random.Generator(np.random.PCG64(seed))
    N = X.shape[0]
    xb = torch.empty((batch,) + tuple(X.shape[1:]), device=X.device)
    yb = torch.empty_like(xb)
    hist = []
    per_epoch = max(1, N // batch)
    total = epochs * per_epoch
    step = 0
    for ep in range(epochs):
        order = rng.permutation(N)
        tot, cnt = 0.0, 0
        for b0 in range(0, N - batch + 1, batch):
            idx = torch.from_numpy(order[b0:b0 + batch].astype(np.int64)).to(X.device)
            torch.index_select(X, 0, idx, out=xb)
            torch.index_select(Y, 0, idx, out=yb)
            rate = lr
            if lr_final is not None:
                rate = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * step / max(1, total - 1)))
            tot += cnn.train_step(xb, yb, rate)
            step += 1
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep + 1}/{epochs}  loss {hist[-1]:.6g}")
    return hist


def infer(cnn: CNN, X, out=None, stream=None):
    """Warm-start images for the FBP images X ([N][n][n]), in chunks of the
    network's batch size."""
    torch = _torch()
    out = torch.empty_like(X) if out is None else out
    for b0 in range(0, X.shape[0], cnn.batch_max):
        cnn.forward(X[b0:b0 + cnn.batch_max], out=out[b0:b0 + cnn.batch_max], stream=stream)
    return out


def evaluate(cnn: CNN, cases, Ks, device, width: int = 48, n_plain: int = N_ITER_TARGET, warm_opts=None,
             keep_images: int = 0, truth=None):
    """Compare, per case, the plain form (FBP start, `n_plain` sub-iterations)
    with FBP start + K and network start + K sub-iterations (K in Ks, and the
    start images themselves at K = 0). Objective Psi from ``mvct_objective``
    (FP64 reduction on the GPU); image relative L2 against the plain result and,
    when `truth` (list of images) is given, against the phantom.
    `warm_opts`: loop options for the network-started runs (e.g. lambda0).
    Returns a list of dicts; the first `keep_images` carry the images on the host."""
    torch = _torch()
    warm_opts = dict(warm_opts or {})
    g = cases[0].geom
    rec = StackReconstructor(g, cases[0].n_subsets, min(width, len(cases)), device)
    out = []
    rel = lambda a, b: float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    try:
        for c0 in range(0, len(cases), rec.width):
            ch = cases[c0:c0 + rec.width]
            m = len(ch)
            rec.load(ch)
            fb = torch.stack([rec.fbp(k, torch.empty((g.n, g.n), device=device)) for k in range(m)])
            cn = infer(cnn, fb)
            betas = [c.beta for c in ch]
            psi = lambda k, img: float(rec.plans[0].objective(img, rec.p[k], rec.w[k], ch[k].beta,
                                                              ch[k].tv_eps).item())
            res = [dict(seed=c.seed) for c in ch]
            imgs = {}
            plain = [t.clone() for t in rec.run(m, betas, list(fb), n_plain)]
            for k in range(m):
                res[k]["psi_plain"] = psi(k, plain[k])
                res[k]["psi_fbp_K0"] = psi(k, fb[k])
                res[k]["psi_cnn_K0"] = psi(k, cn[k])
                res[k]["rel_plain_fbp_K0"] = rel(fb[k], plain[k])
                res[k]["rel_plain_cnn_K0"] = rel(cn[k], plain[k])
                imgs[(k, "plain")] = plain[k]
            for K in Ks:
                for name, starts, opts in (("fbp", fb, {}), ("cnn", cn, warm_opts)):
                    r = rec.run(m, betas, list(starts), K, **opts)
                    for k in range(m):
                        res[k][f"psi_{name}_K{K}"] = psi(k, r[k])
                        res[k][f"rel_plain_{name}_K{K}"] = rel(r[k], plain[k])
                        if truth is not None:
                            t = torch.from_numpy(np.asarray(truth[c0 + k], dtype=np.float32)).to(device)
                            res[k][f"rel_truth_{name}_K{K}"] = rel(r[k], t)
                        imgs[(k, f"{name}_K{K}")] = r[k].clone()
            for k in range(m):
                if c0 + k < keep_images:
                    res[k]["images"] = {key[1]: v.cpu().numpy() for key, v in imgs.items() if key[0] == k}
                    res[k]["images"]["fbp_K0"] = fb[k].cpu().numpy()
                    res[k]["images"]["cnn_K0"] = cn[k].cpu().numpy()
            out += res
    finally:
        rec.close()
    return out


def sub_iterations_to_bar(cnn: Optional[CNN], cases, device, K_grid=K_GRID, width: int = 48, bar: float = BAR,
                          lambda0: Optional[float] = None, details: Optional[dict] = None):
    """The smallest K of K_grid at which every case, started from the network's
    image (cnn) or from the FBP image (cnn None), reaches the plain form's
    objective (FBP start, N_ITER_TARGET sub-iterations) within `bar`:
    (Psi_K - Psi_plain) / Psi_plain <= bar for all cases. Network starts run from
    lambda0 = BAR_LAMBDA0 (unless given), FBP starts from the library default.
    None if no K of the grid does. `details`, if given, receives the gaps of
    every K tried."""
    torch = _torch()
    g = cases[0].geom
    rec = StackReconstructor(g, cases[0].n_subsets, min(width, len(cases)), device)
    opts = {} if cnn is None else {"lambda0": BAR_LAMBDA0 if lambda0 is None else lambda0}
    try:
        chunks = []
        for c0 in range(0, len(cases), rec.width):
            ch = cases[c0:c0 + rec.width]
            rec.load(ch)
            fb = torch.stack([rec.fbp(k, torch.empty((g.n, g.n), device=device)) for k in range(len(ch))])
            starts = fb if cnn is None else infer(cnn, fb)
            psi = lambda k, img: float(rec.plans[0].objective(img, rec.p[k], rec.w[k], ch[k].beta,
                                                              ch[k].tv_eps).item())
            plain = rec.run(len(ch), [c.beta for c in ch], list(fb), N_ITER_TARGET)
            chunks.append((ch, starts.clone(), [psi(k, plain[k]) for k in range(len(ch))]))
        for K in sorted(K_grid):
            gaps = []
            for ch, starts, pp in chunks:
                rec.load(ch)
                psi = lambda k, img: float(rec.plans[0].objective(img, rec.p[k], rec.w[k], ch[k].beta,
                                                                  ch[k].tv_eps).item())
                out = rec.run(len(ch), [c.beta for c in ch], list(starts), K, **opts)
                gaps += [(psi(k, out[k]) - pp[k]) / pp[k] for k in range(len(ch))]
            if details is not None:
                details[K] = gaps
            if max(gaps) <= bar:
                return K
        return None
    finally:
        rec.close()


def summarize(results, Ks, tol: float = 1e-3):
    """Per start and K: the median / worst relative objective gap to the plain
    form, (Psi - Psi_plain) / Psi_plain, and the fraction of cases within `tol`."""
    s = {}
    for name in ("fbp", "cnn"):
        for K in [0] + list(Ks):
            gap = np.array([(r[f"psi_{name}_K{K}"] - r["psi_plain"]) / r["psi_plain"] for r in results])
            rl = np.array([r[f"rel_plain_{name}_K{K}"] for r in results])
            s[f"{name}_K{K}"] = dict(gap_median=float(np.median(gap)), gap_max=float(gap.max()),
                                     within_tol=float(np.mean(gap <= tol)), rel_l2_plain_median=float(np.median(rl)))
    return s


class WarmPipeline:
    """The warm-started, batched reconstruction of a stack of same-geometry slices:
    FBP of every slice (``mvct_fbp``), the network's start images
    (``mvct_cnn_forward``), and K OS-TV sub-iterations of all slices in one
    persistent launch (``mvct_batch_run``), optionally captured as one CUDA graph.

        pipe = WarmPipeline(geom, n_subsets, slices, K, device)
        pipe.load(p, w, betas)          # [B][V][C] tensors (host or device)
        pipe.tune()                     # optional: the batch autotuner
        pipe.capture()                  # optional: one CUDA graph for the chain
        pipe.run()                      # enqueue the chain; images in pipe.img
    """

    def __init__(self, geom, n_subsets: int, slices: int, K: int, device, lambda0: float = FAST_LAMBDA0,
                 weights: Optional[np.ndarray] = None, cnn_batch: int = 16):
        torch = _torch()
        from . import mvct

        self.geom, self.S, self.B, self.K, self.device = geom, n_subsets, slices, K, device
        self.lambda0 = lambda0
        self.plans = [mvct.Plan(geom, n_subsets) for _ in range(slices)]
        self.batch = mvct.Batch(self.plans)
        self.p = torch.zeros((slices, geom.n_views, geom.n_channels), device=device)
        self.w = torch.zeros_like(self.p)
        self.fbp = torch.zeros((slices, geom.n, geom.n), device=device)
        self.img = torch.zeros_like(self.fbp)
        self.cnn = CNN(min(cnn_batch, slices), geom.n, geom.n, load_weights() if weights is None else weights)
        self.stream = torch.cuda.Stream(device=device)
        self.graph = None
        self.betas = None

    def load(self, p, w, betas):
        """Copy the stack's log projections and weights ([B][V][C]) and bind the batch."""
        self.p.copy_(p, non_blocking=True)
        self.w.copy_(w, non_blocking=True)
        betas = [float(b) for b in betas]
        if betas != self.betas:
            self.batch.bind(list(self.p), list(self.w), betas, list(self.img), self.K, init_from_input=True,
                            lambda0=self.lambda0)
            self.betas = betas
            self.graph = None

    def tune(self, n_iter_probe: int = 40) -> dict:
        """The batch autotuner on the loaded stack (view groups per tile)."""
        self.graph = None
        return self.batch.tune(n_iter_probe)

    def _chain(self, st, marks=None):
        torch = _torch()
        if marks:
            marks[0].record(st)
        for k in range(self.B):
            self.plans[k].fbp(self.p[k], out=self.fbp[k], stream=st)
        if marks:
            marks[1].record(st)
        infer(self.cnn, self.fbp, out=self.img, stream=st)
        if marks:
            marks[2].record(st)
        self.batch.run(self.K, stream=st)
        if marks:
            marks[3].record(st)

    def capture(self):
        """Run the chain once, then capture it as one CUDA graph."""
        torch = _torch()
        st = self.stream
        st.wait_stream(torch.cuda.current_stream(self.device))
        self._chain(st)
        torch.cuda.synchronize(self.device)
        self.check()                              # raises if the run failed
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(st):
            with torch.cuda.graph(g, stream=st):
                self._chain(st)
        torch.cuda.synchronize(self.device)
        self.graph = g

    def run(self):
        """Enqueue the chain on the current stream (the captured graph if any)."""
        torch = _torch()
        if self.graph is not None:
            self.graph.replay()
        else:
            self._chain(torch.cuda.current_stream(self.device))

    def stage_ms(self) -> dict:
        """Device time per slice of the three stages of one direct (uncaptured) run."""
        torch = _torch()
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        self._chain(torch.cuda.current_stream(self.device), marks)
        torch.cuda.synchronize(self.device)
        return {"fbp": marks[0].elapsed_time(marks[1]) / self.B, "cnn": marks[1].elapsed_time(marks[2]) / self.B,
                "setup_and_loop": marks[2].elapsed_time(marks[3]) / self.B}

    def check(self):
        """Raise if a run since the last check failed (the network's convolution
        waits; the loop's data check or barrier timeout)."""
        self.cnn.status()
        self.batch.stats(0)

    def close(self):
        self.graph = None
        self.cnn.close()
        self.batch.close()
        for p in self.plans:
            p.close()


def weights_path() -> str:
    import os

    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warmstart_512.npy")


def load_weights(path: Optional[str] = None) -> np.ndarray:
    p = np.load(path or weights_path())
    if p.shape != (PARAM_COUNT,) or p.dtype != np.float32:
        raise ValueError("warm-start weights have the wrong layout")
    return p


def _train_main(args):
    import json
    import os
    import sys
    import time

    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    log = lambda s: print(s, file=sys.stderr, flush=True)
    t0 = time.perf_counter()
    init = load_weights(args.init) if args.init else init_params(args.seed)
    X, Y, tp = make_pairs(range(TRAIN_SEED0, TRAIN_SEED0 + args.pairs), dev, args.width,
                          n_iter=args.target_iterations, workers=args.workers, log=log)
    cnn = CNN(args.batch, X.shape[1], X.shape[2], init)
    t1 = time.perf_counter()
    hist = train(cnn, X, Y, args.epochs, args.batch, args.lr, args.seed, log, lr_final=args.lr_final)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    params = cnn.params()
    cnn.close()
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, params)
    rec = dict(pairs=args.pairs, train_seeds=[TRAIN_SEED0, TRAIN_SEED0 + args.pairs - 1], epochs=args.epochs,
               batch=args.batch, lr=args.lr, lr_final=args.lr_final, seed=args.seed,
               target_iterations=args.target_iterations, target_options="the library defaults",
               init=os.path.basename(args.init) if args.init else None, epoch_loss=hist,
               pair_generation_s=t1 - t0, pair_timing=tp, training_s=t2 - t1,
               steps=args.epochs * (args.pairs // args.batch))
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))
    return 0


def _evaluate_main(args):
    """Held-out evaluation on the GPU: per seed the plain form (FBP start, 500
    sub-iterations) against network start + K and FBP start + K sub-iterations,
    compared by the objective Psi (mvct_objective, FP64 reduction; pinned against
    the FP64 oracle by the tests); one JSON line: the summary per start and K
    and, with --per-seed, every seed's values."""
    import json
    import os
    import time

    torch = _torch()
    seeds = list(range(args.seed0, args.seed0 + args.seeds))
    t0 = time.perf_counter()
    cases = make_cases(seeds, workers=args.workers)
    t_gen = time.perf_counter() - t0
    dev = torch.device("cuda", torch.cuda.current_device())
    cnn = CNN(16, cases[0].geom.n, cases[0].geom.n, load_weights(args.weights))
    warm = {} if args.lambda0 is None else {"lambda0": args.lambda0}
    t0 = time.perf_counter()
    res = evaluate(cnn, cases, args.Ks, dev, width=args.width, warm_opts=warm)
    t_gpu = time.perf_counter() - t0
    cnn.close()
    line = dict(seeds=[seeds[0], seeds[-1]], Ks=args.Ks, warm_opts=warm,
                weights=os.path.basename(args.weights or weights_path()),
                summary=summarize(res, args.Ks), host_gen_s=t_gen, gpu_eval_s=t_gpu)
    if args.bar:
        # the per-slice bar over all the seeds, from the network's start and from FBP
        cnn = CNN(16, cases[0].geom.n, cases[0].geom.n, load_weights(args.weights))
        for name, net in (("cnn", cnn), ("fbp", None)):
            det = {}
            k = sub_iterations_to_bar(net, cases, dev, K_GRID, width=args.width, details=det)
            line[f"bar_{name}"] = dict(K=k, max_gap_by_K={str(kk): float(max(v)) for kk, v in det.items()},
                                       median_gap_by_K={str(kk): float(np.median(v)) for kk, v in det.items()})
        cnn.close()
    if args.per_seed:
        line["per_seed"] = res
    print(json.dumps(line))
    return 0


def _main(argv=None):
    """``python -m paper_1903_10088_gb300.warmstart [train] [--pairs ...]`` trains the
    network on pairs the method generates; ``... evaluate [--seeds 200 ...]`` runs
    the held-out evaluation."""
    import argparse
    import os
    import sys

    argv = list(sys.argv[1:] if argv is None else argv)
    mode = argv.pop(0) if argv and argv[0] in ("train", "evaluate") else "train"
    ap = argparse.ArgumentParser(prog=f"warmstart {mode}")
    ap.add_argument("--width", type=int, default=96 if mode == "train" else 48,
                    help="slices per batched reconstruction")
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    if mode == "train":
        ap.add_argument("--pairs", type=int, default=2000)
        ap.add_argument("--epochs", type=int, default=20)
        ap.add_argument("--batch", type=int, default=16)
        ap.add_argument("--lr", type=float, default=1e-3)
        ap.add_argument("--lr-final", type=float, default=None, help="cosine decay of the step size to this value")
        ap.add_argument("--seed", type=int, default=0)
        ap.add_argument("--target-iterations", type=int, default=N_ITER_TARGET)
        ap.add_argument("--init", default=None, help="start from these weights instead of a fresh network")
        ap.add_argument("--out", default=weights_path())
        return _train_main(ap.parse_args(argv))
    ap.add_argument("--weights", default=None)
    ap.add_argument("--seeds", type=int, default=200)
    ap.add_argument("--seed0", type=int, default=HELDOUT_SEED0)
    ap.add_argument("--Ks", type=int, nargs="+", default=[25, 50, 100])
    ap.add_argument("--lambda0", type=float, default=None, help="lambda0 of the network-started runs")
    ap.add_argument("--per-seed", action="store_true")
    ap.add_argument("--bar", action="store_true", help="also search the smallest K at which every seed is within "
                                                       "1e-3 of the plain form (network and FBP starts)")
    return _evaluate_main(ap.parse_args(argv))


if __name__ == "__main__":
    import sys

    sys.exit(_main())
