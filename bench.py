"""Benchmark of the OS-TV MVCT reconstruction on GB300.

Workload (default): plain OS-TV reconstruction of one 512x512 slice over a
40 cm FOV from 800 views x 738 equiangular channels (fan beam, SAD 85 cm),
20 ordered subsets, 500 sub-iterations, TV beta = 1e-3, eps = 1e-6, I0 = 5e3
Poisson data on a seeded ellipse phantom with low-contrast inserts and rods.
One step = one full reconstruction (set-up + 500 sub-iterations) of one slice
per GPU through the C ABI. Metric: slices/s (whole job).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 it is launched by torchrun, one process per GPU; each rank
reconstructs its own slice (weak scaling, no data-path collective); the time is
the maximum over ranks. ``--impl reference`` times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1903_10088_gb300 import phantom as ph  # noqa: E402

WORKLOAD = dict(workload="plain OS-TV, one 512^2 slice per step (FBP start)", n=512, fov_cm=40.0, n_views=800,
                n_channels=738, sad_cm=85.0, subsets=20, sub_iterations=500, beta=1e-3, tv_eps=1e-6,
                I0=5e3, phantom="water disk + 7 low-contrast inserts + 4 rods (seeded)")
METRIC = "512^2 slices/s at 500 OS-TV iters (plain vs warm-start+batched); GRay/s; %HBM"
BATCH_WORKLOAD = dict(workload="batched uneven helical stack, 96 slices per step in one persistent launch",
                      slices="48 x 512^2 (800 views x 738 ch) + 32 x 384^2 (600 x 552) + 16 x 256^2 (400 x 368)",
                      fov_cm=40.0, sad_cm=85.0, subsets=20, sub_iterations=500, beta=1e-3, tv_eps=1e-6,
                      I0="log-uniform in [2e3, 2e4] per slice", launch="CUDA-graph replay of mvct_batch_run")
SEED0 = 100
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}


# --------------------------------------------------------------------------
# accounting
# --------------------------------------------------------------------------
_TAPS = {}


def tap_counts(geom: ph.Geometry, n_subsets: int) -> np.ndarray:
    key = (geom, n_subsets)
    if key not in _TAPS:
        _TAPS[key] = _tap_counts(geom, n_subsets)
    return _TAPS[key]


def _tap_counts(geom: ph.Geometry, n_subsets: int) -> np.ndarray:
    """In-image Joseph taps (ray, pixel pairs) of every subset: the number of
    interpolation taps the reprojection reads, equal to the number of
    residual reads of the matched backprojection. Pure geometry accounting."""
    n, d = geom.n, geom.delta
    sx, sy, dx, dy = ph.rays(geom)
    pc = (n - 1) / 2.0
    p = np.arange(n, dtype=np.float64) - pc
    counts = np.zeros(n_subsets, dtype=np.int64)
    for v in range(geom.n_views):
        xd = np.abs(dx[v]) >= np.abs(dy[v])
        m = np.where(xd, dy[v] / np.where(xd, dx[v], 1), dx[v] / np.where(xd, 1, dy[v]))
        uc = np.where(xd, (sy[v] - sx[v] * m) / d, (sx[v] - sy[v] * m) / d) + pc
        u = uc[:, None] + m[:, None] * p[None, :]
        i0 = np.floor(u)
        inside = ((i0 >= 0) & (i0 < n)).sum() + ((i0 + 1 >= 0) & (i0 + 1 < n)).sum()
        counts[v % n_subsets] += int(inside)
    return counts


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return PEAKS_FALLBACK, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("mvct_device.cuh", "mvct_recon.cu"):
        with open(os.path.join(ROOT, "paper_1903_10088_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_record():
    """The committed ncu figures of one k_recon launch of the plain workload, if
    they were taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "k_recon_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return d


def ncu_traffic():
    """DRAM bytes per k_recon launch (dram__bytes_read.sum + dram__bytes_write.sum)."""
    d = ncu_record()
    return d.get("dram_bytes_per_launch_full_workload") if d else None


def issue_roofline(warp_instructions, seconds, n_sms, sm_mhz):
    """Instruction-issue view of a kernel: warp instructions per second against
    the issue rate of the GPU, one warp instruction per cycle on each of the 4
    schedulers of every SM at the sampled SM clock. The loop kernel's taps are
    L1/L2 hits, so issue (not HBM) is what bounds it."""
    if not warp_instructions or not seconds or not n_sms or not sm_mhz:
        return None
    peak = 4.0 * n_sms * sm_mhz * 1e6
    achieved = warp_instructions / seconds
    return {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "G warp-instructions/s",
            "frac": achieved / peak,
            "warp_instructions_per_launch": warp_instructions,
            "peak_source": f"4 issue slots x {n_sms} SMs x {sm_mhz:.0f} MHz (median sampled SM clock)",
            "instructions_source": "smsp__inst_executed.sum of the committed ncu capture of this launch"}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, tag: str = ""):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mvct_clocks_gpu{index}{tag}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# distributed helpers (testable on CPU with gloo)
# --------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def slice_seeds(rank: int, per_rank: int):
    """Each rank reconstructs its own seeded slices; no data is exchanged."""
    return [SEED0 + rank * per_rank + k for k in range(per_rank)]


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# --------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# --------------------------------------------------------------------------
def cpu_info() -> dict:
    """Host cores and CPU model (lscpu, else /proc/cpuinfo, else the platform)."""
    import platform

    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except Exception:
        pass
    if not model and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def time_oracle_slice(case, threads: int):
    """One whole slice of the plain form by the oracle, unextrapolated: its FBP
    over all views (threaded view runs), then set-up + every sub-iteration from
    that start, with `threads` threads (the oracle's results do not depend on the
    count). Returns (seconds, sample description)."""
    import oracle
    from oracle import fbp as ofbp

    oracle.build()
    used = oracle.set_threads(threads)
    try:
        t0 = time.perf_counter()
        start = ofbp.fbp(case.geom, case.p, threads=threads)
        t_fbp = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.recon(case.geom, case.n_subsets, case.p, case.w, case.beta, case.n_iter, init=start)
        t_loop = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    sample = (f"FP64 oracle, {used} threads (OpenMP over rays and views, bit-identical to 1 thread), one "
              f"whole slice, not extrapolated: FBP of all {case.geom.n_views} views {t_fbp:.2f} s, set-up + "
              f"{case.n_iter} sub-iterations {t_loop:.2f} s")
    return t_fbp + t_loop, sample, used


def time_oracle(case, sub_iters: int):
    """Oracle FBP start + set-up + `sub_iters` sub-iterations; returns (seconds
    per slice at the full sub-iteration count, sample description). The FBP is
    timed on every tenth view and scaled (its cost is linear in the views)."""
    import dataclasses

    import oracle
    from oracle import fbp as ofbp

    oracle.build()
    g10 = dataclasses.replace(case.geom, n_views=case.geom.n_views // 10)
    t0 = time.perf_counter()
    ofbp.fbp(g10, case.p[::10])
    t_fbp = (time.perf_counter() - t0) * case.geom.n_views / g10.n_views
    t0 = time.perf_counter()
    oracle.setup(case.geom, case.w, case.beta, case.tv_eps)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.recon(case.geom, case.n_subsets, case.p, case.w, case.beta, sub_iters)  # set-up + loop
    t_run = time.perf_counter() - t0
    t_iter = max(t_run - t_setup, 1e-9) / sub_iters
    t_slice = t_fbp + t_setup + case.n_iter * t_iter
    sample = (f"FP64 oracle, 1 thread: FBP start ({t_fbp:.2f} s, timed on {g10.n_views} of "
              f"{case.geom.n_views} views and scaled), set-up ({t_setup:.2f} s) + {sub_iters} "
              f"sub-iterations ({t_iter * 1e3:.1f} ms each) of the full-size workload, scaled to "
              f"{case.n_iter} sub-iterations per slice")
    return t_slice, sample


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, one whole slice of the
    plain form per step (FBP of all views + set-up + 500 sub-iterations), with
    as many threads as the host has cores. Warm-up steps run a short sample."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    case = ph.make_case("full", SEED0)
    threads = args.ref_threads or os.cpu_count() or 1
    short = ph.make_case("full", SEED0, n_iter=2)
    for _ in range(args.warmup):
        time_oracle_slice(short, threads)
    steps, sample, used = [], "", 1
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        t_slice, sample, used = time_oracle_slice(case, threads)
        steps.append(t_slice)
    wall = time.perf_counter() - wall0
    t = float(np.sum(steps)) / max(1, args.steps)
    value = 1.0 / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, l2="n/a (CPU)"),
        "cpu_baseline": dict({"value": value, "unit": "slices/s", "cores": used, "kind": "oracle",
                              "sample": sample, "timed_wall_s": wall}, **cpu_info()),
        "e2e": {"value": value, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1903_10088_gb300 import mvct

    mvct.lib()
    cases = [ph.make_case("full", s) for s in slice_seeds(rank, 1)]
    case = cases[0]
    g = case.geom
    plan = mvct.Plan(g, case.n_subsets)
    p = torch.from_numpy(case.p).to(dev)
    w = torch.from_numpy(case.w).to(dev)
    img = torch.empty((g.n, g.n), device=dev, dtype=torch.float32)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream()

    # launch shape of the loop picked by the autotuner on this slice (untimed)
    tune = plan.tune(p, w, case.beta, 40)

    def step():
        # the plain form: FBP start image, then the OS-TV loop
        plan.fbp(p, out=img)
        return plan.recon(p, w, case.beta, case.n_iter, img=img, init_from_input=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-resident timed region ----------------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    loop_ms, fwd_ms, back_ms = [], [], []
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))          # evict L2 between timed steps
            ev[k][0].record(stream)
            _, res = step()
            ev[k][1].record(stream)
            loop_ms.append(res.loop_ms)
            fwd_ms.append(res.forward_ms)
            back_ms.append(res.back_ms)
        torch.cuda.synchronize()
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = float(np.sum(step_ms))
    t_max = max_over_ranks(t_local, dev)
    slices = ws * args.steps
    value = slices / (t_max / 1e3)

    # ---- end to end through host buffers -------------------------------
    hp = torch.from_numpy(case.p).pin_memory()
    hw = torch.from_numpy(case.w).pin_memory()
    hout = torch.empty((g.n, g.n), dtype=torch.float32).pin_memory()
    e2e_ms = []
    barrier()
    for k in range(max(1, args.steps)):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p.copy_(hp, non_blocking=True)
        w.copy_(hw, non_blocking=True)
        step()
        hout.copy_(img, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_t = max_over_ranks(float(np.sum(e2e_ms)), dev)
    e2e_value = ws * len(e2e_ms) / (e2e_t / 1e3)

    # ---- roofline of the dominant kernel (the persistent loop) ---------
    taps = tap_counts(g, case.n_subsets)
    taps_per_launch = float(sum(taps[n % case.n_subsets] for n in range(case.n_iter)))
    tap_bytes = 2 * 4 * taps_per_launch  # reprojection taps + matched-adjoint residual reads
    loop_s = float(np.mean(loop_ms)) / 1e3
    peaks, peak_kind = load_peaks()
    achieved = tap_bytes / loop_s / 1e9
    traffic = ncu_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": "k_recon (persistent OS-TV loop)",
                "algorithmic_bytes": "4 B x (Joseph reprojection taps + matched-backprojection residual reads) "
                                     f"= {tap_bytes:.4g} B per launch; a tap-byte rate: the taps are served "
                                     "from L1/L2 (the image stays resident), so this is not DRAM traffic "
                                     "(see dram_roofline and issue_roofline)",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst copy)"}
    gray = 2.0 * taps_per_launch / loop_s / 1e9

    # the stand-alone projector and backprojector (mvct_forward / mvct_back) on the
    # same slice: tap bytes per call / event time against the same peak
    def op_time(fn, reps=10):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    Vs = g.n_views // case.n_subsets
    q_all = torch.empty((g.n_views, g.n_channels), device=dev)
    q_sub = torch.empty((Vs, g.n_channels), device=dev)
    b_img = torch.empty((g.n, g.n), device=dev)
    p_sub = p[0::case.n_subsets].contiguous()
    op_bytes = {"all_views": 4.0 * float(taps.sum()), "one_subset": 4.0 * float(taps[0])}
    op_s = {"forward_all_views": op_time(lambda: plan.forward(img, -1, out=q_all)),
            "back_all_views": op_time(lambda: plan.back(p, -1, out=b_img)),
            "forward_one_subset": op_time(lambda: plan.forward(img, 0, out=q_sub)),
            "back_one_subset": op_time(lambda: plan.back(p_sub, 0, out=b_img))}
    operators = {}
    for k, t in op_s.items():
        nb = op_bytes["all_views" if "all" in k else "one_subset"]
        operators[k] = {"ms": t * 1e3, "achieved_gbs": nb / t / 1e9, "frac": nb / t / 1e9 / peaks["hbm_gbs"]}

    # the TV-weight sweep of the workload (beta = 1e-3 is the timed step above)
    sweep = []
    for beta in (1e-4, 1e-3, 1e-2):
        def bstep():
            plan.fbp(p, out=img)
            return plan.recon(p, w, beta, case.n_iter, img=img, init_from_input=True)
        bstep()
        ms = []
        for k in range(3):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bstep()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        psi = float(plan.objective(img, p, w, beta, case.tv_eps).cpu())
        sweep.append({"beta": beta, "slices_per_s": 1e3 / float(np.mean(ms)), "ms_per_slice": float(np.mean(ms)),
                      "psi_500": psi})

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        t_all, sample_all, used = time_oracle_slice(case, args.ref_threads or os.cpu_count() or 1)
        t_one, sample_one = time_oracle(case, args.ref_sub_iters)
        cpu = dict({"value": 1.0 / t_all, "unit": "slices/s", "cores": used, "kind": "oracle",
                    "sample": sample_all,
                    "single_thread": {"value": 1.0 / t_one, "unit": "slices/s", "cores": 1, "sample": sample_one}},
                   **cpu_info())

    batched = None
    if not args.no_batched:
        batched = batched_leg(args, dev, ws, steps=2, warmup=1)

    warm = None
    if not args.no_warm:
        warm = run_warm(args, dev, ws, value)

    launches_per_step = 6  # k_fbp_filter, k_fbp_back, k_forward + k_back_splat + k_setup_merge (set-up), k_recon
    line = {
        "metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD, l2="flushed between timed steps (512 MiB write)",
                       parallelism=f"replicas x{ws}, one slice per GPU per step",
                       launch_shape={"view_groups_per_tile": tune["groups"] or "default rule (balanced plan)",
                                     "grid_blocks": tune["grid_blocks"],
                                     "candidates": [[c["groups"], c["grid_blocks"], round(c["ms_per_iter"], 5)]
                                                    for c in tune["candidates"]],
                                     "autotuned_ms_per_iter": tune["ms_per_iter"],
                                     "default_ms_per_iter": tune["default_ms_per_iter"]}),
        "gray_per_s": gray, "loop_ms_per_slice": float(np.mean(loop_ms)),
        "setup_and_loop_ms_per_slice": float(np.mean(step_ms)),
        "loop_phase_ms_per_slice": {"reprojection+residual": float(np.mean(fwd_ms)),
                                    "estimation+tv+update": float(np.mean(back_ms))},
        # each phase against its half of the tap bytes (the taps the projector reads
        # equal the residual reads of the matched backprojection); phase times include
        # the phase's closing group barrier
        "phase_tap_fraction": {
            "reprojection": 4 * taps_per_launch / (float(np.mean(fwd_ms)) / 1e3) / 1e9 / peaks["hbm_gbs"],
            "backprojection": 4 * taps_per_launch / (float(np.mean(back_ms)) / 1e3) / 1e9 / peaks["hbm_gbs"]},
        "roofline": roofline,
        "operator_roofline": dict(operators, bytes="4 B x in-image Joseph taps of the call (taps read by the "
                                                   "projector = residual reads of the matched backprojection)",
                                  peak_gbs=peaks["hbm_gbs"]),
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "slices/s",
                "h2d_bytes_per_step": int(hp.numel() * 4 + hw.numel() * 4),
                "d2h_bytes_per_step": int(hout.numel() * 4)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "grid_blocks": res.grid_blocks,
        "beta_sweep": sweep,
        "batched_uneven": batched,
        "warm_start_batched": warm,
    }
    rec = ncu_record()
    if traffic:
        # what the loop kernel really moves through HBM (ncu DRAM bytes of one launch,
        # taken on this kernel source) over the same launch time
        line["dram_roofline"] = {"bound": "hbm", "achieved": traffic / loop_s / 1e9, "peak": peaks["hbm_gbs"],
                                 "unit": "GB/s", "frac": traffic / loop_s / 1e9 / peaks["hbm_gbs"],
                                 "bytes_source": "dram__bytes_read.sum + dram__bytes_write.sum of the committed "
                                                 "ncu capture of this launch"}
    line["issue_roofline"] = issue_roofline(rec.get("warp_instructions_per_launch") if rec else None, loop_s,
                                            torch.cuda.get_device_properties(dev).multi_processor_count,
                                            line["clocks"].get("sm_mhz") or line["clocks"].get("sm_max_mhz"))
    if rank == 0:
        print(json.dumps(line))
    plan.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


WARM_WORKLOAD = dict(workload="learned warm start + batched OS-TV: a stack of 48 held-out 512^2 slices per step",
                     slices=48, n=512, n_views=800, n_channels=738, subsets=20, beta=1e-3, tv_eps=1e-6, I0=5e3,
                     chain="FBP -> CNN (8 conv3x3, 32 ch, BF16, tcgen05 tensor cores) -> K OS-TV sub-iterations, "
                           "all slices in one persistent launch, the whole chain one CUDA-graph replay",
                     quality="objective Psi of every slice against the plain form (FBP start, 500 sub-iterations)")


def _time_chain(args, dev, ws, wst, cases, K, lam0, flush):
    """Time the warm chain of the stack at K sub-iterations from lambda0 (CUDA-graph
    replays, L2 flushed between steps) and end to end with host buffers; returns
    the figures and the final images' objectives."""
    import torch

    B = len(cases)
    g = cases[0].geom
    _, rank, local = dist_env()
    pipe = wst.WarmPipeline(g, cases[0].n_subsets, B, K, dev, lambda0=lam0)
    pipe.load(torch.stack([torch.from_numpy(c.p) for c in cases]), torch.stack([torch.from_numpy(c.w) for c in cases]),
              [c.beta for c in cases])
    tune = pipe.tune(40)                             # view groups per tile (untimed; images restored)
    pipe.capture()
    for _ in range(args.warmup):
        pipe.run()
    torch.cuda.synchronize()
    pipe.check()                                     # raises if a run failed
    cur = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local, f"_warm{K}") as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(cur)
            pipe.run()
            ev[k][1].record(cur)
        torch.cuda.synchronize()
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_max = max_over_ranks(float(np.sum(step_ms)), dev)
    value = B * ws * args.steps / (t_max / 1e3)
    stage_ms = pipe.stage_ms()
    # end to end: host sinograms and weights in, host images out
    P, W, IMG = pipe.p, pipe.w, pipe.img
    hP, hW = P.cpu().pin_memory(), W.cpu().pin_memory()
    hI = torch.empty_like(IMG, device="cpu").pin_memory()
    e2e_ms = []
    for k in range(max(1, args.steps)):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        P.copy_(hP, non_blocking=True)
        W.copy_(hW, non_blocking=True)
        pipe.run()
        hI.copy_(IMG, non_blocking=True)
        e1.record(cur)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    pipe.check()                                     # the timed and end-to-end runs succeeded
    e2e_t = max_over_ranks(float(np.sum(e2e_ms)), dev)
    psi = np.array([float(pipe.plans[0].objective(IMG[k], P[k], W[k], cases[k].beta, cases[k].tv_eps).item())
                    for k in range(B)])
    pipe.close()
    return {
        "value": value, "unit": "slices/s", "ms_per_step": t_max / args.steps, "sub_iterations": K,
        "lambda0": lam0,
        "launch_shape": {"view_groups_per_tile": tune["groups"] or "default rule",
                         "autotuned_ms_per_iter": tune["ms_per_iter"], "default_ms_per_iter": tune["default_ms_per_iter"]},
        "stage_ms_per_slice": stage_ms,
        "e2e": {"value": B * ws * len(e2e_ms) / (e2e_t / 1e3), "unit": "slices/s",
                "h2d_bytes_per_step": int(hP.numel() * 4 + hW.numel() * 4),
                "d2h_bytes_per_step": int(hI.numel() * 4)},
        "gpu_launches_per_step": 2 * B + 10 * ((B + 15) // 16) + 2 + 3 * B,
        "clocks": clk.summary(),
    }, psi


def run_warm(args, dev, ws, plain_slices_per_s):
    """The warm-started, batched form: per step, FBP of every slice of the stack,
    the network's start images, and K OS-TV sub-iterations of all slices in one
    persistent launch, replayed as one CUDA graph. Timed at two operating points:
    K = warmstart.FAST_K (near 5x the plain form) and the smallest K of
    warmstart.K_GRID at which every slice of the stack reaches the plain form's
    objective within 1e-3 (searched on the stack, untimed). Quality: Psi of every
    slice against the plain form's Psi (FBP start, 500 sub-iterations)."""
    import torch

    from paper_1903_10088_gb300 import warmstart as wst

    B = WARM_WORKLOAD["slices"]
    _, rank, local = dist_env()
    seeds = range(wst.HELDOUT_SEED0 + rank * B, wst.HELDOUT_SEED0 + (rank + 1) * B)
    cases = wst.make_cases(seeds, workers=min(16, os.cpu_count() or 1))
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev, dtype=torch.float32)
    g = cases[0].geom

    # the plain form's objective of every slice (batched FBP + 500, identical results)
    rec = wst.StackReconstructor(g, cases[0].n_subsets, B, dev)
    rec.load(cases)
    fb = [rec.fbp(k, torch.empty((g.n, g.n), device=dev)) for k in range(B)]
    plain = rec.run(B, [c.beta for c in cases], fb, wst.N_ITER_TARGET)
    psi_plain = np.array([float(rec.plans[0].objective(plain[k], rec.p[k], rec.w[k], cases[k].beta,
                                                       cases[k].tv_eps).item()) for k in range(B)])
    rec.close()

    def gap_stats(psi):
        gap = (psi - psi_plain) / psi_plain
        return {"median": float(np.median(gap)), "max": float(gap.max()), "min": float(gap.min()),
                "within_1e-3": float(np.mean(gap <= 1e-3))}

    fast, psi_fast = _time_chain(args, dev, ws, wst, cases, wst.FAST_K, wst.FAST_LAMBDA0, flush)
    fast["psi_gap_vs_plain"] = gap_stats(psi_fast)
    fast["speedup_vs_plain"] = fast["value"] / plain_slices_per_s if plain_slices_per_s else None

    # the per-slice bar: search K on the stack, then time the chain there
    cnn = wst.CNN(16, g.n, g.n, wst.load_weights())
    details = {}
    k_bar = wst.sub_iterations_to_bar(cnn, cases, dev, wst.K_GRID, width=B, details=details)
    cnn.close()
    at_bar = None
    if k_bar is not None:
        at_bar, psi_bar = _time_chain(args, dev, ws, wst, cases, k_bar, wst.BAR_LAMBDA0, flush)
        at_bar["psi_gap_vs_plain"] = gap_stats(psi_bar)
        at_bar["speedup_vs_plain"] = at_bar["value"] / plain_slices_per_s if plain_slices_per_s else None
    return {
        "value": (at_bar or fast)["value"], "unit": "slices/s",
        "operating_point": "every slice within 1e-3 of the plain form" if at_bar else "fast (bar not reached)",
        "speedup_vs_plain": (at_bar or fast)["speedup_vs_plain"],
        "config": dict(WARM_WORKLOAD, seeds=[seeds[0], seeds[-1]],
                       weights="paper_1903_10088_gb300/weights/warmstart_512.npy",
                       l2="flushed between timed steps (512 MiB write)"),
        "at_per_slice_bar": at_bar,
        "at_fast_k": fast,
        "bar_search": {"K_grid": list(wst.K_GRID), "lambda0": wst.BAR_LAMBDA0, "bar": wst.BAR,
                       "max_gap_by_K": {str(k): float(max(v)) for k, v in details.items()}},
    }


def _make_batch_case(args):
    seed, n, V, C, I0 = args
    g = ph.Geometry(n=n, n_views=V, n_channels=C)
    return ph.make_case("full", seed, geom=g, I0=I0)


def batch_cases(seed0=1000, groups=ph.BATCH_GROUPS, workers=8):
    """The 96-slice uneven stack, generated in spawned worker processes."""
    import concurrent.futures as cf
    import multiprocessing as mp

    jobs = []
    k = 0
    for count, g in groups:
        for _ in range(count):
            rng = np.random.Generator(np.random.PCG64(seed0 + k))
            I0 = float(math.exp(rng.uniform(math.log(2e3), math.log(2e4))))
            jobs.append((seed0 + k, g.n, g.n_views, g.n_channels, I0))
            k += 1
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_make_batch_case, jobs))


def batched_leg(args, dev, ws, steps, warmup):
    """The batched uneven stack (96 slices of three geometries, 500 sub-iterations
    each, one persistent launch per step, autotuned view groups, replayed as one
    CUDA graph). Returns its JSON object; per-slice parity of the batch kernel at
    these sizes is the job of tests/test_gpu_bench_parity.py."""
    import torch

    from paper_1903_10088_gb300 import mvct

    _, rank, local = dist_env()
    stack = getattr(args, "stack_slices", 0) or 0
    groups = [(stack, ph.GEOM_512)] if stack > 0 else ph.BATCH_GROUPS
    cases = batch_cases(seed0=1000 + 96 * rank, groups=groups, workers=min(16, os.cpu_count() or 1))
    n_iter = getattr(args, "stack_iters", 0) or cases[0].n_iter
    plans = [mvct.Plan(c.geom, c.n_subsets) for c in cases]
    p = [torch.from_numpy(c.p).to(dev) for c in cases]
    w = [torch.from_numpy(c.w).to(dev) for c in cases]
    imgs = [torch.zeros((c.geom.n, c.geom.n), device=dev) for c in cases]
    batch = mvct.Batch(plans)
    batch.bind(p, w, [c.beta for c in cases], imgs, n_iter)
    tune = batch.tune(40)                             # view groups per tile (untimed; images restored)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev, dtype=torch.float32)
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    batch.run(n_iter, stream=s)                       # first call outside capture
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            batch.run(n_iter, stream=s)
    torch.cuda.synchronize(dev)
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    batch.stats(0, n_iter)                            # raises if the runs failed
    cur = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local, "_batched") as clk:
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record(cur)
            graph.replay()
            ev[k][1].record(cur)
        torch.cuda.synchronize(dev)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_max = max_over_ranks(float(np.sum(step_ms)), dev)
    n_slices = len(cases) * ws * steps
    value = n_slices / (t_max / 1e3)

    # end to end: every slice's p and w from pinned host memory, every image back
    hp = [torch.from_numpy(c.p).pin_memory() for c in cases]
    hw = [torch.from_numpy(c.w).pin_memory() for c in cases]
    hi = [torch.empty(im.shape, dtype=torch.float32).pin_memory() for im in imgs]
    e2e_ms = []
    for k in range(max(1, steps)):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for a, b in zip(p, hp):
            a.copy_(b, non_blocking=True)
        for a, b in zip(w, hw):
            a.copy_(b, non_blocking=True)
        graph.replay()
        for a, b in zip(hi, imgs):
            a.copy_(b, non_blocking=True)
        e1.record(cur)
        torch.cuda.synchronize(dev)
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_t = max_over_ranks(float(np.sum(e2e_ms)), dev)

    work = [c.geom.n_views / c.n_subsets * c.geom.n_channels * c.geom.n for c in cases]
    w512 = 800 / 20 * 738 * 512
    equiv_slices = sum(work) / w512
    taps = [tap_counts(c.geom, c.n_subsets) for c in cases]
    tap_total = sum(float(sum(t[n % c.n_subsets] for n in range(n_iter))) for t, c in zip(taps, cases))
    peaks, peak_kind = load_peaks()
    t_step = float(np.mean(step_ms)) / 1e3
    achieved = 2 * 4 * tap_total / t_step / 1e9
    out = {
        "value": value, "unit": "slices/s", "ms_per_step": t_max / steps, "steps": steps, "warmup": warmup,
        "config": dict(BATCH_WORKLOAD if stack <= 0 else
                       dict(BATCH_WORKLOAD, workload=f"batched stack of {stack} 512^2 slices (a smaller case)",
                            slices=f"{stack} x 512^2 (800 views x 738 ch)", sub_iterations=n_iter),
                       l2="flushed between timed steps (512 MiB write)",
                       launch_shape={"view_groups_per_tile": tune["groups"] or "default rule",
                                     "autotuned_ms_per_iter": tune["ms_per_iter"],
                                     "default_ms_per_iter": tune["default_ms_per_iter"]}),
        "slices_512_equivalent_per_s": equiv_slices * ws * steps / (t_max / 1e3),
        "us_per_512_equivalent_slice_sub_iteration": t_step * 1e6 / (equiv_slices * n_iter),
        "gray_per_s": 2.0 * tap_total / t_step / 1e9,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "kernel": "batch set-up + k_recon_pb (one graph replay)",
                     "algorithmic_bytes": "4 B x (reprojection taps + backprojection residual reads), "
                                          "served from L1/L2",
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
        "e2e": {"value": len(cases) * ws * len(e2e_ms) / (e2e_t / 1e3), "unit": "slices/s",
                "h2d_bytes_per_step": int(sum(t.numel() * 4 for t in hp + hw)),
                "d2h_bytes_per_step": int(sum(t.numel() * 4 for t in hi))},
        "parity": "tests/test_gpu_bench_parity.py: the batch kernel at 512^2, 384^2 and 256^2 against the "
                  "oracle (40 sub-iterations) and one-slice runs (500)",
        "clocks": clk.summary(),
        "gpu_launches_per_step": 2 + 3 * len(cases),
    }
    batch.close()
    for pl in plans:
        pl.close()
    return out


def run_batched(args):
    """Batched workload on its own: all slices of the stack reconstructed per step."""
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1903_10088_gb300 import mvct

    mvct.lib()
    leg = batched_leg(args, dev, ws, args.steps, args.warmup)
    line = dict({"metric": f"slices/s of the batched stack at {leg['config']['sub_iterations']} OS-TV iters "
                           "(plain start)",
                 "n_gpus": ws, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                 "dtype": "f32", "data": "synthetic", "gpu_launches": leg["gpu_launches_per_step"] * args.steps},
                **leg)
    line["config"] = dict(line["config"], parallelism=f"replicas x{ws}, one stack per GPU per step")
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_subsets(args):
    """The thinning sweep of the paper's Table I on one 512^2 slice: seconds per
    slice (FBP start + 500 sub-iterations) and the objective reached, for
    S in {1, 2, 5, 10, 20, 40}."""
    import torch

    from paper_1903_10088_gb300 import mvct

    mvct.lib()
    dev = torch.device("cuda", 0)
    case = ph.make_case("full", SEED0)
    g = case.geom
    p = torch.from_numpy(case.p).to(dev)
    w = torch.from_numpy(case.w).to(dev)
    img = torch.empty((g.n, g.n), device=dev)
    rows = []
    for S in (1, 2, 5, 10, 20, 40):
        with mvct.Plan(g, S) as plan:
            def step():
                plan.fbp(p, out=img)
                return plan.recon(p, w, case.beta, case.n_iter, img=img, init_from_input=True)
            for _ in range(args.warmup):
                step()
            torch.cuda.synchronize()
            ms = []
            for _ in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                step()
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            psi = float(plan.objective(img, p, w, case.beta, case.tv_eps).cpu())
        rows.append({"subsets": S, "s_per_slice": float(np.mean(ms)) / 1e3, "psi_500": psi})
    print(json.dumps({"metric": "s/slice at 500 sub-iterations vs subsets (paper Table I thinning set)",
                      "unit": "s/slice", "higher_is_better": False, "dtype": "f32", "data": "synthetic",
                      "config": dict(WORKLOAD, workload="one 512^2 slice, FBP start, 500 sub-iterations per S"),
                      "rows": rows, "steps": args.steps, "warmup": args.warmup}))
    return 0


def run_ops(args):
    """Per-operator timing of the C ABI (CUDA events, warm caches, seeded random
    inputs): mvct_forward / mvct_back on one subset and on all views,
    mvct_tv_grad, mvct_objective, mvct_fbp, and the warm-start network (forward,
    and one Adam step, on a batch of --cnn-batch images). One JSON object; also
    the command that the operators' profiler captures run."""
    import torch

    from paper_1903_10088_gb300 import mvct

    mvct.lib()

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    g = ph.Geometry(n=args.n, n_views=args.views, n_channels=args.channels)
    rng = np.random.default_rng(0)
    img = torch.from_numpy(rng.uniform(0, 0.1, (g.n, g.n)).astype(np.float32)).cuda()
    sino = torch.from_numpy(rng.uniform(0, 1, (g.n_views, g.n_channels)).astype(np.float32)).cuda()
    w = torch.from_numpy(rng.uniform(0.1, 1, (g.n_views, g.n_channels)).astype(np.float32)).cuda()
    Vs = g.n_views // args.subsets_ops
    sub = sino[:Vs].contiguous()
    out = {"workload": "operators of the C ABI on seeded random inputs",
           "geometry": dict(n=g.n, views=g.n_views, channels=g.n_channels, subsets=args.subsets_ops), "ms": {}}
    ops = args.ops.split(",")
    with mvct.Plan(g, args.subsets_ops) as plan:
        q_sub = torch.empty((Vs, g.n_channels), device="cuda")
        q_all = torch.empty((g.n_views, g.n_channels), device="cuda")
        b = torch.empty((g.n, g.n), device="cuda")
        if "forward" in ops:
            out["ms"]["forward_subset"] = timed(lambda: plan.forward(img, 0, out=q_sub), args.reps)
            out["ms"]["forward_all"] = timed(lambda: plan.forward(img, -1, out=q_all), args.reps)
        if "back" in ops:
            out["ms"]["back_subset"] = timed(lambda: plan.back(sub, 0, out=b), args.reps)
            out["ms"]["back_all"] = timed(lambda: plan.back(sino, -1, out=b), args.reps)
        if "tv" in ops:
            out["ms"]["tv_grad"] = timed(lambda: plan.tv_grad(img, 1e-6), args.reps)
        if "objective" in ops:
            out["ms"]["objective"] = timed(lambda: plan.objective(img, sino, w, 1e-3, 1e-6), args.reps)
        if "fbp" in ops:
            out["ms"]["fbp"] = timed(lambda: plan.fbp(sino, out=b), args.reps)
    if "cnn" in ops:
        from paper_1903_10088_gb300 import warmstart as wst

        N = args.cnn_batch
        x = torch.from_numpy(rng.uniform(0, 0.1, (N, g.n, g.n)).astype(np.float32)).cuda()
        y = 0.9 * x
        xo = torch.empty_like(x)
        net = wst.CNN(N, g.n, g.n, wst.init_params(0))
        out["ms"]["cnn_forward"] = timed(lambda: net.forward(x, out=xo), args.reps)
        out["ms"]["cnn_train_step"] = timed(lambda: net.train_step(x, y, 1e-5), args.reps)
        net.close()
        flops = 2.0 * N * g.n * g.n * (6 * 9 * 32 * 32 + 2 * 9 * 32)
        out["cnn_batch"] = N
        out["cnn_forward_tflops"] = flops / out["ms"]["cnn_forward"] / 1e9
        out["cnn_train_tflops"] = 3 * flops / out["ms"]["cnn_train_step"] / 1e9
    print(json.dumps(out))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-sub-iters", type=int, default=40,
                    help="oracle sub-iterations timed per reference sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-warm", action="store_true", help="skip the warm-started batched form")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched uneven stack")
    ap.add_argument("--stack-slices", type=int, default=0,
                    help="--workload batched: a stack of this many 512^2 slices instead of the uneven stack")
    ap.add_argument("--stack-iters", type=int, default=0,
                    help="--workload batched: sub-iterations per step instead of 500")
    ap.add_argument("--ref-threads", type=int, default=0,
                    help="oracle threads for the whole-slice CPU timing (0: every host core)")
    ap.add_argument("--workload", choices=["plain", "batched", "subsets", "ops"], default="plain")
    ap.add_argument("--ops", default="forward,back,tv,objective,fbp,cnn", help="--workload ops: which operators")
    ap.add_argument("--reps", type=int, default=20, help="--workload ops: timed calls per operator")
    ap.add_argument("--cnn-batch", type=int, default=16, help="--workload ops: images per network call")
    ap.add_argument("--n", type=int, default=512, help="--workload ops: image side")
    ap.add_argument("--views", type=int, default=800, help="--workload ops: views")
    ap.add_argument("--channels", type=int, default=738, help="--workload ops: channels")
    ap.add_argument("--subsets-ops", type=int, default=20, help="--workload ops: subsets")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "subsets":
        return run_subsets(args)
    if args.workload == "ops":
        return run_ops(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
