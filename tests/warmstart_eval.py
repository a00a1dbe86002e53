"""Evaluation of the learned warm start on held-out seeded phantoms.

    python tests/warmstart_eval.py [--weights W] [--seeds 200] [--Ks 25 50 100]
                                   [--oracle-seeds 8] [--out result.json]

For every held-out seed: the plain form (FBP start, 500 sub-iterations), FBP
start + K and network start + K sub-iterations (batched reconstructions on the
GPU), judged by the objective Psi (GPU FP64 reduction for every seed; the FP64
CPU oracle's objective for the first --oracle-seeds seeds, which also checks
the GPU objective) and by image relative L2 against the plain result and the
phantom. Prints one JSON summary line.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
for _p in (os.path.dirname(HERE), HERE):
    if _p not in sys.path:
        sys.path.insert(0, _p)

import oracle_jobs  # noqa: E402


def main(argv=None):
    from paper_1903_10088_gb300 import warmstart as ws

    ap = argparse.ArgumentParser()
    ap.add_argument("--weights", default=None)
    ap.add_argument("--seeds", type=int, default=200)
    ap.add_argument("--seed0", type=int, default=ws.HELDOUT_SEED0)
    ap.add_argument("--Ks", type=int, nargs="+", default=[25, 50, 100])
    ap.add_argument("--oracle-seeds", type=int, default=8)
    ap.add_argument("--lambda0", type=float, default=None, help="lambda0 of the network-started runs")
    ap.add_argument("--width", type=int, default=48)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    seeds = list(range(args.seed0, args.seed0 + args.seeds))
    # the worker pool is spawned before the first CUDA call
    ex = cf.ProcessPoolExecutor(args.workers, mp_context=mp.get_context("spawn"))
    t0 = time.perf_counter()
    ct = list(ex.map(oracle_jobs.case_and_truth, seeds, chunksize=2))
    cases, truth = [c for c, _ in ct], [t for _, t in ct]
    t_gen = time.perf_counter() - t0

    import torch

    dev = torch.device("cuda", 0)
    cnn = ws.CNN(16, cases[0].geom.n, cases[0].geom.n, ws.load_weights(args.weights))
    warm = {} if args.lambda0 is None else {"lambda0": args.lambda0}
    t0 = time.perf_counter()
    res = ws.evaluate(cnn, cases, args.Ks, dev, width=args.width, warm_opts=warm, keep_images=args.oracle_seeds,
                      truth=truth)
    t_gpu = time.perf_counter() - t0
    cnn.close()

    # FP64 oracle objective for the first seeds: plain and every network-started K
    jobs = []
    for r in res[:args.oracle_seeds]:
        for key in ["plain"] + [f"cnn_K{K}" for K in args.Ks] + [f"fbp_K{K}" for K in args.Ks]:
            jobs.append((r["seed"], key, r["images"][key]))
    vals = list(ex.map(oracle_jobs.full_case_objective, [j[0] for j in jobs], [j[2] for j in jobs]))
    ex.shutdown()
    orc = {}
    for (seed, key, _), v in zip(jobs, vals):
        orc.setdefault(seed, {})[key] = v
    gpu_vs_oracle = []
    for r in res[:args.oracle_seeds]:
        o = orc[r["seed"]]
        r["oracle_psi"] = o
        for key, v in o.items():
            gpu = r["psi_plain"] if key == "plain" else r[f"psi_{key}"]
            gpu_vs_oracle.append(abs(gpu - v) / abs(v))
        del r["images"]
    summary = ws.summarize(res, args.Ks)
    oracle_gap = {}
    for K in args.Ks:
        for name in ("cnn", "fbp"):
            g = [(orc[r["seed"]][f"{name}_K{K}"] - orc[r["seed"]]["plain"]) / orc[r["seed"]]["plain"]
                 for r in res[:args.oracle_seeds]]
            if g:
                oracle_gap[f"{name}_K{K}"] = dict(gap_median=float(np.median(g)), gap_max=float(np.max(g)))
    truth_rel = {f"{name}_K{K}": float(np.median([r[f"rel_truth_{name}_K{K}"] for r in res]))
                 for name in ("fbp", "cnn") for K in args.Ks}
    line = dict(seeds=[seeds[0], seeds[-1]], Ks=args.Ks, warm_opts=warm, gpu_objective=summary,
                oracle_objective=oracle_gap, oracle_seeds=args.oracle_seeds,
                gpu_vs_oracle_psi_max_rel=float(max(gpu_vs_oracle)) if gpu_vs_oracle else None,
                rel_l2_truth_median=truth_rel, host_gen_s=t_gen, gpu_eval_s=t_gpu)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(dict(summary=line, per_seed=res), f, indent=1)
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
