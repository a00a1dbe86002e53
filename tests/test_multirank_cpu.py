"""The N>1 benchmark path on CPU: two gloo ranks (world size 2) shard the slices
(no data-path collective), synchronise with the barrier and take the maximum
time over ranks, exactly as bench.py does under torchrun."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", init_method="env://")
    ws, r, local = bench.dist_env()
    seeds = bench.slice_seeds(r, 3)
    bench.barrier()
    t = bench.max_over_ranks(float(10 * (r + 1)), device=None)
    q.put((r, ws, local, seeds, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, l0, s0, t0), (r1, ws1, l1, s1, t1) = out
    assert (r0, r1) == (0, 1) and ws0 == ws1 == 2 and (l0, l1) == (0, 1)
    assert not set(s0) & set(s1)          # disjoint slices per rank
    assert t0 == t1 == 20.0               # maximum over ranks
