"""Element-wise oracle parity for exactly the configurations the benchmark times.

A. The plain form: 512^2 over 40 cm, 800 views x 738 channels, 20 subsets, 500
   sub-iterations, beta = 1e-3, started from the FBP image (Sec. 4.5 comparison
   image; Sec. 3.3.2: the start image is part of the method). The start is the
   FP64 oracle's FBP rounded to FP32, handed to both sides as the same host
   array; the GPU runs mvct_recon(init_from_input = 1), the oracle recon(init=).
B. The batch kernel (the parameter-space persistent launch that the warm-started
   form uses): three slices of the uneven stack's sizes (512^2/800x738,
   384^2/600x552, 256^2/400x368) in one launch, started from their FBP images
   with the warm chain's lambda0 (0.04); each slice against the
   oracle after 40 sub-iterations, and against a one-slice mvct_recon of 500
   sub-iterations replaying the batch's own lambda sequence.

The oracle runs (about a minute for A on one core) execute in spawned worker
processes while the GPU runs. Tolerances: 1e-4 relative L2 for FP32 images after
the fixed count, the lambda sequence (Eq. 4-5) identical; where a lambda
decision flips on an FP32 rounding of Phi, the run is repeated with the
oracle's own lambda sequence replayed and the flips are reported.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest
import torch

import oracle
from paper_1903_10088_gb300 import phantom as ph

pytestmark = pytest.mark.gpu

SEED = 100
N_ITER = 500
BETA = 1e-3
RTOL_IMG = 1e-4
WARM_LAMBDA0 = 0.04   # warmstart.FAST_LAMBDA0
BATCH_GEOMS = (ph.GEOM_512, ph.GEOM_384, ph.GEOM_256)
BATCH_SEEDS = (50200, 50201, 50202)
BATCH_ORACLE_ITERS = 40


def rel(a, b):
    a, b = np.ravel(np.asarray(a, dtype=np.float64)), np.ravel(np.asarray(b, dtype=np.float64))
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def mvct():
    from paper_1903_10088_gb300 import build, mvct

    build.build()
    mvct.lib()
    return mvct


@pytest.fixture(scope="module")
def pool():
    import oracle_jobs  # noqa: F401  (importable by the spawned workers)

    oracle.build()
    ex = cf.ProcessPoolExecutor(max_workers=4, mp_context=mp.get_context("spawn"))
    yield ex
    ex.shutdown(cancel_futures=True)


def test_plain_form_from_fbp_start_matches_oracle(mvct, pool):
    import oracle_jobs

    c = ph.make_case("full", SEED, beta=BETA, n_iter=N_ITER)
    start = oracle_jobs.fbp_start(c)
    fut = pool.submit(oracle_jobs.full_case_recon_from, SEED, BETA, N_ITER, start)
    p = torch.from_numpy(c.p).cuda()
    w = torch.from_numpy(c.w).cuda()
    with mvct.Plan(c.geom, c.n_subsets) as plan:
        img, res = plan.recon(p, w, BETA, N_ITER, img=torch.from_numpy(start).cuda(), init_from_input=True)
        adaptive = img.double().cpu().numpy()
        ref_img, ref_phi, ref_lam = fut.result(timeout=1200)
        flips = int(np.sum(res.lam != ref_lam))
        img2, res2 = plan.recon(p, w, BETA, N_ITER, img=torch.from_numpy(start).cuda(), init_from_input=True,
                                lambda_schedule=ref_lam)
        replay = img2.double().cpu().numpy()
    e_adapt, e_replay = rel(adaptive, ref_img), rel(replay, ref_img)
    print(f"plain form, FBP start: lambda flips {flips}, adaptive rel L2 {e_adapt:.2e}, "
          f"replay rel L2 {e_replay:.2e}, loop {res.loop_ms:.1f} ms")
    assert e_replay < RTOL_IMG
    assert np.allclose(res2.phi, ref_phi, rtol=1e-4)
    assert np.allclose(res.phi[:50], ref_phi[:50], rtol=1e-4)
    if flips == 0:
        assert e_adapt < RTOL_IMG


def test_bench_start_image_is_the_fbp_the_oracle_computes(mvct):
    """The benchmark's start image is the GPU FBP of the case: it equals the
    oracle's FBP within the FBP tolerance, so test A's start stands for it."""
    import oracle_jobs

    c = ph.make_case("full", SEED, beta=BETA)
    with mvct.Plan(c.geom, c.n_subsets) as plan:
        img = plan.fbp(torch.from_numpy(c.p).cuda()).double().cpu().numpy()
    assert rel(img, oracle_jobs.fbp_start(c)) < 1e-4


def test_batch_kernel_full_sizes_match_oracle_and_one_slice_runs(mvct, pool):
    import oracle_jobs

    cases = [ph.make_case("full", s, geom=g, beta=BETA) for s, g in zip(BATCH_SEEDS, BATCH_GEOMS)]
    starts = [oracle_jobs.fbp_start(c) for c in cases]
    futs = [pool.submit(oracle_jobs.case_recon_from, s, g, BETA, BATCH_ORACLE_ITERS, st, WARM_LAMBDA0)
            for s, g, st in zip(BATCH_SEEDS, BATCH_GEOMS, starts)]
    plans = [mvct.Plan(c.geom, c.n_subsets) for c in cases]
    p = [torch.from_numpy(c.p).cuda() for c in cases]
    w = [torch.from_numpy(c.w).cuda() for c in cases]
    try:
        # 40 sub-iterations against the oracle
        imgs = [torch.from_numpy(st).cuda() for st in starts]
        with mvct.Batch(plans) as b:
            b.bind(p, w, [BETA] * 3, imgs, N_ITER, init_from_input=True, lambda0=WARM_LAMBDA0)
            b.run(BATCH_ORACLE_ITERS)
            st40 = [b.stats(i, BATCH_ORACLE_ITERS) for i in range(3)]
            got40 = [im.double().cpu().numpy() for im in imgs]
            # 500 sub-iterations, then the same slices one at a time
            imgs = [torch.from_numpy(st).cuda() for st in starts]
            b.bind(p, w, [BETA] * 3, imgs, N_ITER, init_from_input=True, lambda0=WARM_LAMBDA0)
            b.run(N_ITER)
            st500 = [b.stats(i, N_ITER) for i in range(3)]
            got500 = [im.double().cpu().numpy() for im in imgs]
        for k, (c, f) in enumerate(zip(cases, futs)):
            ref_img, ref_phi, ref_lam = f.result(timeout=1200)
            e = rel(got40[k], ref_img)
            print(f"batch slice {k} ({c.geom.n}^2): {BATCH_ORACLE_ITERS} sub-iterations vs oracle rel L2 {e:.2e}, "
                  f"lambda flips {int(np.sum(st40[k].lam != ref_lam))}")
            assert np.array_equal(st40[k].lam, ref_lam)
            assert np.allclose(st40[k].phi, ref_phi, rtol=1e-5)
            assert e < RTOL_IMG
        for k, c in enumerate(cases):
            one, res = plans[k].recon(p[k], w[k], BETA, N_ITER, img=torch.from_numpy(starts[k]).cuda(),
                                      init_from_input=True, lambda0=WARM_LAMBDA0)
            flips = int(np.sum(res.lam != st500[k].lam))
            if flips:
                one, res = plans[k].recon(p[k], w[k], BETA, N_ITER, img=torch.from_numpy(starts[k]).cuda(),
                                          init_from_input=True, lambda_schedule=st500[k].lam)
            e = rel(got500[k], one.double().cpu().numpy())
            print(f"batch slice {k} ({c.geom.n}^2): {N_ITER} sub-iterations vs one-slice run rel L2 {e:.2e}, "
                  f"lambda flips {flips}")
            assert e < RTOL_IMG
    finally:
        for pl in plans:
            pl.close()
