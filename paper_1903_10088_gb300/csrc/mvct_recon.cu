// The ordered-subset TV loop as one persistent cooperative kernel, for one
// slice (mvct_recon) or many slices of uneven geometry at once (mvct_batch_*).
//
// The grid is partitioned into block groups; each group reconstructs its own
// list of slices with group-local barriers (one slice: one group of all blocks).
// Per sub-iteration n of a slice (subset s = n mod S; Eq. 3-5, Sec. 3.3.2, 3.4,
// 4.2):
//   phase F  one warp per ray of the subset: Joseph reprojection of mu^(n),
//            residual r = q - p, prescaled weighted residual e = scale*w*r,
//            FP64 partial sums of r^2 per block
//   barrier
//   lambda   a block without a phase-B item reduces the partials in a fixed
//            order and publishes Phi_n (a flag, no barrier); every block derives
//            the same lambda_n (Eq. 4-5) and best-iterate decision from it when
//            its first update needs it (with no such block, every block reduces
//            the partials itself, in the same order)
//   phase B  32x32 pixel tiles: splat of the matched backprojection of e (view
//            groups of one tile merged in group order), TV_eps gradient,
//            surrogate-preconditioned step, clamp at 0, write mu^(n+1) and its
//            transpose
//   barrier
// Images ping-pong between two zero-row-padded plan buffers; the transposes let
// y-driven rays read contiguous memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <queue>
#include <vector>

#include "mvct_plan.h"

namespace mvct {

// Wait until flag == stamp (bounded like the group barrier: tight polls, every
// 64th also reads *err and the timer, sleeps after 4096). Thread 0 only.
__device__ __forceinline__ bool wait_flag(const unsigned int *flag, unsigned int stamp, int *err,
                                          unsigned long long timeout_ns, unsigned long long spin_cap)
{
    if (ld_acquire(flag) == stamp) return true;
    unsigned long long spins = 0, t0 = 0;
    while (ld_acquire(flag) != stamp) {
        ++spins;
        if ((spins & 63u) == 0) {
            if (*(volatile int *)err) return false;
            if (spins == 64) {
                t0 = global_ns();
            } else if (spins > spin_cap || global_ns() - t0 > timeout_ns) {
                atomicExch(err, 1);
                return false;
            }
            if (spins >= 4096) __nanosleep(64);
        }
    }
    return true;
}

// Shared state of one block of the loop kernel.
struct LoopShared {
    double warp[kWarps];
    double lambda, phi_prev, best_pass, pass_prev;
    double phi_n, pass_n;          // Phi_n and the pass sum of the current sub-iteration
    double phi_old, pass_last;     // Phi_{n-S} and the last complete pass sum (n >= S)
    long long best_n;
    float tau;
    int best_flag, ok;
    float acc[kWarps][kAccFloats]; // warp-private splat tiles
    float4 stage[kWarps][32];      // warp-private ray staging
    int4 win[kWinBatch];           // channel windows of the splat's views
    SliceDesc sd;                  // batch launches: the current slice
    GroupDesc grp;                 // batch launches: this block's group
};

// All n_iter sub-iterations of one slice by the blocks of one group (lb = this
// block's index in the group, bk = the group's barrier count so far). Returns
// false if the block must leave the kernel (a wait gave up).
template <typename TS, class SD, class GD>
__device__ __forceinline__ bool run_slice(const SD &sd, const GD &grp, const LoopArgs &a, int lb,
                                          unsigned int &bk, LoopShared &sh, bool timer,
                                          unsigned long long &t_f, unsigned long long &t_b,
                                          unsigned long long &t_mark)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *err = &a.gbar->err;
    const Geo &g = sd.g;
    mvct_recon_state *st = sd.st;
    if (threadIdx.x == 0) {
        sh.lambda = st->lambda;
        sh.phi_prev = st->phi_prev;
        sh.best_pass = st->best_pass;
        sh.best_n = st->best_n;
        sh.pass_prev = st->pass_prev;
    }
    __syncthreads();
    const long long n0 = st->n_done;
    const int Rs = g.Vs * g.C;
    const float S_f = (float)g.S;
    constexpr bool F32 = std::is_same<TS, float>::value;
    const float4 *rays = sd.rays;
    // measured p and w as stored (FP32, or the 16-bit copies)
    const TS *pp = F32 ? (const TS *)sd.p : (const TS *)sd.hp;
    const TS *ww = F32 ? (const TS *)sd.w : (const TS *)sd.hw;
    float4 *e4 = sd.e4;
    

    for (int it = 0; it < a.n_iter; ++it) {
        const long long n = n0 + it;
        const int s = sd.sorder ? sd.sorder[(int)(n % g.S)] : (int)(n % g.S);
        const bool odd = (it & 1) != 0;
        const float *cur = odd ? sd.mu1 : sd.mu0;
        const float *curT = odd ? sd.muT1 : sd.muT0;
        float *nxt = odd ? sd.mu0 : sd.mu1;
        float *nxtT = odd ? sd.muT0 : sd.muT1;
        // the copies the reprojection reads: the FP32 images themselves, or their
        // 16-bit copies (the FP32 iterate is the master for TV and the update)
        const TS *pcur = F32 ? (const TS *)cur : (const TS *)(odd ? sd.hm1 : sd.hm0);
        const TS *pcurT = F32 ? (const TS *)curT : (const TS *)(odd ? sd.hmT1 : sd.hmT0);
        TS *pnxt = F32 ? (TS *)nxt : (TS *)(odd ? sd.hm0 : sd.hm1);
        TS *pnxtT = F32 ? (TS *)nxtT : (TS *)(odd ? sd.hmT0 : sd.hmT1);
        const unsigned int stamp = (unsigned int)it + 1u;

        // ---- phase F: reprojection, residual, square difference ---------
        double acc_phi = 0.0;
        {
            const int gw0 = lb * kWarps + warp, GW = grp.nblocks * kWarps;
            // the next ray's table entry and data are fetched while this ray is walked
            float4 r_nx = make_float4(0.f, 0.f, 0.f, 1.f);
            int range_nx = 0;
            float p_nx = 0.f, w_nx = 0.f;
            if (gw0 < Rs) {
                const int k = gw0 / g.C;
                const size_t rv = (size_t)(s + k * g.S) * g.C + (gw0 - k * g.C);
                r_nx = __ldg(&rays[rv]);
                range_nx = __ldg(sd.ray_range + rv);
                if (lane == 0) {
                    p_nx = ldv<true>(pp + rv);
                    w_nx = ldv<true>(ww + rv);
                }
            }
            for (int ray = gw0; ray < Rs; ray += GW) {
                const float4 r = r_nx;
                const int range = range_nx;
                const float pv = p_nx, wv = w_nx;
                const int nray = ray + GW;
                if (nray < Rs) {
                    const int k = nray / g.C;
                    const size_t rv = (size_t)(s + k * g.S) * g.C + (nray - k * g.C);
                    r_nx = __ldg(&rays[rv]);
                    range_nx = __ldg(sd.ray_range + rv);
                    if (lane == 0) {
                        p_nx = ldv<true>(pp + rv);
                        w_nx = ldv<true>(ww + rv);
                    }
                }
                const float q_ray = joseph_warp<false, TS>(pcur, pcurT, g.n, g.pc, r, range, lane);
                if (lane == 0) {
                    const float res = q_ray - pv;
                    const float ev = a.poisson ? wv - expf(-q_ray) : wv * res;
                    e4[ray] = make_float4(r.x, r.y, r.z * ev, r.w);
                    acc_phi += (double)res * (double)res;
                }
            }
        }
        if (lane == 0) sh.warp[warp] = acc_phi;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kWarps; ++k) t += sh.warp[k];
            grp.partials[lb] = t;
        }
        if (!group_sync(grp.count, err, bk, grp.nblocks, (bk == 0 && a.debug_unreachable) ? 1u : 0u,
                        a.timeout_ns, a.spin_cap))
            return false;
        ++bk;
        if (timer) {
            const unsigned long long now = global_ns();
            t_f += now - t_mark;
            t_mark = now;
        }

        // ---- adaptive lambda (Eq. 4-5) and best iterate (Sec. 4.2) ------
        // Only the update of phase B needs lambda. If the group has a block
        // without a phase-B item, that block (the reducer) sums the partials
        // right away and publishes Phi_n and the pass sum; the other blocks read
        // them when their first update needs them. Otherwise every block sums the
        // partials itself after its first splat. Either way the sums are taken in
        // the same fixed order, so every block derives the same lambda_n and
        // best-iterate decision.
        const int slot_n = (int)(n % g.S);
        const bool full = n >= g.S - 1, seen_pass = n >= g.S;
        const int reducer = sd.reducer;
        // the block that stores Phi_n into the ring (after the closing barrier)
        const int ring_writer = reducer >= 0 ? reducer : 0;
        PhiPub *pub = phi_pub(grp.count);
        const unsigned int pub_stamp = bk;
        // all threads: Phi_n and the pass sum Phi_{n-S+1} + ... + Phi_n into sh
        auto reduce_phi = [&]() {
            {
                constexpr int L = (MVCT_MAX_RECON_GRID + kThreads - 1) / kThreads;
                double v[L];
#pragma unroll
                for (int u = 0; u < L; ++u) {
                    const unsigned int b = threadIdx.x + u * kThreads;
                    v[u] = b < (unsigned int)grp.nblocks ? grp.partials[b] : 0.0;
                }
                double t = 0.0;
#pragma unroll
                for (int u = 0; u < L; ++u) t += v[u];
                t = warp_sum(t);
                if (lane == 0) sh.warp[warp] = t;
            }
            __syncthreads();
            if (warp == 0) {
                double phi = 0.0;
                for (int k = 0; k < kWarps; ++k) phi += sh.warp[k];
                // the last S values of Phi live in the slice's state (global
                // memory), slot k mod S for sub-iteration k. Slot n mod S still
                // holds Phi_{n-S}: the ring writer stores Phi_n only after this
                // sub-iteration's closing barrier, so no block reads a slot while
                // it is written; the barriers order the earlier stores.
                double pass = 0.0, pass_last = 0.0;
                if (full)
                    for (int k = lane; k < g.S; k += 32) {
                        const double v = st->phi_ring[k];
                        pass += (k == slot_n) ? phi : v;
                        pass_last += v;
                    }
                pass = warp_sum(pass);
                pass_last = warp_sum(pass_last);
                if (lane == 0) {
                    sh.phi_n = phi;
                    sh.pass_n = pass;
                    sh.phi_old = seen_pass ? st->phi_ring[slot_n] : 0.0;
                    sh.pass_last = seen_pass ? pass_last : 0.0;
                }
            }
            __syncthreads();
        };
        // Eq. 4-5 and the best-iterate decision from sh.phi_n, sh.pass_n
        auto apply_lambda = [&]() {
            if (threadIdx.x == 0) {
                const double phi = sh.phi_n, pass = sh.pass_n;
                double lam;
                if (sd.sched) {
                    lam = sd.sched[it];
                } else if (n == 0) {
                    lam = a.lambda0;
                } else {
                    // the two square differences this rule compares at n, if any
                    bool decide = false;
                    double now = 0.0, before = 0.0;
                    if (a.lambda_rule == MVCT_LAMBDA_PASS_SLIDING) {
                        decide = seen_pass;
                        now = phi;
                        before = sh.phi_old;
                    } else if (a.lambda_rule == MVCT_LAMBDA_PASS) {
                        decide = n >= 2 * (long long)g.S && slot_n == 0;
                        now = sh.pass_last;
                        before = sh.pass_prev;
                    } else {
                        decide = true;
                        now = phi;
                        before = sh.phi_prev;
                    }
                    lam = sh.lambda;
                    if (decide) {
                        if (now < before) lam += a.dup;
                        else if (now > before) lam -= a.ddown;
                        if (lam < a.lmin) lam = a.lmin;
                    }
                }
                if (a.lambda_rule == MVCT_LAMBDA_PASS && seen_pass && slot_n == 0) sh.pass_prev = sh.pass_last;
                sh.lambda = lam;
                sh.phi_prev = phi;
                int bf = 0;
                if (full && pass < sh.best_pass) {
                    sh.best_pass = pass;
                    sh.best_n = n;
                    bf = 1;
                }
                sh.best_flag = bf;
                sh.tau = (float)(a.kappa * lam);
                if (lb == 0) {
                    sd.phi_hist[it] = phi;
                    sd.lam_hist[it] = lam;
                }
            }
            __syncthreads();
        };
        // lambda_n in this block: from the reducer's publication, or reduced here.
        // False if the wait for the publication gave up.
        auto obtain_lambda = [&]() -> bool {
            if (reducer < 0) {
                reduce_phi();
            } else {
                if (threadIdx.x == 0) {
                    const bool ok = wait_flag(&pub->stamp, pub_stamp, err, a.timeout_ns, a.spin_cap);
                    if (ok) {
                        sh.phi_n = __ldcg(&pub->phi);
                        sh.pass_n = __ldcg(&pub->pass);
                        sh.phi_old = __ldcg(&pub->phi_old);
                        sh.pass_last = __ldcg(&pub->pass_last);
                    }
                    sh.ok = ok;
                }
                __syncthreads();
                if (!sh.ok) return false;
            }
            apply_lambda();
            return true;
        };
        if (lb == reducer) {
            reduce_phi();
            if (threadIdx.x == 0) {
                pub->phi = sh.phi_n;
                pub->pass = sh.pass_n;
                pub->phi_old = sh.phi_old;
                pub->pass_last = sh.pass_last;
                st_release(&pub->stamp, pub_stamp);
            }
            apply_lambda();
        } else if (reducer < 0) {
            // every block reduces: start moving the partials and the ring into L1
            for (int b = threadIdx.x * 16; b < grp.nblocks; b += kThreads * 16) prefetch_l1(grp.partials + b);
            if (full && threadIdx.x * 16 < g.S) prefetch_l1(st->phi_ring + threadIdx.x * 16);
        }
        bool lam_done = lb == reducer;

        // ---- phase B: tile splat (estimation) + TV + preconditioned step
        // Item (tile t, view group h of the tile's Ht groups): group h holds the
        // subset rows h, h + Ht, h + 2Ht, ... Groups h < Ht-1 publish a partial
        // tile in slot slot0 + h; group Ht-1 (the owner) adds the partials in
        // group order and updates the tile. Owners only wait on items that never
        // wait (non-owner items come first in every block's sequence).
        float *best = sd.best;
        const int C = g.C;
        const float beta = sd.beta;
        auto process_item = [&](int t, int h, int Ht, int slot0) -> bool {
            const bool owner = h == Ht - 1;
            const int i_lo = (t / sd.tiles_x) * kTile, j_lo = (t % sd.tiles_x) * kTile;
            const int wpos = splat_views(g, sd.views, s, h, g.Vs, Ht, nullptr, i_lo, j_lo, sh.acc, sh.stage, sh.win,
                                         [e4, C](int k, int) { return StageE4{e4 + (size_t)k * C}; });
            float part_val[4];
            tile_sums(sh.acc, kWarps, wpos, part_val);

            if (!owner) {
                const size_t slot = (size_t)slot0 + h;
                float *dst = sd.tile_part + slot * (kTile * kTile);
#pragma unroll
                for (int u = 0; u < 4; ++u) __stcg(dst + threadIdx.x + u * kThreads, part_val[u]);
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    st_release(sd.tile_flag + slot, stamp);
                }
                __syncthreads(); // sh.acc is zeroed by the next item
                return true;
            }
            if (!lam_done) {
                if (!obtain_lambda()) return false;
                lam_done = true;
            }
            const float tau = sh.tau;
            const bool keep_best = sh.best_flag && best;

            if (threadIdx.x == 0) {
                bool ok = true;
                for (int hh = 0; hh < Ht - 1 && ok; ++hh)
                    ok = wait_flag(sd.tile_flag + (size_t)slot0 + hh, stamp, err, a.timeout_ns, a.spin_cap);
                sh.ok = ok;
            }
            __syncthreads();
            if (!sh.ok) return false;

            // partial tiles of groups 0..Ht-2, added in group order (four pixels' loads
            // in flight per group)
            float gsum[4] = {0.f, 0.f, 0.f, 0.f};
            for (int hh = 0; hh < Ht - 1; ++hh) {
                const float *src = sd.tile_part + ((size_t)slot0 + hh) * (kTile * kTile) + threadIdx.x;
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = __ldcg(src + u * kThreads);
#pragma unroll
                for (int u = 0; u < 4; ++u) gsum[u] += v[u];
            }
            float *tile = sh.acc[0]; // reused for the transposed write-out
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = threadIdx.x + u * kThreads;
                const int ii = idx >> 5, jj = idx & 31;
                const float gs = gsum[u] + part_val[u];
                const int i = i_lo + ii, j = j_lo + jj;
                float nm = 0.f;
                if (i < g.n && j < g.n) {
                    const size_t r = (size_t)i * g.n + j;
                    const float m = cur[r];
                    const float d = __ldg(sd.D + r);
                    if (keep_best) best[r] = m;
                    if (d > 0.f) {
                        const float tg = tv_grad_pixel<false>(cur, g.n, i, j, a.eps, nullptr);
                        nm = fmaxf(0.f, m - tau * d * fmaf(S_f, gs, beta * tg));
                    }
                    nxt[r] = nm;
                    if constexpr (!F32) pnxt[r] = to_storage<TS>(nm);
                }
                part_val[u] = nm;
            }
            __syncthreads(); // every warp has finished reading sh.acc
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = threadIdx.x + u * kThreads;
                tile[(idx >> 5) * kAccStride + (idx & 31)] = part_val[u];
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = threadIdx.x + u * kThreads;
                const int jj = idx >> 5, ii = idx & 31; // transposed: row of muT = column j
                const int i = i_lo + ii, j = j_lo + jj;
                if (i < g.n && j < g.n) pnxtT[(size_t)j * g.n + i] = to_storage<TS>(tile[ii * kAccStride + jj]);
            }
            __syncthreads(); // tile (sh.acc[0]) is zeroed by the next item
            return true;
        };
        if (sd.bitems) {
            // balanced plan: at most one item per block, from the table
            const int4 e = __ldg(sd.bitems + lb);
            if (e.x >= 0 && !process_item(e.x, e.y, e.z, e.w)) return false;
        } else {
            // uniform plan: every tile in H groups; items lb, lb + nblocks, ...
            const int H = sd.groups;
            const int n_items = sd.n_tiles * H, n_nonowner = sd.n_tiles * (H - 1);
            for (int item = lb; item < n_items; item += grp.nblocks) {
                const bool owner = item >= n_nonowner;
                const int t = owner ? item - n_nonowner : item % sd.n_tiles;
                const int h = owner ? H - 1 : item / sd.n_tiles;
                if (!process_item(t, h, H, t * (H - 1))) return false;
            }
        }
        if (!lam_done && !obtain_lambda()) return false; // blocks without an owner item keep the same state
        if (!group_sync(grp.count, err, bk, grp.nblocks, 0u, a.timeout_ns, a.spin_cap)) return false;
        ++bk;
        // every block has read the ring of this sub-iteration: store Phi_n (the next
        // barrier orders it before the next sub-iteration's reads)
        if (lb == ring_writer && threadIdx.x == 0) st->phi_ring[slot_n] = sh.phi_n;
        if (timer) {
            const unsigned long long now = global_ns();
            t_b += now - t_mark;
            t_mark = now;
        }
    }

    if (lb == 0) {
        if (threadIdx.x == 0) {
            st->n_done = n0 + a.n_iter;
            st->lambda = sh.lambda;
            st->phi_prev = sh.phi_prev;
            st->best_pass = sh.best_pass;
            st->best_n = sh.best_n;
            st->pass_prev = sh.pass_prev;
        }
    }
    __syncthreads(); // the next slice re-initialises the shared state
    return true;
}

// The index this block works under. The hardware, not the launch index, picks a
// block's SM (a cooperative launch of 4 blocks per SM put blocks 0-15 on the
// last 4 SMs, four each), so with a.place_per_sm > 0 (a full grid of
// place_per_sm blocks on each of place_sms SMs) a block takes slot * place_sms +
// (its SM), slot = its arrival order on that SM: index b then runs on SM
// b mod place_sms, as the balanced phase-B plan and the phase-F ray deal of the
// one-slice launch assume. The blocks agree through one grid-wide barrier
// (gbar->count, zero at launch) and all keep their launch index if any block
// found the grid spread otherwise. -1: that barrier gave up (leave the kernel).
__device__ __forceinline__ int placed_block(const LoopArgs &a, int *s_vb)
{
    if (a.place_per_sm <= 0) return (int)blockIdx.x;
    if (threadIdx.x == 0) {
        unsigned int sm;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
        int vb = -1;
        if (sm < (unsigned int)a.place_sms) {
            const int slot = atomicAdd(a.sm_slots + sm, 1);
            if (slot < a.place_per_sm) vb = slot * a.place_sms + (int)sm;
        }
        if (vb < 0) atomicExch(&a.gbar->place_err, 1);
        *s_vb = vb;
    }
    if (!group_sync(&a.gbar->count, &a.gbar->err, 0u, gridDim.x, 0u, a.timeout_ns, a.spin_cap)) return -1;
    return *(volatile int *)&a.gbar->place_err ? (int)blockIdx.x : *s_vb;
}

// The loop kernel: BATCH = false reads the one slice and group from the kernel
// parameters; BATCH = true reads each block's group and its slices from global
// descriptor arrays (copied to shared memory).
template <bool BATCH, typename TS = float>
__global__ void __launch_bounds__(kThreads, 4) k_recon(LoopArgs a)
{
    __shared__ LoopShared sh;
    // Set-up flagged bad input: every block sees the same flag and leaves.
    if (*(volatile int *)&a.gbar->data_err) return;
    unsigned int bk = 0; // group barriers passed
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_f = 0, t_b = 0, t_mark = timer ? global_ns() : 0;
    const int vb = placed_block(a, &sh.ok);
    if (vb < 0) return;
    if constexpr (BATCH) {
        if (threadIdx.x == 0) sh.grp = a.groups[a.block_group[vb]];
        __syncthreads();
        const int lb = vb - sh.grp.block0;
        for (int si = 0; si < sh.grp.nslices; ++si) {
            {
                const int *src = (const int *)(a.slices + sh.grp.slice0 + si);
                int *dst = (int *)&sh.sd;
                for (int k = threadIdx.x; k < (int)(sizeof(SliceDesc) / sizeof(int)); k += kThreads) dst[k] = src[k];
            }
            __syncthreads();
            if (!run_slice<TS>(sh.sd, sh.grp, a, lb, bk, sh, timer && si == 0, t_f, t_b, t_mark)) return;
        }
    } else {
        if (!run_slice<TS>(a.one, a.one_group, a, vb, bk, sh, timer, t_f, t_b, t_mark)) return;
    }
    if (timer) {
        a.phase_ns[0] = t_f;
        a.phase_ns[1] = t_b;
    }
}

// dst[k] = src[k] rounded to the 16-bit storage type, k < count.
template <typename TS>
__global__ void k_to_storage(const float *__restrict__ src, TS *__restrict__ dst, size_t count)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (size_t)gridDim.x * blockDim.x)
        dst[k] = to_storage<TS>(src[k]);
}

// The batch loop with its descriptors in the kernel parameters (batches of up
// to kParamSlices slices): each block's group and slices are read in place.
template <typename TS = float>
__global__ void __launch_bounds__(kThreads, 4) k_recon_pb(const __grid_constant__ LoopArgs a,
                                                          const __grid_constant__ BatchParams bp)
{
    __shared__ LoopShared sh;
    if (*(volatile int *)&a.gbar->data_err) return;
    unsigned int bk = 0;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_f = 0, t_b = 0, t_mark = timer ? global_ns() : 0;
    const int vb = placed_block(a, &sh.ok);
    if (vb < 0) return;
    const GroupDesc &grp = bp.gr[__ldg(a.block_group + vb)];
    const int lb = vb - grp.block0;
    for (int si = 0; si < grp.nslices; ++si)
        if (!run_slice<TS>(bp.sl[grp.slice0 + si], grp, a, lb, bk, sh, timer && si == 0, t_f, t_b, t_mark)) return;
    if (timer) {
        a.phase_ns[0] = t_f;
        a.phase_ns[1] = t_b;
    }
}
static_assert(sizeof(LoopArgs) + sizeof(BatchParams) <= 32000, "kernel parameters exceed the 32 KB limit");

// Fresh loop state for `count` slices.
__global__ void k_state_init(mvct_recon_state *st, int count, double lambda0)
{
    for (int b = blockIdx.x; b < count; b += gridDim.x) {
        for (int k = threadIdx.x; k < MVCT_MAX_SUBSETS; k += blockDim.x) st[b].phi_ring[k] = 0.0;
        if (threadIdx.x == 0) {
            st[b].n_done = 0;
            st[b].lambda = lambda0;
            st[b].phi_prev = 0.0;
            st[b].best_pass = INFINITY;
            st[b].best_n = -1;
            st[b].pass_prev = 0.0;
        }
    }
}

int recon_occupancy(mvct_plan_s *P)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_recon<false>, kThreads, 0) != cudaSuccess)
        return 0;
    return std::min(nb * P->num_sms, MVCT_MAX_RECON_GRID);
}

int slice_groups(const mvct_plan_s *P, int nblocks, int override_h)
{
    if (override_h > 0) return std::max(1, std::min(override_h, P->groups_cap));
    if (P->tuned_groups > 0) return std::max(1, std::min(P->tuned_groups, P->groups_cap));
    return std::max(1, std::min(P->groups, nblocks / P->n_tiles));
}

bool balanced_items(int n_tiles, int Vs, int groups_cap, int grid, int num_sms, std::vector<int4> &items,
                    int &idle_block)
{
    if (num_sms < 2 || grid % num_sms != 0) return false;
    const int r = grid / num_sms, cap = std::min(groups_cap, Vs);
    if (r < 2 || cap < 2) return false;
    const int full_items = (r - 1) * num_sms; // rounds 0 .. r-2: two groups of a tile each
    if (full_items % 2) return false;
    const int full_tiles = full_items / 2, rest = n_tiles - full_tiles;
    const int small = num_sms - 1; // round r-1 but its last block: the other tiles, split further
    if (rest < 1 || small < 2 * rest || small > cap * rest) return false;
    std::vector<int4> out(grid, make_int4(-1, 0, 0, 0));
    int slot = 0;
    for (int t = 0; t < full_tiles; ++t) {
        out[2 * t] = make_int4(t, 0, 2, slot);
        out[2 * t + 1] = make_int4(t, 1, 2, slot);
        slot += 1;
    }
    int b = full_items;
    for (int j = 0; j < rest; ++j) {
        const int t = full_tiles + j, ct = small / rest + (j < small % rest ? 1 : 0);
        for (int h = 0; h < ct; ++h) out[b++] = make_int4(t, h, ct, slot);
        slot += ct - 1;
    }
    // every tile once in each of its groups, slots within the partial-tile buffers
    std::vector<int> seen(n_tiles, 0);
    for (const int4 &e : out)
        if (e.x >= 0) seen[e.x] += 1 << e.y;
    for (int t = 0; t < n_tiles; ++t) {
        const int ht = t < full_tiles ? 2 : small / rest + (t - full_tiles < small % rest ? 1 : 0);
        if (seen[t] != (1 << ht) - 1) return false;
    }
    if (b != grid - 1 || slot > n_tiles * (groups_cap - 1)) return false;
    items.swap(out);
    idle_block = grid - 1;
    return true;
}

} // namespace mvct

using namespace mvct;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct Events {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    Events()
    {
        for (auto &x : e) cudaEventCreate(&x);
    }
    ~Events()
    {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
};

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t _e = (call);                                                         \
        if (_e != cudaSuccess)                                                           \
            return mvct_fail(MVCT_ECUDA, "%s: %s", #call, cudaGetErrorString(_e));       \
    } while (0)

} // namespace

extern "C" void mvct_recon_opts_init(mvct_recon_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->lambda0 = 0.01;
    o->dlambda_up = 1e-4;
    o->dlambda_down = 2e-4;
    o->lambda_min = 1e-4;
    o->kappa = 50.0;
    o->lambda_rule = MVCT_LAMBDA_PASS_SLIDING;
    o->tv_eps = 1e-6;
    o->mu0 = 0.05;
    o->barrier_timeout_ms = 2000.0;
}

namespace {

// mvct_recon with opts.psi_record: the loop one pass (S sub-iterations) per call,
// resumed through a loop state (bit-identical to one run), with the objective
// Psi of the iterate after every pass (and of the start image) on the host.
int recon_with_psi(mvct_plan P, const float *d_sino, const float *d_weights, double beta, int32_t n_iter,
                   const mvct_recon_opts &o, float *d_img, mvct_recon_stats *stats, void *stream)
{
    const int S = P->geo.S;
    mvct_recon_state local;
    std::memset(&local, 0, sizeof(local));
    local.lambda = o.lambda0;
    local.best_pass = INFINITY;
    local.best_n = -1;
    mvct_recon_opts oc = o;
    oc.psi_record = nullptr;
    oc.state = o.state ? o.state : &local;
    auto psi_now = [&](double *out) -> int {
        int rc = mvct_objective(P, d_img, d_sino, d_weights, beta, o.tv_eps, P->tv_sum, stream);
        if (rc) return rc;
        cudaError_t e = cudaMemcpyAsync(out, P->tv_sum, sizeof(double), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) return mvct_fail(MVCT_ECUDA, "mvct_recon: psi_record: %s", cudaGetErrorString(e));
        return MVCT_OK;
    };
    mvct_recon_stats sc;
    std::memset(&sc, 0, sizeof(sc));
    int rc = mvct_recon(P, d_sino, d_weights, beta, 0, &oc, d_img, &sc, stream); // set-up: d_img = mu^(0)
    if (rc) return rc;
    if ((rc = psi_now(o.psi_record))) return rc;
    oc.init_from_input = 1;
    double loop_ms = 0, setup_ms = sc.setup_ms, fwd_ms = 0, back_ms = 0;
    for (int done = 0; done < n_iter;) {
        const int chunk = std::min(S, n_iter - done);
        oc.lambda_schedule = o.lambda_schedule ? o.lambda_schedule + done : nullptr;
        std::memset(&sc, 0, sizeof(sc));
        if (stats) {
            sc.phi = stats->phi ? stats->phi + done : nullptr;
            sc.lambda = stats->lambda ? stats->lambda + done : nullptr;
        }
        if ((rc = mvct_recon(P, d_sino, d_weights, beta, chunk, &oc, d_img, &sc, stream))) return rc;
        loop_ms += sc.loop_ms;
        setup_ms += sc.setup_ms;
        fwd_ms += sc.forward_ms;
        back_ms += sc.back_ms;
        done += chunk;
        if (done % S == 0 && (rc = psi_now(o.psi_record + done / S))) return rc;
    }
    if (stats) {
        stats->best_n = oc.state->best_n;
        stats->best_pass = oc.state->best_pass;
        stats->loop_ms = loop_ms;
        stats->setup_ms = setup_ms;
        stats->forward_ms = fwd_ms;
        stats->back_ms = back_ms;
        stats->grid_blocks = P->grid;
        stats->block_threads = kThreads;
    }
    return MVCT_OK;
}

} // namespace

extern "C" int mvct_recon(mvct_plan P, const float *d_sino, const float *d_weights, double beta,
                          int32_t n_iter, const mvct_recon_opts *opts_in, float *d_img_inout,
                          mvct_recon_stats *stats, void *stream)
{
    if (!P) return mvct_fail(MVCT_EINVAL, "mvct_recon: null plan");
    {
        const int rc = mvct_check_ptrs(P->device, stream, "mvct_recon", {d_sino, d_weights, d_img_inout});
        if (rc) return rc;
        if (opts_in && opts_in->d_best_out) {
            const int rc2 = mvct_check_ptrs(P->device, stream, "mvct_recon", {opts_in->d_best_out});
            if (rc2) return rc2;
        }
    }
    if (n_iter < 0) return mvct_fail(MVCT_EINVAL, "mvct_recon: n_iter < 0");
    if (!std::isfinite(beta) || beta < 0) return mvct_fail(MVCT_EINVAL, "mvct_recon: beta must be finite and >= 0");
    mvct_recon_opts o;
    if (opts_in) o = *opts_in;
    else mvct_recon_opts_init(&o);
    if (!mvct_eps_ok(o.tv_eps) || !std::isfinite(o.kappa) || !std::isfinite(o.lambda0) ||
        !std::isfinite(o.mu0) || !(o.barrier_timeout_ms > 0) ||
        (o.data_term != MVCT_DATA_WLS && o.data_term != MVCT_DATA_POISSON) ||
        (o.lambda_rule != MVCT_LAMBDA_SUBSET && o.lambda_rule != MVCT_LAMBDA_PASS &&
         o.lambda_rule != MVCT_LAMBDA_PASS_SLIDING))
        return mvct_fail(MVCT_EINVAL, "mvct_recon: invalid options");
    if (o.state && (o.state->n_done < 0 || (o.state->n_done > 0 && !o.init_from_input)))
        return mvct_fail(MVCT_EINVAL, "mvct_recon: resuming (state->n_done > 0) needs init_from_input = 1");
    if (o.storage != MVCT_STORAGE_F32 && o.storage != MVCT_STORAGE_BF16 && o.storage != MVCT_STORAGE_F16)
        return mvct_fail(MVCT_EINVAL, "mvct_recon: storage %d unknown", o.storage);
    if (o.subset_order) {
        std::vector<char> seen(P->geo.S, 0);
        for (int k = 0; k < P->geo.S; ++k) {
            const int v = o.subset_order[k];
            if (v < 0 || v >= P->geo.S || seen[v])
                return mvct_fail(MVCT_EINVAL, "mvct_recon: subset_order is not a permutation of 0..%d", P->geo.S - 1);
            seen[v] = 1;
        }
    }
    if (P->recon_grid <= 0) return mvct_fail(MVCT_ELAUNCH, "mvct_recon: loop kernel has no occupancy");

    if (P->in_batch) return mvct_fail(MVCT_EINVAL, "mvct_recon: plan belongs to a batch");
    if (o.psi_record) return recon_with_psi(P, d_sino, d_weights, beta, n_iter, o, d_img_inout, stats, stream);
    DeviceGuard dg(P->device);
    cudaStream_t st = (cudaStream_t)stream;
    const Geo &g = P->geo;
    const size_t nn = (size_t)g.n * g.n;

    if (n_iter > P->hist_cap) {
        cudaFree(P->hist);
        cudaFree(P->sched);
        P->hist = nullptr;
        P->sched = nullptr;
        P->hist_cap = 0;
        if (cudaMalloc(&P->hist, 2 * sizeof(double) * (size_t)n_iter) != cudaSuccess ||
            cudaMalloc(&P->sched, sizeof(double) * (size_t)n_iter) != cudaSuccess)
            return mvct_fail(MVCT_ENOMEM, "mvct_recon: cannot allocate %d history entries", n_iter);
        P->hist_cap = n_iter;
    }

    mvct_recon_state hs;
    if (o.state) {
        hs = *o.state;
    } else {
        std::memset(&hs, 0, sizeof(hs));
        hs.lambda = o.lambda0;
        hs.best_pass = INFINITY;
        hs.best_n = -1;
    }
    const int n = g.n;
    float *mu_a = pad_row0(P->pad[0], n), *mu_b = pad_row0(P->pad[1], n);
    float *muT_a = pad_row0(P->pad[2], n), *muT_b = pad_row0(P->pad[3], n);

    const bool half = o.storage != MVCT_STORAGE_F32;
    if (half && !P->p16) {
        // 16-bit copies, 2 bytes per element; zeroed so the pad rows read as 0
        const size_t R = (size_t)g.V * g.C;
        bool ok = true;
        for (int k = 0; k < 4; ++k) ok = ok && cudaMalloc(&P->pad16[k], 2 * pad_floats(n)) == cudaSuccess;
        ok = ok && cudaMalloc(&P->p16, 2 * R) == cudaSuccess && cudaMalloc(&P->w16, 2 * R) == cudaSuccess;
        for (int k = 0; k < 4 && ok; ++k) ok = cudaMemset(P->pad16[k], 0, 2 * pad_floats(n)) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            for (auto &b : P->pad16) {
                cudaFree(b);
                b = nullptr;
            }
            cudaFree(P->p16);
            cudaFree(P->w16);
            P->p16 = P->w16 = nullptr;
            return mvct_fail(MVCT_ENOMEM, "mvct_recon: cannot allocate the 16-bit storage");
        }
    }
    auto h_row0 = [&](int k) { return (void *)((char *)P->pad16[k] + 2 * (size_t)kPadRows * n); };

    SliceDesc sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.g = g;
    sd.rays = P->rays;
    sd.ray_range = P->ray_range;
    sd.views = P->views;
    sd.p = d_sino;
    sd.w = d_weights;
    sd.D = P->D;
    sd.mu0 = mu_a;
    sd.mu1 = mu_b;
    sd.muT0 = muT_a;
    sd.muT1 = muT_b;
    if (half) {
        sd.hm0 = h_row0(0);
        sd.hm1 = h_row0(1);
        sd.hmT0 = h_row0(2);
        sd.hmT1 = h_row0(3);
        sd.hp = P->p16;
        sd.hw = P->w16;
    }
    sd.e4 = P->e4;
    sd.tile_part = P->tile_part;
    sd.tile_flag = P->tile_flag;
    sd.best = o.d_best_out;
    sd.phi_hist = P->hist;
    sd.lam_hist = P->hist + n_iter;
    sd.sched = o.lambda_schedule ? P->sched : nullptr;
    sd.sorder = o.subset_order ? P->sorder : nullptr;
    sd.st = (mvct_recon_state *)P->loop_state;
    sd.tiles_x = P->tiles_x;
    sd.n_tiles = P->n_tiles;
    sd.groups = slice_groups(P, P->grid);
    // the balanced plan for the default shape, else every tile in sd.groups groups
    const bool table = P->bitems && P->tuned_groups == 0 && P->grid == P->recon_grid;
    sd.bitems = table ? P->bitems : nullptr;
    sd.reducer = table ? P->bitems_reducer : (P->n_tiles * sd.groups < P->grid ? P->n_tiles * sd.groups : -1);
    sd.beta = (float)beta;
    GroupDesc gd{0, P->grid, 0, 1, P->d_count, P->partials};

    CK(cudaMemcpyAsync(P->loop_state, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
    if (o.lambda_schedule && n_iter > 0)
        CK(cudaMemcpyAsync(P->sched, o.lambda_schedule, sizeof(double) * n_iter, cudaMemcpyHostToDevice, st));
    if (o.subset_order)
        CK(cudaMemcpyAsync(P->sorder, o.subset_order, sizeof(int) * P->geo.S, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(P->bar, 0, sizeof(Barrier), st));
    CK(cudaMemsetAsync(P->d_count, 0, sizeof(unsigned int) * kGroupSyncWords, st));
    CK(cudaMemsetAsync(P->phase_ns, 0, 2 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(P->tile_flag, 0, sizeof(unsigned int) * (size_t)P->n_tiles * P->groups_cap, st));

    Events ev;
    CK(cudaEventRecord(ev.e[0], st));
    // set-up (a0): w .* A1 over all views (and input validation), then D and mu0
    CK(launch_weight_a1(P, d_weights, d_sino, P->sino_tmp, &P->bar->data_err, st));
    const double cb = beta * 8.0 / std::sqrt(o.tv_eps);
    CK(launch_setup_back(P, P->sino_tmp, (float)cb, (float)o.mu0, o.init_from_input ? 1 : 0,
                         d_img_inout, mu_a, muT_a, st));
    if (half) {
        // the 16-bit copies of p, w and of the start image and its transpose
        const size_t R = (size_t)g.V * g.C;
        const int cg = P->num_sms * 8;
        if (o.storage == MVCT_STORAGE_BF16) {
            k_to_storage<<<cg, kThreads, 0, st>>>(d_sino, (__nv_bfloat16 *)P->p16, R);
            k_to_storage<<<cg, kThreads, 0, st>>>(d_weights, (__nv_bfloat16 *)P->w16, R);
            k_to_storage<<<cg, kThreads, 0, st>>>(P->pad[0], (__nv_bfloat16 *)P->pad16[0], pad_floats(n));
            k_to_storage<<<cg, kThreads, 0, st>>>(P->pad[2], (__nv_bfloat16 *)P->pad16[2], pad_floats(n));
        } else {
            k_to_storage<<<cg, kThreads, 0, st>>>(d_sino, (__half *)P->p16, R);
            k_to_storage<<<cg, kThreads, 0, st>>>(d_weights, (__half *)P->w16, R);
            k_to_storage<<<cg, kThreads, 0, st>>>(P->pad[0], (__half *)P->pad16[0], pad_floats(n));
            k_to_storage<<<cg, kThreads, 0, st>>>(P->pad[2], (__half *)P->pad16[2], pad_floats(n));
        }
        CK(cudaGetLastError());
    }
    CK(cudaEventRecord(ev.e[1], st));

    if (n_iter > 0) {
        LoopArgs a;
        std::memset(&a, 0, sizeof(a));
        a.one = sd;
        a.one_group = gd;
        a.gbar = P->bar;
        a.phase_ns = P->phase_ns;
        a.n_iter = n_iter;
        a.lambda0 = o.lambda0;
        a.dup = o.dlambda_up;
        a.ddown = o.dlambda_down;
        a.lmin = o.lambda_min;
        a.kappa = o.kappa;
        a.eps = (float)o.tv_eps;
        a.timeout_ns = (unsigned long long)(o.barrier_timeout_ms * 1e6);
        a.spin_cap = std::max<unsigned long long>(a.timeout_ns / 50ull, 1000ull);
        a.debug_unreachable = o.debug_unreachable_barrier ? 1 : 0;
        a.poisson = o.data_term == MVCT_DATA_POISSON ? 1 : 0;
        a.lambda_rule = o.lambda_rule;
        // a full grid of r blocks on every SM is numbered by where its blocks run
        a.sm_slots = P->sm_slots;
        a.place_sms = P->num_sms;
        a.place_per_sm = (P->grid == P->recon_grid && P->grid % P->num_sms == 0) ? P->grid / P->num_sms : 0;
        if (a.place_per_sm > 0) CK(cudaMemsetAsync(P->sm_slots, 0, sizeof(int) * P->num_sms, st));
        void *args[] = {&a};
        const void *kern = o.storage == MVCT_STORAGE_BF16  ? (const void *)k_recon<false, __nv_bfloat16>
                           : o.storage == MVCT_STORAGE_F16 ? (const void *)k_recon<false, __half>
                                                           : (const void *)k_recon<false, float>;
        cudaError_t le = cudaLaunchCooperativeKernel(kern, dim3(P->grid), dim3(kThreads), args, 0, st);
        if (le == cudaErrorCooperativeLaunchTooLarge)
            return mvct_fail(MVCT_ELAUNCH, "mvct_recon: %d blocks cannot be co-resident", P->grid);
        if (le != cudaSuccess)
            return mvct_fail(MVCT_ECUDA, "mvct_recon: cooperative launch: %s", cudaGetErrorString(le));
    }
    CK(cudaMemcpyAsync(d_img_inout, (n_iter & 1) ? mu_b : mu_a, nn * sizeof(float), cudaMemcpyDeviceToDevice,
                       st));
    CK(cudaEventRecord(ev.e[2], st));

    Barrier hb;
    CK(cudaMemcpyAsync(&hb, P->bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
    unsigned long long hphase[2] = {0, 0};
    CK(cudaMemcpyAsync(hphase, P->phase_ns, sizeof(hphase), cudaMemcpyDeviceToHost, st));
    mvct_recon_state out_state;
    CK(cudaMemcpyAsync(&out_state, P->loop_state, sizeof(out_state), cudaMemcpyDeviceToHost, st));
    std::vector<double> hist(2 * (size_t)n_iter);
    if (n_iter > 0)
        CK(cudaMemcpyAsync(hist.data(), P->hist, 2 * sizeof(double) * n_iter, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));

    if (hb.data_err) return mvct_fail(MVCT_EDATA, "mvct_recon: non-finite projections/weights or negative weights");
    if (hb.err)
        return mvct_fail(MVCT_ETIMEOUT, "mvct_recon: grid barrier wait exceeded %.1f ms", o.barrier_timeout_ms);

    if (o.state) *o.state = out_state;
    if (stats) {
        if (stats->phi && n_iter > 0) std::memcpy(stats->phi, hist.data(), sizeof(double) * n_iter);
        if (stats->lambda && n_iter > 0) std::memcpy(stats->lambda, hist.data() + n_iter, sizeof(double) * n_iter);
        stats->best_n = out_state.best_n;
        stats->best_pass = out_state.best_pass;
        float t1 = 0.f, t2 = 0.f;
        cudaEventElapsedTime(&t1, ev.e[0], ev.e[1]);
        cudaEventElapsedTime(&t2, ev.e[1], ev.e[2]);
        stats->setup_ms = t1;
        stats->loop_ms = t2;
        stats->forward_ms = hphase[0] * 1e-6;
        stats->back_ms = hphase[1] * 1e-6;
        stats->grid_blocks = P->grid;
        stats->block_threads = kThreads;
    }
    return MVCT_OK;
}

// ---------------------------------------------------------------------------
// Batches: many slices of uneven geometry in one persistent launch.
// ---------------------------------------------------------------------------
struct mvct_batch_s {
    int device = 0, count = 0, grid = 0, ngroups = 0, max_iter = 0;
    int groups_override = 0;            // > 0: view groups per tile of every slice (autotuner)
    bool param_kernel = false;          // launch k_recon_pb (descriptors in the kernel parameters)
    std::vector<mvct_plan_s *> plans;   // user order
    std::vector<int> pos;               // user slice -> position in the descriptor array
    std::vector<int> group_blocks;      // blocks of the group of each user slice
    SliceDesc *d_slices = nullptr;
    GroupDesc *d_groups = nullptr;
    int *d_block_group = nullptr;
    unsigned int *d_counts = nullptr;   // [ngroups][kGroupSyncWords]
    double *d_partials = nullptr;       // [grid]
    Barrier *d_bar = nullptr;
    unsigned long long *d_phase = nullptr;
    mvct_recon_state *d_states = nullptr; // [count] in descriptor order
    double *d_hist = nullptr;           // [count][2][max_iter] in descriptor order
    std::vector<float *> imgs;          // user order
    std::vector<const float *> sinos, weights;
    std::vector<double> betas;
    mvct_recon_opts opts;
    std::vector<SliceDesc> h_slices;    // descriptor order (for the parameter-space launch)
    std::vector<GroupDesc> h_groups;
    bool bound = false;
    int last_n_iter = 0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
};

namespace {

void free_batch(mvct_batch_s *b)
{
    if (!b) return;
    void *ptrs[] = {b->d_slices, b->d_groups, b->d_block_group, b->d_counts, b->d_partials,
                    b->d_bar, b->d_phase, b->d_states, b->d_hist};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &e : b->ev)
        if (e) cudaEventDestroy(e);
    for (auto *p : b->plans)
        if (p) p->in_batch = false;
    delete b;
}

double slice_work(const mvct_plan_s *P)
{
    // both loop phases scale with the rays of a subset times the image side
    return (double)P->geo.Vs * P->geo.C * P->geo.n;
}

} // namespace

extern "C" int mvct_batch_create(const mvct_plan *plans, int32_t count, mvct_batch *out)
{
    if (!out) return mvct_fail(MVCT_EINVAL, "mvct_batch_create: out is NULL");
    *out = nullptr;
    if (!plans || count < 1) return mvct_fail(MVCT_EINVAL, "mvct_batch_create: need at least one plan");
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return mvct_fail(MVCT_EINVAL, "mvct_batch_create: plan %d is NULL", i);
        if (plans[i]->in_batch) return mvct_fail(MVCT_EINVAL, "mvct_batch_create: plan %d is in another batch", i);
        if (plans[i]->device != plans[0]->device)
            return mvct_fail(MVCT_EINVAL, "mvct_batch_create: plans on different devices");
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return mvct_fail(MVCT_EINVAL, "mvct_batch_create: plan %d appears twice", i);
    }
    DeviceGuard dg(plans[0]->device);
    mvct_batch_s *b = new mvct_batch_s();
    b->device = plans[0]->device;
    b->count = count;
    b->grid = plans[0]->recon_grid;
    b->plans.assign(plans, plans + count);
    const int G = b->grid;
    if (G <= 0) {
        free_batch(b);
        return mvct_fail(MVCT_ELAUNCH, "mvct_batch_create: loop kernel has no occupancy");
    }

    // Partition the grid into groups. Up to G slices: one group per slice, at
    // least one block each, further blocks dealt one at a time to the slice with
    // the largest work per block.
    // More slices: G one-block groups, slices dealt longest-first to the least
    // loaded group.
    std::vector<double> work(count);
    for (int i = 0; i < count; ++i) work[i] = slice_work(plans[i]);
    std::vector<std::vector<int>> members;
    std::vector<int> nblocks;
    if (count <= G) {
        // highest averages: each further block goes to the slice with the most work
        // per block, which minimises the largest work per block (the launch ends
        // with its slowest group)
        nblocks.assign(count, 1);
        std::priority_queue<std::pair<double, int>> pq;
        for (int i = 0; i < count; ++i) pq.push({work[i], -i});
        for (int left = G - count; left > 0; --left) {
            const int i = -pq.top().second;
            pq.pop();
            nblocks[i] += 1;
            pq.push({work[i] / nblocks[i], -i});
        }
        for (int i = 0; i < count; ++i) members.push_back({i});
    } else {
        std::vector<int> idx(count);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return work[x] > work[y]; });
        members.assign(G, {});
        std::vector<double> load(G, 0.0);
        for (int i : idx) {
            const int gmin = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            members[gmin].push_back(i);
            load[gmin] += work[i];
        }
        nblocks.assign(G, 1);
    }
    b->ngroups = (int)members.size();
    std::vector<GroupDesc> groups(b->ngroups);
    std::vector<int> block_group(G);
    b->pos.assign(count, 0);
    b->group_blocks.assign(count, 1);
    int block0 = 0, slice0 = 0;
    for (int gi = 0; gi < b->ngroups; ++gi) {
        groups[gi] = GroupDesc{block0, nblocks[gi], slice0, (int)members[gi].size(), nullptr, nullptr};
        for (int k = 0; k < nblocks[gi]; ++k) block_group[block0 + k] = gi;
        for (int i : members[gi]) {
            b->pos[i] = slice0++;
            b->group_blocks[i] = nblocks[gi];
        }
        block0 += nblocks[gi];
    }
    bool ok = cudaMalloc(&b->d_slices, sizeof(SliceDesc) * count) == cudaSuccess &&
              cudaMalloc(&b->d_groups, sizeof(GroupDesc) * b->ngroups) == cudaSuccess &&
              cudaMalloc(&b->d_block_group, sizeof(int) * G) == cudaSuccess &&
              cudaMalloc(&b->d_counts, sizeof(unsigned int) * kGroupSyncWords * (size_t)b->ngroups) == cudaSuccess &&
              cudaMalloc(&b->d_partials, sizeof(double) * G) == cudaSuccess &&
              cudaMalloc(&b->d_bar, sizeof(Barrier)) == cudaSuccess &&
              cudaMalloc(&b->d_phase, 2 * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&b->d_states, sizeof(mvct_recon_state) * count) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_batch(b);
        return mvct_fail(MVCT_ENOMEM, "mvct_batch_create: device allocation failed");
    }
    for (int gi = 0; gi < b->ngroups; ++gi) {
        groups[gi].count = b->d_counts + kGroupSyncWords * gi;
        groups[gi].partials = b->d_partials + groups[gi].block0;
    }
    b->h_groups = groups;
    cudaError_t e = cudaMemcpy(b->d_groups, groups.data(), sizeof(GroupDesc) * b->ngroups, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_block_group, block_group.data(), sizeof(int) * G, cudaMemcpyHostToDevice);
    for (auto &ev : b->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
        free_batch(b);
        return mvct_fail(MVCT_ECUDA, "mvct_batch_create: %s", cudaGetErrorString(e));
    }
    // The parameter-space kernel serves batches whose descriptors fit its
    // parameters, if the whole grid of it can be co-resident; the choice is made
    // here so that a launch (possibly captured into a graph) never has to retry.
    if (count <= kParamSlices && b->ngroups <= kParamSlices) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_recon_pb<float>, kThreads, 0) != cudaSuccess) {
            cudaGetLastError();
            nb = 0;
        }
        b->param_kernel = (long long)nb * plans[0]->num_sms >= G;
    }
    for (auto *p : b->plans) p->in_batch = true;
    *out = b;
    return MVCT_OK;
}

extern "C" void mvct_batch_destroy(mvct_batch b)
{
    if (!b) return;
    DeviceGuard dg(b->device);
    cudaDeviceSynchronize();
    free_batch(b);
}

extern "C" int mvct_batch_bind(mvct_batch b, const float *const *d_sinos, const float *const *d_weights,
                               const double *betas, float *const *d_imgs, int32_t max_iter,
                               const mvct_recon_opts *opts_in)
{
    if (!b) return mvct_fail(MVCT_EINVAL, "mvct_batch_bind: null batch");
    if (!d_sinos || !d_weights || !betas || !d_imgs || max_iter < 0)
        return mvct_fail(MVCT_EINVAL, "mvct_batch_bind: null array or negative max_iter");
    mvct_recon_opts o;
    if (opts_in) o = *opts_in;
    else mvct_recon_opts_init(&o);
    if (o.lambda_schedule || o.state || o.d_best_out || o.subset_order || o.psi_record)
        return mvct_fail(MVCT_EINVAL, "mvct_batch_bind: lambda_schedule, state, d_best_out, subset_order and "
                         "psi_record are one-slice options");
    if (!mvct_eps_ok(o.tv_eps) || !std::isfinite(o.kappa) || !std::isfinite(o.lambda0) ||
        !std::isfinite(o.mu0) || !(o.barrier_timeout_ms > 0) ||
        (o.data_term != MVCT_DATA_WLS && o.data_term != MVCT_DATA_POISSON) ||
        (o.lambda_rule != MVCT_LAMBDA_SUBSET && o.lambda_rule != MVCT_LAMBDA_PASS &&
         o.lambda_rule != MVCT_LAMBDA_PASS_SLIDING))
        return mvct_fail(MVCT_EINVAL, "mvct_batch_bind: invalid options");
    if (o.storage != MVCT_STORAGE_F32) return mvct_fail(MVCT_EINVAL, "mvct_batch_bind: only FP32 storage");
    for (int i = 0; i < b->count; ++i) {
        if (!d_sinos[i] || !d_weights[i] || !d_imgs[i])
            return mvct_fail(MVCT_EINVAL, "mvct_batch_bind: null device pointer for slice %d", i);
        const int rc = mvct_check_ptrs(b->device, nullptr, "mvct_batch_bind", {d_sinos[i], d_weights[i], d_imgs[i]});
        if (rc) return rc;
        if (!std::isfinite(betas[i]) || betas[i] < 0)
            return mvct_fail(MVCT_EINVAL, "mvct_batch_bind: beta of slice %d must be finite and >= 0", i);
    }
    DeviceGuard dg(b->device);
    if (max_iter > b->max_iter || !b->d_hist) {
        if (b->d_hist) cudaFree(b->d_hist);
        b->d_hist = nullptr;
        if (cudaMalloc(&b->d_hist, sizeof(double) * 2 * std::max(1, max_iter) * (size_t)b->count) != cudaSuccess)
            return mvct_fail(MVCT_ENOMEM, "mvct_batch_bind: cannot allocate history");
    }
    b->max_iter = std::max(max_iter, b->max_iter);
    std::vector<SliceDesc> h(b->count);
    for (int i = 0; i < b->count; ++i) {
        mvct_plan_s *P = b->plans[i];
        const int n = P->geo.n, q = b->pos[i];
        SliceDesc &sd = h[q];
        std::memset(&sd, 0, sizeof(sd));
        sd.g = P->geo;
        sd.rays = P->rays;
        sd.ray_range = P->ray_range;
        sd.views = P->views;
        sd.p = d_sinos[i];
        sd.w = d_weights[i];
        sd.D = P->D;
        sd.mu0 = pad_row0(P->pad[0], n);
        sd.mu1 = pad_row0(P->pad[1], n);
        sd.muT0 = pad_row0(P->pad[2], n);
        sd.muT1 = pad_row0(P->pad[3], n);
        sd.e4 = P->e4;
        sd.tile_part = P->tile_part;
        sd.tile_flag = P->tile_flag;
        sd.phi_hist = b->d_hist + (size_t)q * 2 * b->max_iter;
        sd.lam_hist = sd.phi_hist + b->max_iter;
        sd.st = b->d_states + q;
        sd.tiles_x = P->tiles_x;
        sd.n_tiles = P->n_tiles;
        sd.groups = slice_groups(P, b->group_blocks[i], b->groups_override);
        sd.bitems = nullptr;
        sd.reducer = P->n_tiles * sd.groups < b->group_blocks[i] ? P->n_tiles * sd.groups : -1;
        sd.beta = (float)betas[i];
    }
    cudaError_t e = cudaMemcpy(b->d_slices, h.data(), sizeof(SliceDesc) * b->count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return mvct_fail(MVCT_ECUDA, "mvct_batch_bind: %s", cudaGetErrorString(e));
    b->h_slices = h;
    b->imgs.assign(d_imgs, d_imgs + b->count);
    b->sinos.assign(d_sinos, d_sinos + b->count);
    b->weights.assign(d_weights, d_weights + b->count);
    b->betas.assign(betas, betas + b->count);
    b->opts = o;
    b->bound = true;
    return MVCT_OK;
}

extern "C" int mvct_batch_run(mvct_batch b, int32_t n_iter, void *stream)
{
    if (!b || !b->bound) return mvct_fail(MVCT_EINVAL, "mvct_batch_run: batch not bound");
    if (n_iter < 0 || n_iter > b->max_iter)
        return mvct_fail(MVCT_EINVAL, "mvct_batch_run: n_iter %d outside 0..%d", n_iter, b->max_iter);
    DeviceGuard dg(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    const mvct_recon_opts &o = b->opts;
    CK(cudaEventRecord(b->ev[0], st));
    CK(cudaMemsetAsync(b->d_bar, 0, sizeof(Barrier), st));
    CK(cudaMemsetAsync(b->d_counts, 0, sizeof(unsigned int) * kGroupSyncWords * (size_t)b->ngroups, st));
    CK(cudaMemsetAsync(b->d_phase, 0, 2 * sizeof(unsigned long long), st));
    k_state_init<<<std::min(b->count, 1024), 256, 0, st>>>(b->d_states, b->count, o.lambda0);
    CK(cudaGetLastError());
    // set-up of every slice (a0): w .* A1 with the input check, then D and mu0
    for (int i = 0; i < b->count; ++i) {
        mvct_plan_s *P = b->plans[i];
        const int n = P->geo.n;
        CK(cudaMemsetAsync(P->tile_flag, 0, sizeof(unsigned int) * (size_t)P->n_tiles * P->groups_cap, st));
        CK(launch_weight_a1(P, b->weights[i], b->sinos[i], P->sino_tmp, &b->d_bar->data_err, st));
        const double cb = b->betas[i] * 8.0 / std::sqrt(o.tv_eps);
        CK(launch_setup_back(P, P->sino_tmp, (float)cb, (float)o.mu0, o.init_from_input ? 1 : 0, b->imgs[i],
                             pad_row0(P->pad[0], n), pad_row0(P->pad[2], n), st));
    }
    CK(cudaEventRecord(b->ev[1], st));
    if (n_iter > 0) {
        LoopArgs a;
        std::memset(&a, 0, sizeof(a));
        a.slices = b->d_slices;
        a.groups = b->d_groups;
        a.block_group = b->d_block_group;
        a.gbar = b->d_bar;
        a.phase_ns = b->d_phase;
        a.n_iter = n_iter;
        a.lambda0 = o.lambda0;
        a.dup = o.dlambda_up;
        a.ddown = o.dlambda_down;
        a.lmin = o.lambda_min;
        a.kappa = o.kappa;
        a.eps = (float)o.tv_eps;
        a.timeout_ns = (unsigned long long)(o.barrier_timeout_ms * 1e6);
        a.spin_cap = std::max<unsigned long long>(a.timeout_ns / 50ull, 1000ull);
        a.debug_unreachable = o.debug_unreachable_barrier ? 1 : 0;
        a.poisson = o.data_term == MVCT_DATA_POISSON ? 1 : 0;
        a.lambda_rule = o.lambda_rule;
        // batches keep the launch index (numbering the blocks by their SM made the
        // 48-slice stack 5 % slower while it made the one-slice loop 3 % faster)
        a.place_per_sm = 0;
        cudaError_t le;
        if (b->param_kernel) {
            // descriptors in the kernel parameters (copied at launch, captured by graphs)
            std::unique_ptr<BatchParams> bp(new BatchParams());
            std::memcpy(bp->sl, b->h_slices.data(), sizeof(SliceDesc) * b->count);
            std::memcpy(bp->gr, b->h_groups.data(), sizeof(GroupDesc) * b->ngroups);
            void *args[] = {&a, bp.get()};
            le = cudaLaunchCooperativeKernel((const void *)k_recon_pb<float>, dim3(b->grid), dim3(kThreads), args, 0,
                                             st);
        } else {
            void *args[] = {&a};
            le = cudaLaunchCooperativeKernel((const void *)k_recon<true>, dim3(b->grid), dim3(kThreads), args, 0, st);
        }
        if (le == cudaErrorCooperativeLaunchTooLarge)
            return mvct_fail(MVCT_ELAUNCH, "mvct_batch_run: %d blocks cannot be co-resident", b->grid);
        if (le != cudaSuccess)
            return mvct_fail(MVCT_ECUDA, "mvct_batch_run: cooperative launch: %s", cudaGetErrorString(le));
    }
    for (int i = 0; i < b->count; ++i) {
        mvct_plan_s *P = b->plans[i];
        const int n = P->geo.n;
        CK(cudaMemcpyAsync(b->imgs[i], pad_row0(P->pad[(n_iter & 1) ? 1 : 0], n), (size_t)n * n * sizeof(float),
                           cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaEventRecord(b->ev[2], st));
    b->last_n_iter = n_iter;
    return MVCT_OK;
}

extern "C" int mvct_batch_stats(mvct_batch b, int32_t slice, mvct_recon_stats *stats)
{
    if (!b || !b->bound) return mvct_fail(MVCT_EINVAL, "mvct_batch_stats: batch not bound");
    if (slice < 0 || slice >= b->count) return mvct_fail(MVCT_EINVAL, "mvct_batch_stats: slice %d out of range", slice);
    DeviceGuard dg(b->device);
    // the run may have been replayed from a CUDA graph (its event records are then
    // graph nodes, not these events): wait for the whole device
    CK(cudaDeviceSynchronize());
    Barrier hb;
    CK(cudaMemcpy(&hb, b->d_bar, sizeof(hb), cudaMemcpyDeviceToHost));
    if (hb.data_err) return mvct_fail(MVCT_EDATA, "mvct_batch: non-finite projections/weights or negative weights");
    if (hb.err)
        return mvct_fail(MVCT_ETIMEOUT, "mvct_batch: group barrier wait exceeded %.1f ms", b->opts.barrier_timeout_ms);
    if (!stats) return MVCT_OK;
    const int q = b->pos[slice], n_iter = b->last_n_iter;
    mvct_recon_state hs;
    CK(cudaMemcpy(&hs, b->d_states + q, sizeof(hs), cudaMemcpyDeviceToHost));
    if (n_iter > 0) {
        const double *src = b->d_hist + (size_t)q * 2 * b->max_iter;
        if (stats->phi) CK(cudaMemcpy(stats->phi, src, sizeof(double) * n_iter, cudaMemcpyDeviceToHost));
        if (stats->lambda) CK(cudaMemcpy(stats->lambda, src + b->max_iter, sizeof(double) * n_iter, cudaMemcpyDeviceToHost));
    }
    stats->best_n = hs.best_n;
    stats->best_pass = hs.best_pass;
    float t1 = -1.f, t2 = -1.f; // -1: the last run was a graph replay (times not available)
    if (cudaEventElapsedTime(&t1, b->ev[0], b->ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&t2, b->ev[1], b->ev[2]) != cudaSuccess) {
        cudaGetLastError();
        t1 = t2 = -1.f;
    }
    stats->setup_ms = t1;
    stats->loop_ms = t2;
    stats->forward_ms = 0.0;
    stats->back_ms = 0.0;
    stats->grid_blocks = b->group_blocks[slice];
    stats->block_threads = kThreads;
    return MVCT_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: short loop runs over launch-shape candidates on the caller's data.
// Candidates change only how the work is split (blocks of the loop launch, view
// groups per tile), so every candidate computes the same sums up to the order
// of the per-group partial tiles.
// ---------------------------------------------------------------------------
namespace {

void report_add(mvct_tune_report *r, int groups, int grid, double ms)
{
    if (!r || r->n_candidates >= MVCT_TUNE_MAX) return;
    r->cand_groups[r->n_candidates] = groups;
    r->cand_grid[r->n_candidates] = grid;
    r->cand_ms_per_iter[r->n_candidates] = ms;
    r->n_candidates += 1;
}

} // namespace

extern "C" int mvct_plan_tune(mvct_plan P, const float *d_sino, const float *d_weights, double beta,
                              int32_t n_iter_probe, mvct_tune_report *report, void *stream)
{
    if (!P) return mvct_fail(MVCT_EINVAL, "mvct_plan_tune: null plan");
    {
        const int rc = mvct_check_ptrs(P->device, stream, "mvct_plan_tune", {d_sino, d_weights});
        if (rc) return rc;
    }
    if (n_iter_probe < 1) return mvct_fail(MVCT_EINVAL, "mvct_plan_tune: n_iter_probe must be >= 1");
    if (P->in_batch) return mvct_fail(MVCT_EINVAL, "mvct_plan_tune: plan belongs to a batch");
    DeviceGuard dg(P->device);
    if (report) std::memset(report, 0, sizeof(*report));
    float *scratch = nullptr;
    if (cudaMalloc(&scratch, sizeof(float) * (size_t)P->geo.n * P->geo.n) != cudaSuccess) {
        cudaGetLastError();
        return mvct_fail(MVCT_ENOMEM, "mvct_plan_tune: scratch image");
    }
    const int saved_grid = P->grid, saved_tuned = P->tuned_groups;
    const int default_groups = slice_groups(P, P->recon_grid, 0);
    auto probe = [&](int grid, int groups, double *ms) -> int {
        P->grid = grid;
        P->tuned_groups = groups;
        mvct_recon_opts o;
        mvct_recon_opts_init(&o);
        mvct_recon_stats st;
        std::memset(&st, 0, sizeof(st));
        double best = INFINITY;
        for (int rep = 0; rep < 2; ++rep) { // the first run warms caches and clocks
            int rc = mvct_recon(P, d_sino, d_weights, beta, n_iter_probe, &o, scratch, &st, stream);
            if (rc) return rc;
            if (rep > 0) best = std::min(best, st.loop_ms / n_iter_probe);
        }
        *ms = best;
        return MVCT_OK;
    };
    // the default rule first (groups 0: the balanced plan where there is one)
    const int default_report = P->bitems ? 0 : default_groups;
    double default_ms = 0.0;
    int rc = probe(P->recon_grid, default_report, &default_ms);
    int best_grid = P->recon_grid, best_groups = default_report;
    double best_ms = default_ms;
    report_add(report, default_report, P->recon_grid, default_ms);
    const int max_bps = P->recon_grid / std::max(1, P->num_sms);
    const int hs[] = {1, 2, 3, 4, 6, 8};
    for (int bps = max_bps; rc == MVCT_OK && bps >= std::max(1, max_bps - 2); --bps) {
        const int grid = std::min(P->recon_grid, bps * P->num_sms);
        for (int h : hs) {
            if (h > P->groups_cap || (grid == P->recon_grid && h == default_report)) continue;
            double ms = 0.0;
            rc = probe(grid, h, &ms);
            if (rc) break;
            report_add(report, h, grid, ms);
            if (ms < best_ms) {
                best_ms = ms;
                best_grid = grid;
                best_groups = h;
            }
        }
    }
    cudaFree(scratch);
    if (rc) {
        P->grid = saved_grid;
        P->tuned_groups = saved_tuned;
        return rc;
    }
    P->grid = best_grid;
    P->tuned_groups = best_groups;
    if (report) {
        report->groups = best_groups;
        report->grid_blocks = best_grid;
        report->ms_per_iter = best_ms;
        report->default_ms_per_iter = default_ms;
    }
    return MVCT_OK;
}

extern "C" int mvct_plan_set_shape(mvct_plan P, int32_t groups, int32_t grid_blocks)
{
    if (!P) return mvct_fail(MVCT_EINVAL, "mvct_plan_set_shape: null plan");
    if (groups < 0 || groups > P->groups_cap)
        return mvct_fail(MVCT_EINVAL, "mvct_plan_set_shape: groups %d outside 0..%d", groups, P->groups_cap);
    if (grid_blocks < 0 || grid_blocks > P->recon_grid)
        return mvct_fail(MVCT_EINVAL, "mvct_plan_set_shape: grid %d outside 0..%d", grid_blocks, P->recon_grid);
    P->tuned_groups = groups;
    P->grid = grid_blocks > 0 ? grid_blocks : P->recon_grid;
    return MVCT_OK;
}

extern "C" int mvct_batch_tune(mvct_batch b, int32_t n_iter_probe, mvct_tune_report *report, void *stream)
{
    if (!b || !b->bound) return mvct_fail(MVCT_EINVAL, "mvct_batch_tune: batch not bound");
    if (n_iter_probe < 1) return mvct_fail(MVCT_EINVAL, "mvct_batch_tune: n_iter_probe must be >= 1");
    DeviceGuard dg(b->device);
    if (report) std::memset(report, 0, sizeof(*report));
    const int n_it = std::min<int>(n_iter_probe, b->max_iter);
    if (n_it < 1) return mvct_fail(MVCT_EINVAL, "mvct_batch_tune: the batch was bound with max_iter 0");
    cudaStream_t st = (cudaStream_t)stream;
    // the runs overwrite the bound images: keep copies of the start images
    std::vector<float *> saved(b->count, nullptr);
    int rc = MVCT_OK;
    for (int i = 0; i < b->count && rc == MVCT_OK; ++i) {
        const size_t bytes = sizeof(float) * (size_t)b->plans[i]->geo.n * b->plans[i]->geo.n;
        if (cudaMalloc(&saved[i], bytes) != cudaSuccess ||
            cudaMemcpyAsync(saved[i], b->imgs[i], bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            rc = mvct_fail(MVCT_ENOMEM, "mvct_batch_tune: image copies");
        }
    }
    auto restore = [&]() {
        for (int i = 0; i < b->count; ++i)
            if (saved[i])
                cudaMemcpyAsync(b->imgs[i], saved[i], sizeof(float) * (size_t)b->plans[i]->geo.n * b->plans[i]->geo.n,
                                cudaMemcpyDeviceToDevice, st);
    };
    const int saved_override = b->groups_override;
    auto probe = [&](int h, double *ms) -> int {
        b->groups_override = h;
        // re-bind so the descriptors carry this candidate's view groups
        std::vector<const float *> s(b->sinos), w(b->weights);
        std::vector<float *> im(b->imgs);
        std::vector<double> be(b->betas);
        const mvct_recon_opts o = b->opts;
        int r = mvct_batch_bind(b, s.data(), w.data(), be.data(), im.data(), b->max_iter, &o);
        if (r) return r;
        double best = INFINITY;
        for (int rep = 0; rep < 2; ++rep) {
            restore();
            r = mvct_batch_run(b, n_it, stream);
            if (r) return r;
            mvct_recon_stats stt;
            std::memset(&stt, 0, sizeof(stt));
            r = mvct_batch_stats(b, 0, &stt);
            if (r) return r;
            if (rep > 0) best = std::min(best, stt.loop_ms / n_it);
        }
        *ms = best;
        return MVCT_OK;
    };
    double default_ms = 0.0, best_ms = 0.0;
    int best_h = 0;
    if (rc == MVCT_OK) rc = probe(0, &default_ms);
    best_ms = default_ms;
    report_add(report, 0, b->grid, default_ms);
    const int hs[] = {1, 2, 3, 4, 6, 8};
    for (int h : hs) {
        if (rc) break;
        double ms = 0.0;
        rc = probe(h, &ms);
        if (rc) break;
        report_add(report, h, b->grid, ms);
        if (ms < best_ms) {
            best_ms = ms;
            best_h = h;
        }
    }
    b->groups_override = rc ? saved_override : best_h;
    int rc2 = MVCT_OK;
    {
        std::vector<const float *> s(b->sinos), w(b->weights);
        std::vector<float *> im(b->imgs);
        std::vector<double> be(b->betas);
        const mvct_recon_opts o = b->opts;
        rc2 = mvct_batch_bind(b, s.data(), w.data(), be.data(), im.data(), b->max_iter, &o);
    }
    restore();
    cudaStreamSynchronize(st);
    for (float *p : saved)
        if (p) cudaFree(p);
    if (rc) return rc;
    if (rc2) return rc2;
    if (report) {
        report->groups = best_h;
        report->grid_blocks = b->grid;
        report->ms_per_iter = best_ms;
        report->default_ms_per_iter = default_ms;
    }
    return MVCT_OK;
}
