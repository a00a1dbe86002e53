// The ordered-subset TV loop as one persistent cooperative kernel.
//
// Per sub-iteration n (subset s = n mod S; Eq. 3-5, Sec. 3.3.2, 3.4, 4.2):
//   phase F  one warp per ray of the subset: Joseph reprojection of mu^(n),
//            residual r = q - p, prescaled weighted residual e = scale*w*r,
//            FP64 partial sums of r^2 per block
//   barrier
//   lambda   every block reduces the partials in the same fixed order, so every
//            block derives the same Phi_n, lambda_n (Eq. 4-5) and best-iterate
//            decision without another barrier
//   phase B  one thread per pixel (warps own 8x4 pixel patches): gathered
//            matched backprojection of e, TV_eps gradient, surrogate-
//            preconditioned step, clamp at 0, write mu^(n+1) and its transpose
//   barrier
// The image ping-pongs between the caller's buffer and a plan buffer; the
// transpose copy lets y-driven rays read contiguous memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mvct_plan.h"

namespace mvct {

// Largest persistent grid (8 co-resident blocks on each of up to 160 SMs).
#define MVCT_MAX_RECON_GRID 1280

struct ReconArgs {
    Geo g;
    const float4 *rays;
    const float4 *views;
    const float *p;
    const float *w;
    const float *D;
    float *mu0, *mu1;   // image ping-pong: sub-iteration it reads mu[it & 1]
    float *muT0, *muT1; // and their transposes
    float4 *e4;         // [Vs*C] (u_c, m, prescaled residual, flag) of the subset's rays
    double *partials;
    float *tile_part;   // [T][H-1][1024] partial tiles of the non-owner view groups
    unsigned int *tile_flag; // [T][H-1] sub-iteration stamp of each published partial
    float *best;
    double *phi_hist;
    double *lam_hist;
    const double *sched;
    mvct_recon_state *st;
    Barrier *bar;
    unsigned long long *phase_ns; // [2] block 0's time in phase F (+ barrier 1) and phase B (+ barrier 2)
    long long n0;
    int n_iter;
    int tiles_x, n_tiles, groups; // phase B: 32x32 tiles x view groups
    double lambda0, dup, ddown, lmin, kappa;
    float beta, eps;
    unsigned long long timeout_ns, spin_cap;
    int debug_unreachable;
};

// Wait until flag == stamp (bounded like the grid barrier). Thread 0 only.
__device__ __forceinline__ bool wait_flag(const unsigned int *flag, unsigned int stamp, Barrier *bar,
                                          unsigned long long timeout_ns, unsigned long long spin_cap)
{
    if (ld_acquire(flag) == stamp) return true;
    const unsigned long long t0 = global_ns();
    unsigned long long spins = 0;
    while (ld_acquire(flag) != stamp) {
        if (*(volatile int *)&bar->err) return false;
        ++spins;
        if (spins > spin_cap || ((spins & 31u) == 0 && global_ns() - t0 > timeout_ns)) {
            atomicExch(&bar->err, 1);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

__global__ void __launch_bounds__(kThreads, 4) k_recon(ReconArgs a)
{
    __shared__ double s_ring[MVCT_MAX_SUBSETS];
    __shared__ double s_warp[kWarps];
    __shared__ double s_lambda, s_phi_prev, s_best_pass;
    __shared__ long long s_best_n;
    __shared__ float s_tau;
    __shared__ int s_best_flag, s_ok;
    __shared__ float s_acc[kWarps][kAccFloats];
    __shared__ float4 s_stage[kWarps][32];

    const Geo g = a.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned int G = gridDim.x;
    const int gw0 = blockIdx.x * kWarps + warp;
    const int GW = (int)G * kWarps;

    // Set-up flagged bad input: every block sees the same flag and leaves.
    if (*(volatile int *)&a.bar->data_err) return;

    for (int k = threadIdx.x; k < g.S; k += kThreads) s_ring[k] = a.st->phi_ring[k];
    if (threadIdx.x == 0) {
        s_lambda = a.st->lambda;
        s_phi_prev = a.st->phi_prev;
        s_best_pass = a.st->best_pass;
        s_best_n = a.st->best_n;
    }
    __syncthreads();

    const int Rs = g.Vs * g.C;
    const float S_f = (float)g.S;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_f = 0, t_b = 0, t_mark = timer ? global_ns() : 0;

    for (int it = 0; it < a.n_iter; ++it) {
        const long long n = a.n0 + it;
        const int s = (int)(n % g.S);
        const bool odd = (it & 1) != 0;
        const float *cur = odd ? a.mu1 : a.mu0;
        const float *curT = odd ? a.muT1 : a.muT0;
        float *nxt = odd ? a.mu0 : a.mu1;
        float *nxtT = odd ? a.muT0 : a.muT1;
        const unsigned int stamp = (unsigned int)it + 1u;

        // ---- phase F: reprojection, residual, square difference -------------
        double acc_phi = 0.0;
        {
            // the next ray's table entry and data are fetched while this ray is walked
            float4 r_nx = make_float4(0.f, 0.f, 0.f, 1.f);
            float p_nx = 0.f, w_nx = 0.f;
            size_t rv_nx = 0;
            if (gw0 < Rs) {
                const int k = gw0 / g.C;
                rv_nx = (size_t)(s + k * g.S) * g.C + (gw0 - k * g.C);
                r_nx = __ldg(&a.rays[rv_nx]);
                if (lane == 0) {
                    p_nx = __ldg(a.p + rv_nx);
                    w_nx = __ldg(a.w + rv_nx);
                }
            }
            for (int ray = gw0; ray < Rs; ray += GW) {
                const float4 r = r_nx;
                const float pv = p_nx, wv = w_nx;
                const int nray = ray + GW;
                if (nray < Rs) {
                    const int k = nray / g.C;
                    rv_nx = (size_t)(s + k * g.S) * g.C + (nray - k * g.C);
                    r_nx = __ldg(&a.rays[rv_nx]);
                    if (lane == 0) {
                        p_nx = __ldg(a.p + rv_nx);
                        w_nx = __ldg(a.w + rv_nx);
                    }
                }
                const float q_ray = joseph_warp<false>(cur, curT, g.n, g.pc, r, lane);
                if (lane == 0) {
                    const float res = q_ray - pv;
                    a.e4[ray] = make_float4(r.x, r.y, r.z * wv * res, r.w);
                    acc_phi += (double)res * (double)res;
                }
            }
        }
        if (lane == 0) s_warp[warp] = acc_phi;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kWarps; ++k) t += s_warp[k];
            a.partials[blockIdx.x] = t;
        }
        if (!grid_sync(a.bar, 2u * it, (it == 0 && a.debug_unreachable) ? 1u : 0u, a.timeout_ns,
                       a.spin_cap))
            return;
        if (timer) {
            const unsigned long long now = global_ns();
            t_f += now - t_mark;
            t_mark = now;
        }

        // ---- adaptive lambda (Eq. 4-5) and best iterate (Sec. 4.2) ----------
        // Every block sums the G partials in the same fixed order: each thread
        // its strided share, then the warp trees, then the warps in order.
        {
            // all loads first (one round trip), then the fixed-order sums
            constexpr int L = (MVCT_MAX_RECON_GRID + kThreads - 1) / kThreads;
            double v[L];
#pragma unroll
            for (int u = 0; u < L; ++u) {
                const unsigned int b = threadIdx.x + u * kThreads;
                v[u] = b < G ? a.partials[b] : 0.0;
            }
            double t = 0.0;
#pragma unroll
            for (int u = 0; u < L; ++u) t += v[u];
            t = warp_sum(t);
            if (lane == 0) s_warp[warp] = t;
        }
        __syncthreads();
        if (warp == 0) {
            double phi = 0.0;
            for (int k = 0; k < kWarps; ++k) phi += s_warp[k];
            const int slot_n = (int)(n % g.S);
            if (lane == 0) s_ring[slot_n] = phi;
            __syncwarp();
            // pass sum Phi_{n-S+1} + ... + Phi_n: lane-strided, then the warp tree
            double pass = 0.0;
            const bool full = n >= g.S - 1;
            if (full)
                for (int k = lane; k < g.S; k += 32) pass += s_ring[k];
            pass = warp_sum(pass);
            if (lane == 0) {
                double lam;
                if (a.sched) {
                    lam = a.sched[it];
                } else if (n == 0) {
                    lam = a.lambda0;
                } else {
                    lam = s_lambda;
                    if (phi < s_phi_prev) lam += a.dup;
                    else if (phi > s_phi_prev) lam -= a.ddown;
                    if (lam < a.lmin) lam = a.lmin;
                }
                s_lambda = lam;
                s_phi_prev = phi;
                int bf = 0;
                if (full && pass < s_best_pass) {
                    s_best_pass = pass;
                    s_best_n = n;
                    bf = 1;
                }
                s_best_flag = bf;
                s_tau = (float)(a.kappa * lam);
                if (blockIdx.x == 0) {
                    a.phi_hist[it] = phi;
                    a.lam_hist[it] = lam;
                }
            }
        }
        __syncthreads();

        // ---- phase B: tile splat (estimation) + TV + preconditioned step ----
        // Items: (tile t, view group h), group h holding the subset rows
        // h, h + H, h + 2H, ... Groups h < H-1 publish a partial tile; group
        // H-1 (the owner) adds the partials in group order and updates the tile.
        // Non-owner items come first in every block's sequence, so an owner only
        // ever waits on items that never wait.
        const float tau = s_tau;
        const bool keep_best = s_best_flag && a.best;
        const int H = a.groups;
        const int n_items = a.n_tiles * H, n_nonowner = a.n_tiles * (H - 1);
        const float4 *e4 = a.e4;
        const int C = g.C;
        for (int item = blockIdx.x; item < n_items; item += G) {
            const bool owner = item >= n_nonowner;
            const int t = owner ? item - n_nonowner : item % a.n_tiles;
            const int h = owner ? H - 1 : item / a.n_tiles;
            const int i_lo = (t / a.tiles_x) * kTile, j_lo = (t % a.tiles_x) * kTile;
            const int wpos = splat_views(g, a.views, s, h, g.Vs, H, i_lo, j_lo, s_acc, s_stage,
                                         [e4, C](int k, int) { return StageE4{e4 + (size_t)k * C}; });
            float part_val[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) part_val[u] = tile_sum(s_acc, threadIdx.x + u * kThreads, kWarps, wpos);

            if (!owner) {
                const size_t slot = (size_t)t * (H - 1) + h;
                float *dst = a.tile_part + slot * (kTile * kTile);
#pragma unroll
                for (int u = 0; u < 4; ++u) __stcg(dst + threadIdx.x + u * kThreads, part_val[u]);
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    st_release(a.tile_flag + slot, stamp);
                }
                __syncthreads(); // s_acc is zeroed by the next item
                continue;
            }

            if (threadIdx.x == 0) {
                bool ok = true;
                for (int hh = 0; hh < H - 1 && ok; ++hh)
                    ok = wait_flag(a.tile_flag + (size_t)t * (H - 1) + hh, stamp, a.bar, a.timeout_ns,
                                   a.spin_cap);
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) return;

            // partial tiles of groups 0..H-2: all loads first, then the sums in group order
            float prev[kMaxGroups - 1][4];
#pragma unroll
            for (int hh = 0; hh < kMaxGroups - 1; ++hh)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    prev[hh][u] = hh < H - 1 ? __ldcg(a.tile_part + ((size_t)t * (H - 1) + hh) * (kTile * kTile) +
                                                      threadIdx.x + u * kThreads)
                                             : 0.f;
            float *tile = s_acc[0]; // reused for the transposed write-out
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = threadIdx.x + u * kThreads;
                const int ii = idx >> 5, jj = idx & 31;
                float gs = 0.f;
#pragma unroll
                for (int hh = 0; hh < kMaxGroups - 1; ++hh)
                    if (hh < H - 1) gs += prev[hh][u];
                gs += part_val[u];
                const int i = i_lo + ii, j = j_lo + jj;
                float nm = 0.f;
                if (i < g.n && j < g.n) {
                    const size_t r = (size_t)i * g.n + j;
                    const float m = cur[r];
                    const float d = __ldg(a.D + r);
                    if (keep_best) a.best[r] = m;
                    if (d > 0.f) {
                        const float tg = tv_grad_pixel<false>(cur, g.n, i, j, a.eps, nullptr);
                        nm = fmaxf(0.f, m - tau * d * fmaf(S_f, gs, a.beta * tg));
                    }
                    nxt[r] = nm;
                }
                part_val[u] = nm;
            }
            __syncthreads(); // every warp has finished reading s_acc
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
                if (i < g.n && j < g.n) nxtT[(size_t)j * g.n + i] = tile[ii * kAccStride + jj];
            }
            __syncthreads(); // tile (s_acc[0]) is zeroed by the next item
        }
        if (!grid_sync(a.bar, 2u * it + 1u, 0u, a.timeout_ns, a.spin_cap)) return;
        if (timer) {
            const unsigned long long now = global_ns();
            t_b += now - t_mark;
            t_mark = now;
        }
    }

    if (timer) {
        a.phase_ns[0] = t_f;
        a.phase_ns[1] = t_b;
    }
    if (blockIdx.x == 0) {
        for (int k = threadIdx.x; k < g.S; k += kThreads) a.st->phi_ring[k] = s_ring[k];
        if (threadIdx.x == 0) {
            a.st->n_done = a.n0 + a.n_iter;
            a.st->lambda = s_lambda;
            a.st->phi_prev = s_phi_prev;
            a.st->best_pass = s_best_pass;
            a.st->best_n = s_best_n;
        }
    }
}

int recon_occupancy(mvct_plan_s *P)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_recon, kThreads, 0) != cudaSuccess)
        return 0;
    return std::min(nb * P->num_sms, MVCT_MAX_RECON_GRID);
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
    o->kappa = 100.0;
    o->tv_eps = 1e-6;
    o->mu0 = 0.05;
    o->barrier_timeout_ms = 2000.0;
}

extern "C" int mvct_recon(mvct_plan P, const float *d_sino, const float *d_weights, double beta,
                          int32_t n_iter, const mvct_recon_opts *opts_in, float *d_img_inout,
                          mvct_recon_stats *stats, void *stream)
{
    if (!P) return mvct_fail(MVCT_EINVAL, "mvct_recon: null plan");
    if (!d_sino || !d_weights || !d_img_inout)
        return mvct_fail(MVCT_EINVAL, "mvct_recon: null device pointer");
    if (n_iter < 0) return mvct_fail(MVCT_EINVAL, "mvct_recon: n_iter < 0");
    if (!std::isfinite(beta) || beta < 0) return mvct_fail(MVCT_EINVAL, "mvct_recon: beta must be finite and >= 0");
    mvct_recon_opts o;
    if (opts_in) o = *opts_in;
    else mvct_recon_opts_init(&o);
    if (!(o.tv_eps > 0) || !std::isfinite(o.tv_eps) || !std::isfinite(o.kappa) || !std::isfinite(o.lambda0) ||
        !std::isfinite(o.mu0) || !(o.barrier_timeout_ms > 0))
        return mvct_fail(MVCT_EINVAL, "mvct_recon: invalid options");
    if (o.state && (o.state->n_done < 0 || (o.state->n_done > 0 && !o.init_from_input)))
        return mvct_fail(MVCT_EINVAL, "mvct_recon: resuming (state->n_done > 0) needs init_from_input = 1");
    if (P->recon_grid <= 0) return mvct_fail(MVCT_ELAUNCH, "mvct_recon: loop kernel has no occupancy");

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
    CK(cudaMemcpyAsync(P->loop_state, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
    if (o.lambda_schedule && n_iter > 0)
        CK(cudaMemcpyAsync(P->sched, o.lambda_schedule, sizeof(double) * n_iter, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(P->bar, 0, sizeof(Barrier), st));
    CK(cudaMemsetAsync(P->phase_ns, 0, 2 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(P->tile_flag, 0, sizeof(unsigned int) * (size_t)P->n_tiles * P->groups, st));

    Events ev;
    CK(cudaEventRecord(ev.e[0], st));
    // set-up (a0): w .* A1 over all views (and input validation), then D and mu0
    const int n = g.n;
    float *mu_a = pad_row0(P->pad[0], n), *mu_b = pad_row0(P->pad[1], n);
    float *muT_a = pad_row0(P->pad[2], n), *muT_b = pad_row0(P->pad[3], n);
    const float *ones = pad_row0(P->pad_ones, n);
    CK(launch_forward(P, ones, ones, P->sino_tmp, -1, d_weights, d_sino, &P->bar->data_err, st));
    const double cb = beta * 8.0 / std::sqrt(o.tv_eps);
    CK(launch_setup_back(P, P->sino_tmp, (float)cb, (float)o.mu0, o.init_from_input ? 1 : 0,
                         d_img_inout, mu_a, muT_a, st));
    CK(cudaEventRecord(ev.e[1], st));

    if (n_iter > 0) {
        ReconArgs a;
        std::memset(&a, 0, sizeof(a));
        a.g = g;
        a.rays = P->rays;
        a.views = P->views;
        a.p = d_sino;
        a.w = d_weights;
        a.D = P->D;
        a.mu0 = mu_a;
        a.mu1 = mu_b;
        a.muT0 = muT_a;
        a.muT1 = muT_b;
        a.e4 = P->e4;
        a.partials = P->partials;
        a.tile_part = P->tile_part;
        a.tile_flag = P->tile_flag;
        a.tiles_x = P->tiles_x;
        a.n_tiles = P->n_tiles;
        a.groups = P->groups;
        a.best = o.d_best_out;
        a.phi_hist = P->hist;
        a.lam_hist = P->hist + n_iter;
        a.sched = o.lambda_schedule ? P->sched : nullptr;
        a.st = (mvct_recon_state *)P->loop_state;
        a.bar = P->bar;
        a.phase_ns = P->phase_ns;
        a.n0 = hs.n_done;
        a.n_iter = n_iter;
        a.lambda0 = o.lambda0;
        a.dup = o.dlambda_up;
        a.ddown = o.dlambda_down;
        a.lmin = o.lambda_min;
        a.kappa = o.kappa;
        a.beta = (float)beta;
        a.eps = (float)o.tv_eps;
        a.timeout_ns = (unsigned long long)(o.barrier_timeout_ms * 1e6);
        a.spin_cap = std::max<unsigned long long>(a.timeout_ns / 50ull, 1000ull);
        a.debug_unreachable = o.debug_unreachable_barrier ? 1 : 0;
        void *args[] = {&a};
        cudaError_t le = cudaLaunchCooperativeKernel((const void *)k_recon, dim3(P->recon_grid),
                                                     dim3(kThreads), args, 0, st);
        if (le == cudaErrorCooperativeLaunchTooLarge)
            return mvct_fail(MVCT_ELAUNCH, "mvct_recon: %d blocks cannot be co-resident", P->recon_grid);
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
        stats->grid_blocks = P->recon_grid;
        stats->block_threads = kThreads;
    }
    return MVCT_OK;
}
