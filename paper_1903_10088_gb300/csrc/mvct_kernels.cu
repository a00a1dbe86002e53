// Stand-alone kernels behind mvct_forward / mvct_back / mvct_tv_grad /
// mvct_objective and the set-up step of mvct_recon.
#include <algorithm>

#include "mvct_plan.h"

namespace mvct {

// Copy an n x n image into a zero-row-padded buffer and its transpose into
// another (both pointers at row 0), 32x32 tiles through shared memory.
__global__ void __launch_bounds__(kThreads) k_pad_transpose(const float *__restrict__ src,
                                                            float *__restrict__ dst,
                                                            float *__restrict__ dstT, int n)
{
    __shared__ float tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5; // 32 x 8 threads
    for (int r = ty; r < 32; r += 8) {
        const int i = by + r, j = bx + tx;
        if (i < n && j < n) {
            const float v = __ldg(src + (size_t)i * n + j);
            tile[r][tx] = v;
            dst[(size_t)i * n + j] = v;
        }
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = bx + r, j = by + tx; // dstT row = src column
        if (i < n && j < n) dstT[(size_t)i * n + j] = tile[tx][r];
    }
}

// One warp per ray (grid-stride). out[k*C + c] = (A img)_(v_k, c) * mul[v_k*C + c]
// (mul optional). check_p/data_err: set-up validation of p and w.
__global__ void __launch_bounds__(kThreads)
k_forward(Geo g, const float4 *__restrict__ rays, const int *__restrict__ ranges, const float *__restrict__ img,
          const float *__restrict__ imgT, float *__restrict__ out, int subset, int rows,
          const float *__restrict__ mul, const float *__restrict__ check_p, int *data_err)
{
    const int lane = threadIdx.x & 31;
    const int total = rows * g.C;
    const int gw0 = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int gws = gridDim.x * kWarps;
    for (int ray = gw0; ray < total; ray += gws) {
        const int k = ray / g.C, c = ray - k * g.C;
        const int v = subset < 0 ? k : subset + k * g.S;
        const size_t rv = (size_t)v * g.C + c;
        const float4 r = __ldg(&rays[rv]);
        float q = joseph_warp<true>(img, imgT, g.n, g.pc, r, __ldg(ranges + rv), lane);
        if (lane == 0) {
            if (mul) {
                const float wv = __ldg(mul + rv);
                if (check_p) {
                    const float pv = __ldg(check_p + rv);
                    if (!isfinite(pv) || !isfinite(wv) || wv < 0.f) atomicExch(data_err, 1);
                }
                q *= wv;
            }
            out[ray] = q;
        }
    }
}

// Set-up product w .* (A 1) from the plan's cached A 1 (the same FP32 product
// k_forward forms with mul = w), with the input check of p and w.
__global__ void __launch_bounds__(kThreads)
k_weight_a1(const float *__restrict__ a1, const float *__restrict__ w, const float *__restrict__ p,
            float *__restrict__ out, size_t count, int *data_err)
{
    bool bad = false;
    for (size_t k = (size_t)blockIdx.x * kThreads + threadIdx.x; k < count; k += (size_t)gridDim.x * kThreads) {
        const float wv = __ldg(w + k), pv = __ldg(p + k);
        bad |= !isfinite(pv) || !isfinite(wv) || wv < 0.f;
        out[k] = __ldg(a1 + k) * wv;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(data_err, 1);
}

// Per-block FP64 sum of w * (A img - p)^2 over all views (one warp per ray).
__global__ void __launch_bounds__(kThreads)
k_residual(Geo g, const float4 *__restrict__ rays, const int *__restrict__ ranges, const float *__restrict__ img,
           const float *__restrict__ imgT, const float *__restrict__ p, const float *__restrict__ w,
           double *__restrict__ partials, float *__restrict__ e_out)
{
    __shared__ double s[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int total = g.V * g.C;
    double acc = 0.0;
    for (int ray = blockIdx.x * kWarps + warp; ray < total; ray += gridDim.x * kWarps) {
        const float q = joseph_warp<true>(img, imgT, g.n, g.pc, __ldg(&rays[ray]), __ldg(ranges + ray), lane);
        const float pv = __ldg(p + ray), wv = __ldg(w + ray);
        const double r = (double)q - (double)pv;
        acc += (double)wv * r * r;
        if (e_out && lane == 0) e_out[ray] = wv * (q - pv);
    }
    if (lane == 0) s[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kWarps; ++k) t += s[k];
        partials[blockIdx.x] = t;
    }
}

// Stand-alone matched backprojection as a tile splat: block = (tile t, view
// group h) with t = blockIdx.x % T, h = blockIdx.x / T; group h takes the rows
// h, h + H, h + 2H, ... With one group the tile
// is written straight into the image; otherwise each group writes its partial
// tile and k_merge_tiles adds the groups in order (deterministic).
__global__ void __launch_bounds__(kThreads)
k_back_splat(Geo g, const float4 *__restrict__ rays, const float4 *__restrict__ views,
             const float *__restrict__ sino, int subset, int rows, int H, int tiles_x,
             float *__restrict__ img, float *__restrict__ part)
{
    __shared__ float s_acc[kWarps][kAccFloats];
    __shared__ float4 s_stage[kWarps][32];
    __shared__ int4 s_win[kWinBatch];
    const int T = tiles_x * tiles_x;
    const int t = blockIdx.x % T, h = blockIdx.x / T;
    const int i_lo = (t / tiles_x) * kTile, j_lo = (t % tiles_x) * kTile;
    const int C = g.C;
    const int wpos = splat_views(g, views, subset, h, rows, H, nullptr, i_lo, j_lo, s_acc, s_stage, s_win,
                                 [rays, sino, C](int k, int v) {
                                     return StageSino{rays + (size_t)v * C, sino + (size_t)k * C};
                                 });
    float vals[4];
    tile_sums(s_acc, kWarps, wpos, vals);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int idx = threadIdx.x + u * kThreads;
        const float val = vals[u];
        if (H == 1) {
            const int i = i_lo + (idx >> 5), j = j_lo + (idx & 31);
            if (i < g.n && j < g.n) img[(size_t)i * g.n + j] = val;
        } else {
            part[((size_t)t * H + h) * (kTile * kTile) + idx] = val;
        }
    }
}

// img = sum over groups h (in order) of the partial tiles.
__global__ void __launch_bounds__(kThreads)
k_merge_tiles(const float *__restrict__ part, int H, int tiles_x, int n, float *__restrict__ img)
{
    const int t = blockIdx.x;
    const int i_lo = (t / tiles_x) * kTile, j_lo = (t % tiles_x) * kTile;
    for (int idx = threadIdx.x; idx < kTile * kTile; idx += kThreads) {
        float v = 0.f;
        for (int h = 0; h < H; ++h) v += part[((size_t)t * H + h) * (kTile * kTile) + idx];
        const int i = i_lo + (idx >> 5), j = j_lo + (idx & 31);
        if (i < n && j < n) img[(size_t)i * n + j] = v;
    }
}

// Set-up of the loop from the merged A^T(w .* A1) partial tiles:
// D = 1/(A^T(w .* A1) + cb) on the support (a1t > 0), else 0;
// mu0 = support ? (init_from_input ? init : mu0) : 0, written with its transpose.
__global__ void __launch_bounds__(kThreads)
k_setup_merge(const float *__restrict__ part, int H, int tiles_x, int n, const float *__restrict__ a1t,
              float cb, float mu0, int init_from_input, const float *__restrict__ init,
              float *__restrict__ D, float *__restrict__ mu, float *__restrict__ muT)
{
    __shared__ float tile[kTile][kTile + 1];
    const int t = blockIdx.x;
    const int i_lo = (t / tiles_x) * kTile, j_lo = (t % tiles_x) * kTile;
    for (int idx = threadIdx.x; idx < kTile * kTile; idx += kThreads) {
        float den = cb;
        float v = 0.f;
        for (int h = 0; h < H; ++h) v += part[((size_t)t * H + h) * (kTile * kTile) + idx];
        den += v;
        const int ii = idx >> 5, jj = idx & 31, i = i_lo + ii, j = j_lo + jj;
        float m0 = 0.f;
        if (i < n && j < n) {
            const size_t r = (size_t)i * n + j;
            const bool on = __ldg(a1t + r) > 0.f && den > 0.f;
            D[r] = on ? 1.f / den : 0.f;
            m0 = on ? (init_from_input ? __ldg(init + r) : mu0) : 0.f;
            mu[r] = m0;
        }
        tile[ii][jj] = m0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTile * kTile; idx += kThreads) {
        const int jj = idx >> 5, ii = idx & 31, i = i_lo + ii, j = j_lo + jj;
        if (i < n && j < n) muT[(size_t)j * n + i] = tile[ii][jj];
    }
}

// TV gradient per pixel and per-block FP64 partial sums of TV_eps.
__global__ void __launch_bounds__(kThreads)
k_tv(int n, const float *__restrict__ img, float eps, float *__restrict__ grad,
     double *__restrict__ partials)
{
    __shared__ double s[kWarps];
    const int nn = n * n;
    double acc = 0.0;
    for (int r = blockIdx.x * kThreads + threadIdx.x; r < nn; r += gridDim.x * kThreads) {
        const int i = r / n, j = r - i * n;
        float phi;
        const float gv = tv_grad_pixel<true>(img, n, i, j, eps, &phi);
        if (grad) grad[r] = gv;
        acc += (double)phi;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kWarps; ++k) t += s[k];
        partials[blockIdx.x] = t;
    }
}

// out = ca * sum(a) + cb * sum(b), each summed in a fixed order (one warp).
__global__ void k_final_sum(const double *__restrict__ a, int na, double ca,
                            const double *__restrict__ b, int nb, double cb, double *out)
{
    const int lane = threadIdx.x;
    double sa = 0.0, sb = 0.0;
    for (int k = lane; k < na; k += 32) sa += a[k];
    for (int k = lane; k < nb; k += 32) sb += b[k];
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if (lane == 0) *out = ca * sa + (nb > 0 ? cb * sb : 0.0);
}

__global__ void k_fill(float *dst, size_t count, float value)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (size_t)gridDim.x * blockDim.x)
        dst[k] = value;
}

static int rows_of(const mvct_plan_s *P, int subset)
{
    return subset < 0 ? P->geo.V : P->geo.Vs;
}

static int ray_grid(const mvct_plan_s *P, long long rays)
{
    const long long want = (rays + kWarps - 1) / kWarps;
    return (int)std::max<long long>(1, std::min<long long>(want, (long long)P->num_sms * 16));
}

cudaError_t launch_pad_transpose(const float *src, float *dst, float *dstT, int n, cudaStream_t st)
{
    dim3 grid((n + 31) / 32, (n + 31) / 32);
    k_pad_transpose<<<grid, kThreads, 0, st>>>(src, dst, dstT, n);
    return cudaGetLastError();
}

cudaError_t launch_forward(const mvct_plan_s *P, const float *img, const float *imgT, float *out,
                           int subset, const float *mul, const float *check_p, int *data_err,
                           cudaStream_t st)
{
    const int rows = rows_of(P, subset);
    k_forward<<<ray_grid(P, (long long)rows * P->geo.C), kThreads, 0, st>>>(
        P->geo, P->rays, P->ray_range, img, imgT, out, subset, rows, mul, check_p, data_err);
    return cudaGetLastError();
}

cudaError_t launch_weight_a1(const mvct_plan_s *P, const float *w, const float *p, float *out, int *data_err,
                             cudaStream_t st)
{
    const size_t R = (size_t)P->geo.V * P->geo.C;
    const int grid = (int)std::max<size_t>(1, std::min<size_t>((R + kThreads - 1) / kThreads, (size_t)P->num_sms * 8));
    k_weight_a1<<<grid, kThreads, 0, st>>>(P->a1, w, p, out, R, data_err);
    return cudaGetLastError();
}

cudaError_t launch_residual(const mvct_plan_s *P, const float *img, const float *imgT,
                            const float *p, const float *w, double *partials, float *e_out, cudaStream_t st)
{
    k_residual<<<P->reduce_grid, kThreads, 0, st>>>(P->geo, P->rays, P->ray_range, img, imgT, p, w, partials,
                                                    e_out);
    return cudaGetLastError();
}

// y[k] += a * x[k], k < count.
__global__ void k_axpy(float *__restrict__ y, const float *__restrict__ x, float a, size_t count)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (size_t)gridDim.x * blockDim.x)
        y[k] = fmaf(a, x[k], y[k]);
}

cudaError_t launch_axpy(const mvct_plan_s *P, float *y, const float *x, float a, size_t count, cudaStream_t st)
{
    k_axpy<<<P->reduce_grid, kThreads, 0, st>>>(y, x, a, count);
    return cudaGetLastError();
}

// View groups per tile for the stand-alone splat, at most 8 and at most one group
// per view: one subset's rows (<= 64) fill the GPU about once (512^2 / 40 views:
// 3 groups, 33.8 us against 37.7 us with 8), longer row sets fill it a few times
// over (all 800 views: 8 groups, 0.347 ms against 0.41 ms with 3).
static int back_groups(const mvct_plan_s *P, int rows)
{
    const int per_sm = rows <= kWinBatch ? 4 : 16;
    const int want = (per_sm * P->num_sms + P->n_tiles - 1) / P->n_tiles;
    return std::max(1, std::min(std::min(8, rows), want));
}

cudaError_t launch_back(const mvct_plan_s *P, const float *sino, float *img, int subset,
                        cudaStream_t st)
{
    const int rows = rows_of(P, subset);
    const int H = back_groups(P, rows);
    k_back_splat<<<P->n_tiles * H, kThreads, 0, st>>>(P->geo, P->rays, P->views, sino, subset, rows, H,
                                                      P->tiles_x, img, P->back_part);
    if (H > 1) k_merge_tiles<<<P->n_tiles, kThreads, 0, st>>>(P->back_part, H, P->tiles_x, P->geo.n, img);
    return cudaGetLastError();
}

cudaError_t launch_setup_back(const mvct_plan_s *P, const float *wa1, float cb, float mu0,
                              int init_from_input, const float *init, float *mu, float *muT,
                              cudaStream_t st)
{
    const int H = back_groups(P, P->geo.V);
    k_back_splat<<<P->n_tiles * H, kThreads, 0, st>>>(P->geo, P->rays, P->views, wa1, -1, P->geo.V, H,
                                                      P->tiles_x, nullptr, P->back_part);
    k_setup_merge<<<P->n_tiles, kThreads, 0, st>>>(P->back_part, H, P->tiles_x, P->geo.n, P->a1t, cb, mu0,
                                                   init_from_input, init, P->D, mu, muT);
    return cudaGetLastError();
}

cudaError_t launch_tv(const mvct_plan_s *P, const float *img, float eps, float *grad,
                      double *partials, cudaStream_t st)
{
    k_tv<<<P->reduce_grid, kThreads, 0, st>>>(P->geo.n, img, eps, grad, partials);
    return cudaGetLastError();
}

cudaError_t launch_tv_grid(int n, const float *img, float eps, float *grad, double *partials, int grid,
                           cudaStream_t st)
{
    k_tv<<<grid, kThreads, 0, st>>>(n, img, eps, grad, partials);
    return cudaGetLastError();
}

cudaError_t launch_final_sum(const double *a, int na, double ca, const double *b, int nb, double cb,
                             double *out, cudaStream_t st)
{
    k_final_sum<<<1, 32, 0, st>>>(a, na, ca, b, nb, cb, out);
    return cudaGetLastError();
}

cudaError_t launch_fill(float *dst, size_t count, float value, cudaStream_t st)
{
    k_fill<<<256, kThreads, 0, st>>>(dst, count, value);
    return cudaGetLastError();
}

} // namespace mvct
