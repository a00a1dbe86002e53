// Stand-alone kernels behind mvct_forward / mvct_back / mvct_tv_grad /
// mvct_objective and the set-up step of mvct_recon.
#include <algorithm>

#include "mvct_plan.h"

namespace mvct {

// 32x32 tiled transpose through shared memory (padded against bank conflicts).
__global__ void __launch_bounds__(kThreads) k_transpose(const float *__restrict__ src,
                                                        float *__restrict__ dst, int n)
{
    __shared__ float tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5; // 32 x 8 threads
    for (int r = ty; r < 32; r += 8) {
        const int i = by + r, j = bx + tx;
        if (i < n && j < n) tile[r][tx] = __ldg(src + (size_t)i * n + j);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = bx + r, j = by + tx; // dst row = src column
        if (i < n && j < n) dst[(size_t)i * n + j] = tile[tx][r];
    }
}

// One warp per ray (grid-stride). out[k*C + c] = (A img)_(v_k, c) * mul[v_k*C + c]
// (mul optional). check_p/data_err: set-up validation of p and w.
__global__ void __launch_bounds__(kThreads)
k_forward(Geo g, const float4 *__restrict__ rays, const float *__restrict__ img,
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
        float q = joseph_warp<true>(img, imgT, g.n, g.pc, r, lane);
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

// Per-block FP64 sum of w * (A img - p)^2 over all views (one warp per ray).
__global__ void __launch_bounds__(kThreads)
k_residual(Geo g, const float4 *__restrict__ rays, const float *__restrict__ img,
           const float *__restrict__ imgT, const float *__restrict__ p, const float *__restrict__ w,
           double *__restrict__ partials)
{
    __shared__ double s[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int total = g.V * g.C;
    double acc = 0.0;
    for (int ray = blockIdx.x * kWarps + warp; ray < total; ray += gridDim.x * kWarps) {
        const float q = joseph_warp<true>(img, imgT, g.n, g.pc, __ldg(&rays[ray]), lane);
        const double r = (double)q - (double)__ldg(p + ray);
        acc += (double)__ldg(w + ray) * r * r;
    }
    if (lane == 0) s[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kWarps; ++k) t += s[k];
        partials[blockIdx.x] = t;
    }
}

// One thread per pixel (grid-stride): img[i][j] = sum over the subset's rays.
__global__ void __launch_bounds__(kThreads)
k_back(Geo g, const float4 *__restrict__ rays, const float4 *__restrict__ views,
       const float *__restrict__ sino, float *__restrict__ img, int subset, int rows)
{
    const int nn = g.n * g.n;
    for (int r = blockIdx.x * kThreads + threadIdx.x; r < nn; r += gridDim.x * kThreads) {
        const int i = r / g.n, j = r - i * g.n;
        img[r] = gather_pixel<false, true>(g, rays, views, sino, i, j, subset, rows);
    }
}

// Set-up of the loop: D = 1/(A^T(w .* A1) + cb) on the support (a1t > 0), else 0;
// mu0 = support ? (init_from_input ? mu : mu0) : 0, written with its transpose.
__global__ void __launch_bounds__(kThreads)
k_setup_back(Geo g, const float4 *__restrict__ rays, const float4 *__restrict__ views,
             const float *__restrict__ wa1, const float *__restrict__ a1t, float cb, float mu0,
             int init_from_input, float *__restrict__ D, float *mu, float *__restrict__ muT)
{
    const int nn = g.n * g.n;
    for (int r = blockIdx.x * kThreads + threadIdx.x; r < nn; r += gridDim.x * kThreads) {
        const int i = r / g.n, j = r - i * g.n;
        const float den = gather_pixel<false, true>(g, rays, views, wa1, i, j, -1, g.V) + cb;
        const bool on = __ldg(a1t + r) > 0.f && den > 0.f;
        D[r] = on ? 1.f / den : 0.f;
        const float m0 = on ? (init_from_input ? mu[r] : mu0) : 0.f;
        mu[r] = m0;
        muT[(size_t)j * g.n + i] = m0;
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

static int pixel_grid(const mvct_plan_s *P, long long pixels)
{
    const long long want = (pixels + kThreads - 1) / kThreads;
    return (int)std::max<long long>(1, std::min<long long>(want, (long long)P->num_sms * 16));
}

cudaError_t launch_transpose(const float *src, float *dst, int n, cudaStream_t st)
{
    dim3 grid((n + 31) / 32, (n + 31) / 32);
    k_transpose<<<grid, kThreads, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_forward(const mvct_plan_s *P, const float *img, const float *imgT, float *out,
                           int subset, const float *mul, const float *check_p, int *data_err,
                           cudaStream_t st)
{
    const int rows = rows_of(P, subset);
    k_forward<<<ray_grid(P, (long long)rows * P->geo.C), kThreads, 0, st>>>(
        P->geo, P->rays, img, imgT, out, subset, rows, mul, check_p, data_err);
    return cudaGetLastError();
}

cudaError_t launch_residual(const mvct_plan_s *P, const float *img, const float *imgT,
                            const float *p, const float *w, double *partials, cudaStream_t st)
{
    k_residual<<<P->reduce_grid, kThreads, 0, st>>>(P->geo, P->rays, img, imgT, p, w, partials);
    return cudaGetLastError();
}

cudaError_t launch_back(const mvct_plan_s *P, const float *sino, float *img, int subset,
                        cudaStream_t st)
{
    k_back<<<pixel_grid(P, (long long)P->geo.n * P->geo.n), kThreads, 0, st>>>(
        P->geo, P->rays, P->views, sino, img, subset, rows_of(P, subset));
    return cudaGetLastError();
}

cudaError_t launch_setup_back(const mvct_plan_s *P, const float *wa1, float cb, float mu0,
                              int init_from_input, float *mu, float *muT, cudaStream_t st)
{
    k_setup_back<<<pixel_grid(P, (long long)P->geo.n * P->geo.n), kThreads, 0, st>>>(
        P->geo, P->rays, P->views, wa1, P->a1t, cb, mu0, init_from_input, P->D, mu, muT);
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
