// Fan-beam filtered backprojection (equiangular detector): the comparison image
// of Sec. 1 / 4.5 and the loop's plain start. Textbook steps:
//   1. cosine pre-weighting   R'(beta, gamma) = R * D cos(gamma)
//   2. filtering along gamma  Q = a * (R' conv g), g the fan-beam ramp
//      g(0) = 1/(8 a^2), g(n a) = -1/(2 pi^2 sin^2(n a)) for odd n, 0 for even n
//   3. weighted backprojection  f = dbeta * sum_v Q(beta_v, gamma') / L^2
// Both kernels are deterministic (fixed summation order, no atomics).
#include <cmath>
#include <vector>

#include "mvct_plan.h"

namespace mvct {

// One block per view: q[v][c] = a * sum_k R'[k] g[c - k], R' = R * D cos(gamma_k).
// Only k = c and odd c - k contribute (even offsets of the ramp are zero). q rows
// are padded: channel c is stored at c + 2 of a row of C + 4 floats whose two
// entries at each end are 0, so the backprojection reads channels -2 .. C + 1
// without bounds tests.
__global__ void __launch_bounds__(kThreads) k_fbp_filter(Geo g, const float *__restrict__ sino,
                                                        const float *__restrict__ gtab,
                                                        const float *__restrict__ cosw, float a,
                                                        float *__restrict__ q)
{
    extern __shared__ float s_pre[]; // [C]
    const int v = blockIdx.x, C = g.C;
    float *qv = q + (size_t)v * (C + 4);
    for (int c = threadIdx.x; c < C; c += kThreads) s_pre[c] = __ldg(sino + (size_t)v * C + c) * __ldg(cosw + c);
    if (threadIdx.x < 4) qv[threadIdx.x < 2 ? threadIdx.x : C + threadIdx.x] = 0.f;
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += kThreads) {
        float acc = s_pre[c] * __ldg(gtab + (C - 1));
        // odd offsets d = c - k: k = c - 1, c - 3, ... and k = c + 1, c + 3, ...
        for (int k = c - 1; k >= 0; k -= 2) acc = fmaf(s_pre[k], __ldg(gtab + (C - 1) + (c - k)), acc);
        for (int k = c + 1; k < C; k += 2) acc = fmaf(s_pre[k], __ldg(gtab + (C - 1) + (c - k)), acc);
        qv[c + 2] = a * acc;
    }
}

// arctan(t) for |t| <= 0.42 from its Taylor (Gregory) series
// t - t^3/3 + t^5/5 - ... through the t^17 term, in Horner form in z = t^2;
// the first omitted term is below 0.42^19 / 19 < 4e-9 rad.
__device__ __forceinline__ float atan_series(float t)
{
    const float z = t * t;
    float s = 1.f / 17.f;
    s = fmaf(s, z, -1.f / 15.f);
    s = fmaf(s, z, 1.f / 13.f);
    s = fmaf(s, z, -1.f / 11.f);
    s = fmaf(s, z, 1.f / 9.f);
    s = fmaf(s, z, -1.f / 7.f);
    s = fmaf(s, z, 1.f / 5.f);
    s = fmaf(s, z, -1.f / 3.f);
    s = fmaf(s, z, 1.f);
    return t * s;
}

// Ray angle gamma' of a pixel seen from the source: atan(crs / dot) from the
// series when |crs / dot| <= 0.42 (every pixel of a clinical fan, half-angle
// about 0.24 rad), else atan2f.
__device__ __forceinline__ float ray_angle(float dot, float crs)
{
    const float t = __fdividef(crs, dot);
    return (dot > 0.f && fabsf(t) <= 0.42f) ? atan_series(t) : atan2f(crs, dot);
}

// Q(beta_v, gamma') / L^2 of one pixel from the padded filtered row qv (channel c
// at c + 2): linear interpolation in gamma, channels outside the detector read 0.
__device__ __forceinline__ float fbp_sample(const Geo &g, const float *__restrict__ qv, float dot, float crs)
{
    const float u = fmaf(ray_angle(dot, crs), g.inv_dgamma, g.c_mid);
    const float fl = floorf(u);
    const int k = min(max((int)fl, -2), g.C) + 2;
    const float f = u - fl;
    const float a0 = __ldg(qv + k), a1 = __ldg(qv + k + 1);
    return fmaf(f, a1 - a0, a0) * __fdividef(1.f, fmaf(dot, dot, crs * crs));
}

// Two horizontally adjacent pixels per thread: f = dbeta * sum_v Q(beta_v,
// gamma'(x, y)) / L^2, views in order. The second pixel's source-relative
// coordinates are the first's plus delta along x.
__global__ void __launch_bounds__(kThreads) k_fbp_back(Geo g, const float4 *__restrict__ views,
                                                      const float *__restrict__ q, float dbeta,
                                                      float *__restrict__ img)
{
    const int half = (g.n + 1) >> 1, total = g.n * half;
    const int Cp = g.C + 4;
    for (int r = blockIdx.x * kThreads + threadIdx.x; r < total; r += gridDim.x * kThreads) {
        const int i = r / half, j = 2 * (r - i * half);
        const float x = ((float)j - g.pc) * g.delta, y = ((float)i - g.pc) * g.delta;
        float acc0 = 0.f, acc1 = 0.f;
        for (int v = 0; v < g.V; ++v) {
            const float4 vw = __ldg(&views[v]);
            const float px = x - vw.x, py = y - vw.y;
            const float dot = fmaf(px, vw.z, py * vw.w);
            const float crs = fmaf(vw.z, py, -vw.w * px);
            const float *qv = q + (size_t)v * Cp;
            acc0 += fbp_sample(g, qv, dot, crs);
            acc1 += fbp_sample(g, qv, fmaf(g.delta, vw.z, dot), fmaf(-g.delta, vw.w, crs));
        }
        const size_t o = (size_t)i * g.n + j;
        img[o] = dbeta * acc0;
        if (j + 1 < g.n) img[o + 1] = dbeta * acc1;
    }
}

} // namespace mvct

using namespace mvct;

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t _e = (call);                                                         \
        if (_e != cudaSuccess)                                                           \
            return mvct_fail(MVCT_ECUDA, "%s: %s", #call, cudaGetErrorString(_e));       \
    } while (0)

int mvct_fbp_tables(mvct_plan_s *P)
{
    // fan-beam ramp table g(k a), k = -(C-1) .. C-1, and the cosine weights D cos(gamma_c)
    const int C = P->geo.C;
    const double fan = P->g.fan_angle_rad > 0 ? P->g.fan_angle_rad
                                              : 2.0 * std::asin((P->g.fov_cm / 2.0) / P->g.sad_cm);
    const double a = fan / C, pi = 3.14159265358979323846;
    std::vector<float> gt(2 * C - 1), cw(C);
    for (int k = -(C - 1); k <= C - 1; ++k) {
        double v = 0.0;
        if (k == 0) v = 1.0 / (8.0 * a * a);
        else if (k % 2 != 0) {
            const double sn = std::sin(k * a);
            v = -1.0 / (2.0 * pi * pi * sn * sn);
        }
        gt[k + C - 1] = (float)v;
    }
    for (int c = 0; c < C; ++c)
        cw[c] = (float)(P->g.sad_cm * std::cos((c - (C - 1) / 2.0 + P->g.channel_offset) * a));
    if (cudaMalloc(&P->fbp_g, sizeof(float) * (2 * C - 1)) != cudaSuccess ||
        cudaMalloc(&P->fbp_cos, sizeof(float) * C) != cudaSuccess ||
        cudaMalloc(&P->fbp_q, sizeof(float) * (size_t)P->geo.V * (C + 4)) != cudaSuccess)
        return mvct_fail(MVCT_ENOMEM, "mvct_plan_create: FBP tables");
    if (cudaMemcpy(P->fbp_g, gt.data(), sizeof(float) * (2 * C - 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->fbp_cos, cw.data(), sizeof(float) * C, cudaMemcpyHostToDevice) != cudaSuccess)
        return mvct_fail(MVCT_ECUDA, "mvct_plan_create: FBP table upload");
    P->fbp_a = (float)a;
    return MVCT_OK;
}

extern "C" int mvct_fbp(mvct_plan P, const float *d_sino, float *d_img, void *stream)
{
    if (!P) return mvct_fail(MVCT_EINVAL, "mvct_fbp: null plan");
    {
        const int rc = mvct_check_ptrs(P->device, stream, "mvct_fbp", {d_sino, d_img});
        if (rc) return rc;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != P->device) cudaSetDevice(P->device);
    cudaStream_t st = (cudaStream_t)stream;
    const Geo &g = P->geo;
    k_fbp_filter<<<g.V, kThreads, sizeof(float) * g.C, st>>>(g, d_sino, P->fbp_g, P->fbp_cos, P->fbp_a,
                                                             P->fbp_q);
    const int work = g.n * ((g.n + 1) / 2);
    const int grid = std::max(1, std::min((work + kThreads - 1) / kThreads, P->num_sms * 16));
    k_fbp_back<<<grid, kThreads, 0, st>>>(g, P->views, P->fbp_q, (float)(2.0 * 3.14159265358979323846 / g.V),
                                          d_img);
    cudaError_t e = cudaGetLastError();
    if (prev != P->device && prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return mvct_fail(MVCT_ECUDA, "mvct_fbp: %s", cudaGetErrorString(e));
    return MVCT_OK;
}
