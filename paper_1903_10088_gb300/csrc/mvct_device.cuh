// Device-side building blocks of the OS-TV loop (sm_103a).
//
//  * joseph_warp   -- Joseph reprojection of one fan-beam ray by one warp
//                     (Sec. 4.4 "reprojection"): lanes walk consecutive samples
//                     along the driving axis, so the two interpolation taps of a
//                     warp step hit one or two 128-byte rows of the image.
//  * gather_pixel  -- the matched adjoint (Sec. 4.4 "estimation") evaluated per
//                     pixel: for every view of the subset only the channels whose
//                     ray passes within one pixel of the pixel centre can carry a
//                     non-zero Joseph weight; their weights are recomputed from
//                     the same ray table the projector uses. No atomics.
//  * tv_grad_pixel -- gradient of the smoothed isotropic TV (Sec. 2).
//  * grid_sync     -- grid-wide barrier of the persistent loop with a bounded
//                     wait (global timer limit plus a spin cap).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mvct {

// Geometry constants in the form the kernels use them.
struct Geo {
    int n;            // image side
    int V, C;         // views, channels
    int S, Vs;        // subsets, views per subset
    float pc;         // (n - 1) / 2, the centre index
    float delta;      // pixel size (cm)
    float inv_dgamma; // 1 / channel pitch (1/rad)
    float c_mid;      // channel coordinate of the central ray: (C-1)/2 - offset
};

// Per-ray table entry (FP32, built in FP64 on the host):
//   x = u_c   : interpolation coordinate (row index for an x-driven ray, column
//               index for a y-driven ray) where the ray crosses the centre line
//   y = m     : change of that coordinate per sample step along the driving axis
//   z = scale : delta / |d_major|, path length per sample step
//   w = 1 for an x-driven ray (|dx| >= |dy|), 0 for a y-driven ray
// Sample p (column j for x-driven, row i for y-driven) is interpolated at
//   u(p) = fmaf(m, p - pc, u_c).
// Per-view table entry: (S_x, S_y, e_x, e_y), source point and unit central-ray
// direction e = -S/|S|.

template <bool RO>
__device__ __forceinline__ float ldf(const float *p)
{
    if constexpr (RO) return __ldg(p);
    else return *p;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Joseph line integral of one ray, computed by the whole warp (all lanes return
// the same value). img is row-major; imgT is its transpose: a y-driven ray walks
// the rows of img, which are the columns of imgT, so reading imgT keeps the
// warp's accesses contiguous. RO selects read-only-cache loads (only legal when
// the image is not written during the kernel).
template <bool RO>
__device__ __forceinline__ float joseph_warp(const float *img, const float *imgT, int n, float pc,
                                             float4 r, int lane)
{
    const float *src = (r.w > 0.5f) ? img : imgT;
    const float uc = r.x, m = r.y;
    // Samples whose taps can fall inside the image: u(p) in (-1, n). The bounds
    // are widened by one sample; every tap is still bounds-checked below.
    int p_lo = 0, p_hi = n - 1;
    if (m != 0.f) {
        float a = __fdividef(-1.f - uc, m), b = __fdividef((float)n - uc, m);
        float lo = fmaxf(fminf(a, b) + pc, -2.f), hi = fminf(fmaxf(a, b) + pc, (float)n + 1.f);
        p_lo = max(0, (int)floorf(lo) - 1);
        p_hi = min(n - 1, (int)ceilf(hi) + 1);
    } else if (!(uc > -1.f && uc < (float)n)) {
        p_hi = -1;
    }
    float acc = 0.f;
    for (int p = p_lo + lane; p <= p_hi; p += 32) {
        const float u = fmaf(m, (float)p - pc, uc);
        const float fl = floorf(u);
        const int i0 = (int)fl;
        const float f = u - fl;
        const float a = ((unsigned)i0 < (unsigned)n) ? ldf<RO>(src + (size_t)i0 * n + p) : 0.f;
        const float b = ((unsigned)(i0 + 1) < (unsigned)n) ? ldf<RO>(src + (size_t)(i0 + 1) * n + p) : 0.f;
        acc += fmaf(f, b - a, a);
    }
    return warp_sum(acc) * r.z;
}

// sum_k sum_c A[(v_k, c), (i, j)] * val[k*C + c] over the rows k of a subset
// (subset < 0: all views). PRESCALED: val already carries the ray's scale.
// RO: val may be read through the read-only cache.
template <bool PRESCALED, bool RO>
__device__ __forceinline__ float gather_pixel(const Geo &g, const float4 *__restrict__ rays,
                                              const float4 *__restrict__ views, const float *val,
                                              int i, int j, int subset, int rows)
{
    const float fic = (float)i - g.pc, fjc = (float)j - g.pc; // centred indices (exact)
    const float fi = (float)i, fj = (float)j;
    const float x = fjc * g.delta, y = fic * g.delta;          // pixel centre (cm)
    const float d2 = g.delta * g.delta;
    const float hw_scale = g.delta * g.inv_dgamma;
    float acc = 0.f;
    for (int k = 0; k < rows; ++k) {
        const int v = subset < 0 ? k : subset + k * g.S;
        const float4 vw = __ldg(&views[v]);
        const float px = x - vw.x, py = y - vw.y;
        const float dot = fmaf(px, vw.z, py * vw.w);   // along the central ray (> 0)
        const float crs = fmaf(vw.z, py, -vw.w * px);  // across it
        // channel coordinate of the ray through the pixel centre
        const float cc = fmaf(atanf(__fdividef(crs, dot)), g.inv_dgamma, g.c_mid);
        // a ray with a non-zero weight passes within delta of the centre, i.e.
        // within asin(delta/dist) <= delta/sqrt(dist^2 - delta^2) of its angle
        const float hw = fmaf(hw_scale, rsqrtf(fmaxf(fmaf(dot, dot, fmaf(crs, crs, -d2)), 1e-30f)), 0.02f);
        const int c0 = max(0, (int)ceilf(fmaxf(cc - hw, -1.f)));
        const int c1 = min(g.C - 1, (int)floorf(fminf(cc + hw, (float)g.C)));
        const float4 *rr = rays + (size_t)v * g.C;
        const float *vv = val + (size_t)k * g.C;
        for (int c = c0; c <= c1; ++c) {
            const float4 r = __ldg(&rr[c]);
            const bool xd = r.w > 0.5f;
            const float u = fmaf(r.y, xd ? fjc : fic, r.x);
            const float wgt = fmaxf(0.f, 1.f - fabsf(u - (xd ? fi : fj)));
            const float s = ldf<RO>(vv + c);
            acc = fmaf(wgt, PRESCALED ? s : s * r.z, acc);
        }
    }
    return acc;
}

// ---------------------------------------------------------------------------
// Tile splat: the matched backprojection of one subset onto a 32x32 pixel tile.
//
// For a view, every ray that can reach the tile is walked across the tile's 32
// columns (x-driven ray: lane = column, taps at rows i0 and i0+1) or 32 rows
// (y-driven ray: lane = row, taps at columns j0 and j0+1), with exactly the
// projector's weights: u = fmaf(m, p - pc, u_c), (1-f) to tap i0 and f to tap
// i0+1, times the ray's prescaled residual. Each lane only touches its own
// column (or row) of a warp-private accumulator tile, in channel order, so the
// result is deterministic without atomics.
//
// Accumulator layout: 32 rows x 33 floats. Rays whose slope (dy/dx for x-driven,
// dx/dy for y-driven) is >= 0 use column index j, rays with negative slopes use
// the mirrored column 31 - j; either way the 32 lanes of a step fall in at least
// 16 distinct banks.
// ---------------------------------------------------------------------------
constexpr int kTile = 32;
constexpr int kAccStride = 33;
constexpr int kAccFloats = kTile * kAccStride;

// Channel window [x, y] of the rays of a view that can carry a non-zero weight to
// a pixel of the tile whose first row/column are (i_lo, j_lo): a ray with a
// non-zero Joseph weight passes within one pixel of that pixel's centre, so it
// crosses the box of pixel centres grown by one pixel; the window is that box's
// angular extent seen from the source, widened by one channel. Whole warp calls.
__device__ __forceinline__ int2 tile_window(const Geo &g, float4 vw, int i_lo, int j_lo, int lane)
{
    const int corner = lane & 3;
    const float jj = (corner & 1) ? (float)(j_lo + kTile) : (float)(j_lo - 1);
    const float ii = (corner & 2) ? (float)(i_lo + kTile) : (float)(i_lo - 1);
    const float px = (jj - g.pc) * g.delta - vw.x, py = (ii - g.pc) * g.delta - vw.y;
    const float dot = fmaf(px, vw.z, py * vw.w);
    const float crs = fmaf(vw.z, py, -vw.w * px);
    float lo, hi;
    if (dot > 0.f) {
        lo = hi = fmaf(atanf(__fdividef(crs, dot)), g.inv_dgamma, g.c_mid);
    } else { // source inside the grown box (extreme geometry): every channel
        lo = -INFINITY;
        hi = INFINITY;
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int c0 = max(0, (int)floorf(fmaxf(lo, -2.f)) - 1);
    const int c1 = min(g.C - 1, (int)ceilf(fminf(hi, (float)g.C + 1.f)) + 1);
    return make_int2(c0, c1);
}

// Splat channels [c0, c1] of one view onto the warp's accumulator tile.
// e4row[c] = (u_c, m, prescaled residual, x-driven flag) of the view's rays.
// pj = j_lo + lane - pc, pi = i_lo + lane - pc. RO: e4row may use the
// read-only cache (not when it was written earlier in the same kernel).
template <bool MIRROR, bool RO>
__device__ __forceinline__ void splat_channels(float *acc, float4 *stage, const float4 *e4row, int c0,
                                               int c1, float pj, float pi, int i_lo, int j_lo, int lane)
{
    for (int cb = c0; cb <= c1; cb += 32) {
        const int c = cb + lane;
        if (c <= c1) {
            if constexpr (RO) stage[lane] = __ldg(e4row + c);
            else stage[lane] = e4row[c];
        }
        __syncwarp();
        const int cnt = min(32, c1 - cb + 1);
        for (int t = 0; t < cnt; ++t) {
            const float4 r = stage[t];
            if (r.w > 0.5f) { // x-driven: this lane's column, rows a and a+1
                const float u = fmaf(r.y, pj, r.x);
                const float fl = floorf(u);
                const int a = (int)fl - i_lo;
                const float w1 = (u - fl) * r.z, w0 = r.z - w1;
                const int col = MIRROR ? (kTile - 1) - lane : lane;
                if ((unsigned)a < (unsigned)kTile) acc[a * kAccStride + col] += w0;
                if ((unsigned)(a + 1) < (unsigned)kTile) acc[(a + 1) * kAccStride + col] += w1;
            } else {          // y-driven: this lane's row, columns a and a+1
                const float u = fmaf(r.y, pi, r.x);
                const float fl = floorf(u);
                const int a = (int)fl - j_lo;
                const float w1 = (u - fl) * r.z, w0 = r.z - w1;
                float *row = acc + lane * kAccStride;
                if ((unsigned)a < (unsigned)kTile) row[MIRROR ? (kTile - 1) - a : a] += w0;
                if ((unsigned)(a + 1) < (unsigned)kTile) row[MIRROR ? (kTile - 2) - a : a + 1] += w1;
            }
        }
        __syncwarp();
    }
}

// d/dmu[i][j] of TV_eps = sum sqrt(dx^2 + dy^2 + eps) with forward differences
// and zero differences across the last column / row. If phi is non-null it
// receives sqrt(dx^2 + dy^2 + eps) of the term anchored at (i, j).
template <bool RO>
__device__ __forceinline__ float tv_grad_pixel(const float *img, int n, int i, int j, float eps,
                                               float *phi)
{
    const size_t r = (size_t)i * n + j;
    const float m = ldf<RO>(img + r);
    const float right = (j + 1 < n) ? ldf<RO>(img + r + 1) : m;
    const float down = (i + 1 < n) ? ldf<RO>(img + r + n) : m;
    const float dx = right - m, dy = down - m;
    const float q = fmaf(dx, dx, fmaf(dy, dy, eps));
    float gsum = -(dx + dy) * rsqrtf(q);
    if (phi) *phi = sqrtf(q);
    if (j > 0) {
        const float a = ldf<RO>(img + r - 1);
        const float dxl = m - a;
        const float dyl = (i + 1 < n) ? ldf<RO>(img + r - 1 + n) - a : 0.f;
        gsum += dxl * rsqrtf(fmaf(dxl, dxl, fmaf(dyl, dyl, eps)));
    }
    if (i > 0) {
        const float b = ldf<RO>(img + r - n);
        const float dyu = m - b;
        const float dxu = (j + 1 < n) ? ldf<RO>(img + r - n + 1) - b : 0.f;
        gsum += dyu * rsqrtf(fmaf(dxu, dxu, fmaf(dyu, dyu, eps)));
    }
    return gsum;
}

// ---------------------------------------------------------------------------
// Grid barrier with a bounded wait.
// ---------------------------------------------------------------------------
struct Barrier {
    unsigned int count;   // arrivals at the current barrier
    unsigned int gen;     // barrier generation
    int err;              // 1: a block gave up waiting (timeout)
    int data_err;         // 1: non-finite / negative input detected in set-up
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Every block calls this with the same `expected` (the grid size). Returns false
// in every thread of the block if any block timed out; the caller then leaves
// the kernel. The wait ends at timeout_ns of global time or after spin_cap polls
// (each poll is an L2 round trip plus a short sleep), whichever comes first.
__device__ __forceinline__ bool grid_sync(Barrier *bar, unsigned int expected,
                                          unsigned long long timeout_ns,
                                          unsigned long long spin_cap)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int gen = ld_acquire(&bar->gen);
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
        if (arrived == expected) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            st_release(&bar->gen, gen + 1u);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned long long spins = 0;
            while (ld_acquire(&bar->gen) == gen) {
                if (*(volatile int *)&bar->err) { ok = 0; break; }
                ++spins;
                if (spins > spin_cap ||
                    ((spins & 31u) == 0 && global_ns() - t0 > timeout_ns)) {
                    atomicExch(&bar->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(40);
            }
        }
        __threadfence();
        if (*(volatile int *)&bar->err) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

} // namespace mvct
