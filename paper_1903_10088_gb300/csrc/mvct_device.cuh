// Device-side building blocks of the OS-TV loop (sm_103a).
//
//  * joseph_warp   -- Joseph reprojection of one fan-beam ray by one warp
//                     (Sec. 4.4 "reprojection"): lanes walk consecutive samples
//                     along the driving axis, so the two interpolation taps of a
//                     warp step hit one or two 128-byte rows of the image.
//  * splat_views   -- the matched adjoint (Sec. 4.4 "estimation") of one subset
//                     on a 32x32 pixel tile: each ray that can reach the tile is
//                     walked across it with the projector's own weights into
//                     warp-private shared-memory tiles. No atomics.
//  * tv_grad_pixel -- gradient of the smoothed isotropic TV (Sec. 2).
//  * group_sync    -- barrier of a group of blocks of the persistent loop with a
//                     bounded wait (global timer limit plus a spin cap).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

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

// Load one stored element (FP32, BF16 or FP16) widened to FP32.
template <bool RO, typename TS>
__device__ __forceinline__ float ldv(const TS *p)
{
    if constexpr (std::is_same<TS, float>::value) {
        return ldf<RO>(p);
    } else if constexpr (std::is_same<TS, __nv_bfloat16>::value) {
        if constexpr (RO) return __bfloat162float(__ldg(p));
        else return __bfloat162float(*p);
    } else {
        if constexpr (RO) return __half2float(__ldg(p));
        else return __half2float(*p);
    }
}

// Round an FP32 value to the storage type (round to nearest even).
template <typename TS>
__device__ __forceinline__ TS to_storage(float v)
{
    if constexpr (std::is_same<TS, float>::value) return v;
    else if constexpr (std::is_same<TS, __nv_bfloat16>::value) return __float2bfloat16_rn(v);
    else return __float2half_rn(v);
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

// floor(u) for |u| < 2^22 without conversion instructions: adding 1.5 * 2^23
// with round-toward-minus-infinity leaves floor(u) in the low mantissa bits of
// the sum (the spacing there is 1). Returns floor(u) as int and u - floor(u).
// The projector and the backprojection both use it, so their taps and weights
// agree bit for bit.
__device__ __forceinline__ int floor_frac(float u, float &frac)
{
    const float t = __fadd_rd(u, 12582912.0f);
    frac = u - (t - 12582912.0f);
    return __float_as_int(t) - 0x4B400000;
}

// Images used by the projector carry kPadRows zero rows above and below
// (row-major, width n): row index r of the image is stored at (r + kPadRows) * n.
// A tap row clamped into [-kPadRows, n + kPadRows - 1] therefore needs no bounds
// test: every clamped tap lands on a zero row, exactly like a tap outside the image.
constexpr int kPadRows = 2;

// Joseph line integral of one ray, computed by the whole warp (all lanes return
// the same value). img is row-major; imgT is its transpose: a y-driven ray walks
// the rows of img, which are the columns of imgT, so reading imgT keeps the
// warp's accesses contiguous. RO selects read-only-cache loads (only legal when
// the image is not written during the kernel). TS is the stored element type
// (FP32, BF16 or FP16); taps are widened to FP32 and the sum is FP32. range
// packs the samples p_lo .. p_hi the ray walks (those whose taps can fall inside
// the image, widened by one; taps outside land on the zero rows), computed on
// the host with the plan's ray table: p_lo | (p_hi + 1) << 16.
template <bool RO, typename TS = float>
__device__ __forceinline__ float joseph_warp(const TS *img, const TS *imgT, int n, float pc,
                                             float4 r, int range, int lane)
{
    // img / imgT point at row 0 of zero-row-padded buffers (see kPadRows)
    const TS *src = (r.w > 0.5f) ? img : imgT;
    const float uc = r.x, m = r.y;
    const int p_lo = range & 0xffff, p_hi = (range >> 16) - 1;
    const int rmin = -kPadRows, rmax = n + kPadRows - 2;
    // Four samples per lane per step, all eight taps loaded before use.
    constexpr int U = 4;
    float acc = 0.f;
    int p = p_lo + lane;
    float pf = (float)p - pc;
    for (; p + (U - 1) * 32 <= p_hi; p += U * 32, pf += (float)(U * 32)) {
        float f[U], ta[U], tb[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const float u = fmaf(m, pf + (float)(q * 32), uc);
            const int i0 = min(max(floor_frac(u, f[q]), rmin), rmax);
            const TS *t = src + (i0 * n + p + q * 32);
            ta[q] = ldv<RO>(t);
            tb[q] = ldv<RO>(t + n);
        }
#pragma unroll
        for (int q = 0; q < U; ++q) acc += fmaf(f[q], tb[q] - ta[q], ta[q]);
    }
    for (; p <= p_hi; p += 32, pf += 32.f) {
        float f;
        const int i0 = min(max(floor_frac(fmaf(m, pf, uc), f), rmin), rmax);
        const TS *t = src + (i0 * n + p);
        const float a = ldv<RO>(t), b = ldv<RO>(t + n);
        acc += fmaf(f, b - a, a);
    }
    return warp_sum(acc) * r.z;
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
// Accumulator layout: 32 x 32 floats per warp, row-major for the warps that take
// the views whose central ray is x-driven and column-major for the warps that
// take the y-driven ones. A ray of the warp's own type then touches element
// lane + 32 a (bank = lane) for any slope: no bank conflicts; rays of the other
// type (views within the fan's half-angle of 45 degrees) touch 32 lane + a, whose
// rows a spread over the banks at slopes near +-1. The block sum transposes the
// column-major part through a padded 32 x 33 scratch tile.
// ---------------------------------------------------------------------------
constexpr int kTile = 32;
constexpr int kAccStride = 33; // row pitch of the padded scratch tile
constexpr int kAccFloats = kTile * kAccStride;
constexpr float kWinMargin = 0.01f; // channels

// Channel window [x, y] of the rays of a view that can carry a non-zero weight to
// a pixel of the tile whose first row/column are (i_lo, j_lo): a ray with a
// non-zero Joseph weight passes within one pixel of that pixel's centre, so it
// crosses the box of pixel centres grown by one pixel; the window holds the
// channels inside that box's angular extent seen from the source, widened by
// kWinMargin channels against rounding (the FP32 angle is good to ~2e-4
// channels, a ray's FP32 tap decisions to ~1e-4). Whole warp calls.
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
    const int c0 = max(0, (int)ceilf(fmaxf(lo, -2.f) - kWinMargin));
    const int c1 = min(g.C - 1, (int)floorf(fminf(hi, (float)g.C + 1.f) + kWinMargin));
    return make_int2(c0, c1);
}

// Staging of a view's rays for the splat: (u_c, m, path length x value, flag).
// StageE4: the loop kernel's per-subset buffer, already in that form.
// StageSino: the ray table plus a sinogram row, read through the read-only cache.
struct StageE4 {
    const float4 *row; // e4 + k*C
    __device__ __forceinline__ float4 operator()(int c) const { return row[c]; }
};
struct StageSino {
    const float4 *rays; // ray table row of the view: rays + v*C
    const float *vals;  // sinogram row: sino + k*C
    __device__ __forceinline__ float4 operator()(int c) const
    {
        const float4 r = __ldg(rays + c);
        return make_float4(r.x, r.y, r.z * __ldg(vals + c), r.w);
    }
};

// 32-bit shared-memory addressing for the splat's accumulator read-modify-writes.
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void smem_add(unsigned addr, float v)
{
    float old;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(old) : "r"(addr));
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(old + v));
}

// Splat channels [c0, c1] of one view onto the warp's accumulator tile.
// pj = j_lo + lane - pc, pi = i_lo + lane - pc. Per batch of 32 staged rays a
// warp vote picks a loop without the per-ray type test when all of them are
// x-driven (or all y-driven), the usual case away from the 45-degree directions.
template <bool TRANS, class Stage>
__device__ __forceinline__ void splat_channels(float *acc, float4 *stage, const Stage &load, int c0,
                                               int c1, float pj, float pi, int i_lo, int j_lo, int lane)
{
    const unsigned acc0 = smem_addr(acc);
    // element (row r, col c) of the tile: r*32 + c (TRANS = false) or c*32 + r
    const unsigned lane_major = acc0 + 4u * (unsigned)lane;   // + 128 a: bank = lane
    const unsigned lane_minor = acc0 + 128u * (unsigned)lane; // + 4 a
    auto x_step = [&](const float4 &r) { // x-driven: this lane's column, rows a and a+1
        float f;
        const int a = floor_frac(fmaf(r.y, pj, r.x), f) - i_lo;
        const float w1 = f * r.z, w0 = r.z - w1;
        const unsigned ad = TRANS ? lane_minor + 4u * (unsigned)a : lane_major + 128u * (unsigned)a;
        if ((unsigned)a < (unsigned)kTile) smem_add(ad, w0);
        if ((unsigned)(a + 1) < (unsigned)kTile) smem_add(ad + (TRANS ? 4u : 128u), w1);
    };
    auto y_step = [&](const float4 &r) { // y-driven: this lane's row, columns a and a+1
        float f;
        const int a = floor_frac(fmaf(r.y, pi, r.x), f) - j_lo;
        const float w1 = f * r.z, w0 = r.z - w1;
        const unsigned ad = TRANS ? lane_major + 128u * (unsigned)a : lane_minor + 4u * (unsigned)a;
        if ((unsigned)a < (unsigned)kTile) smem_add(ad, w0);
        if ((unsigned)(a + 1) < (unsigned)kTile) smem_add(ad + (TRANS ? 128u : 4u), w1);
    };
    for (int cb = c0; cb <= c1; cb += 32) {
        const int c = cb + lane;
        bool xd = true, yd = true; // lanes past c1 stage nothing and agree with both
        if (c <= c1) {
            const float4 r = load(c);
            stage[lane] = r;
            xd = r.w > 0.5f;
            yd = !xd;
        }
        const bool all_x = __all_sync(0xffffffffu, xd), all_y = __all_sync(0xffffffffu, yd);
        __syncwarp();
        const int cnt = min(32, c1 - cb + 1);
        if (all_x) {
            for (int t = 0; t < cnt; ++t) x_step(stage[t]);
        } else if (all_y) {
            for (int t = 0; t < cnt; ++t) y_step(stage[t]);
        } else {
            for (int t = 0; t < cnt; ++t) {
                const float4 r = stage[t];
                if (r.w > 0.5f) x_step(r);
                else y_step(r);
            }
        }
        __syncwarp();
    }
}

// Largest number of view groups (blocks) that share one tile.
constexpr int kMaxGroups = 8;
// Views whose windows are staged in shared memory at a time by splat_views.
constexpr int kWinBatch = 64;

// One block splats subset rows onto the 32x32 tile (i_lo, j_lo): the rows
// k = order[j] (or k = j without an order) for j = ja, ja + jstep, ... (< jb).
// Views whose central ray is x-driven go to warps [0, wpos) (row-major
// accumulators), the others to warps [wpos, nw) (column-major), wpos = nw/2.
// Per batch of up to kWinBatch views, the warps first compute the views' channel windows into
// s_win; then the channels of each class, concatenated in view order, are cut
// into equal contiguous runs, one per warp of the class (a run may span several
// views or part of one). Returns wpos; after the closing block barrier tile_sums
// gives the tile.
template <class MakeStage>
__device__ __forceinline__ int splat_views(const Geo &g, const float4 *__restrict__ views, int subset,
                                           int ja, int jb, int jstep, const int *__restrict__ order,
                                           int i_lo, int j_lo, float (*s_acc)[kAccFloats],
                                           float4 (*s_stage)[32], int4 *s_win, const MakeStage &make_stage)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int wpos = nw / 2;
    const bool trans = warp >= wpos;
    const int nmine = trans ? nw - wpos : wpos;
    const int q = trans ? warp - wpos : warp;
    float *acc = s_acc[warp];
    float4 *stage = s_stage[warp];
    const float pj = (float)(j_lo + lane) - g.pc, pi = (float)(i_lo + lane) - g.pc;
    for (int k = lane; k < kAccFloats; k += 32) acc[k] = 0.f;
    __syncwarp();
    const int nviews = jb > ja ? (jb - ja + jstep - 1) / jstep : 0;
    for (int base = 0; base < nviews; base += kWinBatch) {
        const int cnt = min(kWinBatch, nviews - base);
        // windows: (c0, c1, layout class, v) of view `idx` of the batch
        for (int idx = warp; idx < cnt; idx += nw) {
            const int j = ja + (base + idx) * jstep;
            const int k = order ? __ldg(order + j) : j;
            const int v = subset < 0 ? k : subset + k * g.S;
            const float4 vw = __ldg(&views[v]);
            const int2 win = tile_window(g, vw, i_lo, j_lo, lane);
            if (lane == 0) s_win[idx] = make_int4(win.x, win.y, (fabsf(vw.z) < fabsf(vw.w)) ? 1 : 0, k);
        }
        __syncthreads();
        // this class's channel counts of entries lane and lane + 32, exclusive prefix sums
        int len[2], pre[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int idx = lane + 32 * h;
            len[h] = 0;
            if (idx < cnt) {
                const int4 w = s_win[idx];
                if ((w.z != 0) == trans) len[h] = max(0, w.y - w.x + 1);
            }
            int x = len[h];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            pre[h] = x - len[h];
        }
        const int tot0 = __shfl_sync(0xffffffffu, pre[0] + len[0], 31);
        pre[1] += tot0;
        const int total = tot0 + __shfl_sync(0xffffffffu, pre[1] - tot0 + len[1], 31);
        const int lo = (int)(((long long)q * total) / nmine), hi = (int)(((long long)(q + 1) * total) / nmine);
        for (int idx = 0; idx < cnt && lo < hi; ++idx) {
            const int h = idx >> 5, src = idx & 31;
            const int p0 = __shfl_sync(0xffffffffu, h ? pre[1] : pre[0], src);
            const int l0 = __shfl_sync(0xffffffffu, h ? len[1] : len[0], src);
            if (l0 == 0 || p0 + l0 <= lo) continue;
            if (p0 >= hi) break;
            const int4 w = s_win[idx];
            const int c0 = w.x + (max(lo, p0) - p0), c1 = w.x + (min(hi, p0 + l0) - p0) - 1;
            const int k = w.w;
            const int v = subset < 0 ? k : subset + k * g.S;
            const auto st = make_stage(k, v);
            if (trans) splat_channels<true>(acc, stage, st, c0, c1, pj, pi, i_lo, j_lo, lane);
            else splat_channels<false>(acc, stage, st, c0, c1, pj, pi, i_lo, j_lo, lane);
        }
        __syncthreads(); // s_win is rewritten by the next batch
    }
    __syncthreads();
    return wpos;
}

// Block sums of the tile (after splat_views): v[u] = pixel idx = threadIdx.x + u*256,
// (ii, jj) = (idx / 32, idx % 32): the row-major accumulators of warps [0, wpos)
// in warp order, plus the column-major ones of warps [wpos, nw) in warp order,
// transposed through s_acc[0] (padded rows of 33). Whole block; s_acc is
// overwritten. Requires 4 * blockDim.x == 1024.
__device__ __forceinline__ void tile_sums(float (*s_acc)[kAccFloats], int nw, int wpos, float v[4])
{
    float vt[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int idx = threadIdx.x + u * blockDim.x;
        float a = 0.f, b = 0.f;
        for (int w = 0; w < wpos; ++w) a += s_acc[w][idx];
        for (int w = wpos; w < nw; ++w) b += s_acc[w][idx];
        v[u] = a;
        vt[u] = b; // column-major element idx: pixel (idx % 32, idx / 32)
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int idx = threadIdx.x + u * blockDim.x;
        s_acc[0][(idx >> 5) * kAccStride + (idx & 31)] = vt[u];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int idx = threadIdx.x + u * blockDim.x;
        v[u] += s_acc[0][(idx & 31) * kAccStride + (idx >> 5)];
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
    unsigned int count;   // arrivals since launch (monotonic; barrier k completes at (k+1)*G)
    unsigned int pad0[31];
    int err;              // 1: a block gave up waiting (timeout)
    int data_err;         // 1: non-finite / negative input detected in set-up
    int place_err;        // 1: the loop's blocks were not spread over the SMs as its launch assumed
    unsigned int pad1[29];
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

__device__ __forceinline__ unsigned int ld_relaxed(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void add_release(unsigned int *p, unsigned int v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acquire() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Start moving the 128-byte line holding p into this SM's L1 (no register result).
__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Barrier number k (0, 1, 2, ... counted identically by every block) among the
// nblocks blocks that share `count`: each block adds one arrival with release
// semantics and polls (relaxed) until the counter reaches (k+1)*nblocks + extra,
// then takes an acquire fence. extra > 0 makes the barrier unreachable (test
// knob). The poll is tight; every 64th poll also reads *err and the global
// timer, and after 4096 polls each of those adds a short sleep. Returns false in
// every thread of the block if the wait hit timeout_ns or spin_cap, or if any
// block has set *err; the caller then leaves the kernel.
__device__ __forceinline__ bool group_sync(unsigned int *count, int *err, unsigned int k,
                                           unsigned int nblocks, unsigned int extra,
                                           unsigned long long timeout_ns, unsigned long long spin_cap)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int target = (k + 1u) * nblocks + extra;
        add_release(count, 1u);
        unsigned long long spins = 0, t0 = 0;
        while ((int)(ld_relaxed(count) - target) < 0) {
            ++spins;
            if ((spins & 63u) == 0) {
                if (*(volatile int *)err) {
                    ok = 0;
                    break;
                }
                if (spins == 64) {
                    t0 = global_ns();
                } else if (spins > spin_cap || global_ns() - t0 > timeout_ns) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
                if (spins >= 4096) __nanosleep(64);
            }
        }
        fence_acquire();
        if (*(volatile int *)err) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

} // namespace mvct
