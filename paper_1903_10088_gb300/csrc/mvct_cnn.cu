// Learned warm start: an 8-layer 3x3 CNN (1 -> 32 -> ... -> 32 -> 1 channels,
// ReLU after layers 1-7, residual output out = x + f(x)) that maps a scaled FBP
// image to a scaled start image for the OS-TV loop. BF16 weights and
// activations, FP32 accumulation, hand-written forward and backward kernels:
//  * 32 -> 32 layers: the forward convolution and the input gradient (the same
//    kernel with the flipped, transposed kernel) on the 5th-generation tensor
//    cores (tcgen05.mma into TMEM, mvct_cnn_tc.cuh); the weight gradient (pixels
//    as the reduction dimension, per-block partials summed in a fixed order) on
//    mma.sync m16n8k16 tiles, FP32 accumulate;
//  * the 1 -> 32 and 32 -> 1 layers: CUDA-core FP32 arithmetic on BF16 data;
//  * fused mean-squared-error loss and Adam.
// Every reduction has a fixed order: training is deterministic.
//
// Layouts: activations [N][H+2][4][W+2][8] BF16 (per padded row four planes of
// channel octets, zero one-pixel border that no kernel writes; see aoff), the
// scaled input x and the output-layer gradient [N][H+2][W+2] FP32. Convolution = cross-correlation:
// y[p] = sum_{tap} x[p + off(tap)] w[tap], tap = 3 ky + kx, off = (ky-1, kx-1).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "mvct_plan.h"

namespace mvct {
namespace cnn {

constexpr int CH = 32;              // hidden channels
constexpr int MID = 6;              // 32 -> 32 layers (2..7)
constexpr int SPAD = 40;            // smem row stride (bf16) of a pixel / kernel row: 80 B, conflict-free ldmatrix
constexpr int TH = 8, TW = 16;      // pixel tile of the weight-gradient kernel k_dw32 (one warp per tile row)

// Parameter vector (FP32): W1[9][32], b1[32], {W_l[9][32 ci][32 co], b_l[32]} x 6, W8[9][32], b8[1]
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + 9 * CH;
constexpr int OFF_MID = OFF_B1 + CH;
constexpr int MID_SIZE = 9 * CH * CH + CH;
constexpr int OFF_W8 = OFF_MID + MID * MID_SIZE;
constexpr int OFF_B8 = OFF_W8 + 9 * CH;
constexpr int NPARAM = OFF_B8 + 1;

__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void ldsm_x4_t(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float *d, unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ size_t apix(int n, int y, int x, int H, int W)
{
    // padded pixel index of image pixel (y, x) (y, x may be -1 .. H / W)
    return ((size_t)n * (H + 2) + (y + 1)) * (W + 2) + (x + 1);
}

// 32-channel activations: per padded row, four planes of channel octets,
// [N][H+2][4][W+2][8] BF16 with a zero one-pixel border. Element offset of octet
// q (channels 8q .. 8q+7, 16 bytes) of pixel (y, x), y in -1..H, x in -1..W: a
// warp's 16-byte accesses to consecutive pixels of one octet are contiguous, and
// the tensor memory accelerator fetches a tile's strip as whole octet rows.
__device__ __forceinline__ size_t aoff(int n, int y, int x, int q, int H, int W)
{
    return (((size_t)n * (H + 2) + (y + 1)) * 4 + q) * (size_t)(W + 2) * 8 + (size_t)(x + 1) * 8;
}

__device__ __forceinline__ uint4 pack_bf16x8(const float *v)
{
    uint4 o;
    __nv_bfloat162 *b = (__nv_bfloat162 *)&o;
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    return o;
}

// ---- weight and bias gradient of a 32 -> 32 layer on tensor cores ---------
// part[block][tap][ci][co] = sum over the block's pixels p of
//   a[p + off(tap)][ci] * d[p][co]   (a: layer input, d: pre-activation gradient)
// part[block][9*32*32 + co] = sum over the block's pixels of d[p][co]
// (the row stride of part is MID_SIZE, the layer's slice of the parameter vector).
// One warp per tap (9 warps) on mma.sync tensor-core tiles; warps 0-7 also sum the bias
// gradient, one tile row each. Blocks stride over the output tiles.
__global__ void __launch_bounds__(288) k_dw32(const __nv_bfloat16 *__restrict__ a,
                                              const __nv_bfloat16 *__restrict__ d, float *__restrict__ part,
                                              int N, int H, int W)
{
    __shared__ __align__(16) __nv_bfloat16 s_a[(TH + 2) * (TW + 2) * SPAD];
    __shared__ __align__(16) __nv_bfloat16 s_d[TH * TW * SPAD];
    __shared__ float s_b[TH][CH];
    const int tid = threadIdx.x, lane = tid & 31, tap = tid >> 5;
    const int ky = tap / 3, kx = tap - 3 * (tap / 3);
    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    const int n_tiles = N * tiles_x * tiles_y;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
    float bsum = 0.f; // warps 0-7: channel `lane` of tile row `tap`
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int n = tile / (tiles_x * tiles_y), rem = tile - n * tiles_x * tiles_y;
        const int y0 = (rem / tiles_x) * TH, x0 = (rem % tiles_x) * TW;
        __syncthreads();
        for (int k = tid; k < (TH + 2) * (TW + 2) * 4; k += 288) {
            const int px = k >> 2, q = k & 3;
            const int ty = px / (TW + 2), tx = px - ty * (TW + 2);
            const int gy = y0 + ty - 1, gx = x0 + tx - 1;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (gy <= H && gx <= W) v = *(const uint4 *)(a + aoff(n, gy, gx, q, H, W));
            *((uint4 *)(s_a + px * SPAD) + q) = v;
        }
        for (int k = tid; k < TH * TW * 4; k += 288) {
            const int px = k >> 2, q = k & 3;
            const int ty = px / TW, tx = px - ty * TW;
            const int gy = y0 + ty, gx = x0 + tx;
            uint4 v = make_uint4(0, 0, 0, 0); // outside the image: zero gradient
            if (gy < H && gx < W) v = *(const uint4 *)(d + aoff(n, gy, gx, q, H, W));
            *((uint4 *)(s_d + px * SPAD) + q) = v;
        }
        __syncthreads();
        if (tap < TH) {
#pragma unroll 4
            for (int j = 0; j < TW; ++j) bsum += __bfloat162float(s_d[(tap * TW + j) * SPAD + lane]);
        }
#pragma unroll 1
        for (int r = 0; r < TH; ++r) { // k-step: the 16 pixels of output row r
            const int q = lane >> 3, rr = lane & 7;
            // A[m = ci][k = px]: stored as pixel rows; matrix q -> (ci block q & 1, px block q >> 1)
            unsigned a_f[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
                ldsm_x4_t(a_f[mt][0], a_f[mt][1], a_f[mt][2], a_f[mt][3],
                          s_a + ((r + ky) * (TW + 2) + kx + (q >> 1) * 8 + rr) * SPAD + mt * 16 + (q & 1) * 8);
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                // B[k = px][n = co]: matrix q -> (co block 2 np + (q >> 1), px block q & 1)
                unsigned b0, b1, b2, b3;
                ldsm_x4_t(b0, b1, b2, b3, s_d + (r * TW + (q & 1) * 8 + rr) * SPAD + (2 * np + (q >> 1)) * 8);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_bf16(acc[mt][2 * np], a_f[mt][0], a_f[mt][1], a_f[mt][2], a_f[mt][3], b0, b1);
                    mma_bf16(acc[mt][2 * np + 1], a_f[mt][0], a_f[mt][1], a_f[mt][2], a_f[mt][3], b2, b3);
                }
            }
        }
    }
    // write this block's partial: rows ci = mt*16 + g (+8), cols co = nt*8 + 2t (+1)
    const int g = lane >> 2, t = lane & 3;
    float *dst = part + (size_t)blockIdx.x * MID_SIZE + tap * CH * CH;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int ci = mt * 16 + g, co = nt * 8 + 2 * t;
            dst[ci * CH + co] = acc[mt][nt][0];
            dst[ci * CH + co + 1] = acc[mt][nt][1];
            dst[(ci + 8) * CH + co] = acc[mt][nt][2];
            dst[(ci + 8) * CH + co + 1] = acc[mt][nt][3];
        }
    if (tap < TH) s_b[tap][lane] = bsum;
    __syncthreads();
    if (tid < CH) {
        float sb = 0.f;
#pragma unroll
        for (int r = 0; r < TH; ++r) sb += s_b[r][tid];
        part[(size_t)blockIdx.x * MID_SIZE + 9 * CH * CH + tid] = sb;
    }
}

// out[k] = sum over b < nb of part[b * stride + k], k < len, in a fixed order:
// warp w of a block sums b = w, w + 8, ... for 32 consecutive k (one per lane),
// then the 8 warp sums are added in warp order.
__global__ void __launch_bounds__(256) k_reduce_parts(const float *__restrict__ part, int nb, int len, int stride,
                                                      float *__restrict__ out)
{
    __shared__ float s[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    float acc = 0.f;
    if (k < len)
        for (int b = warp; b < nb; b += 8) acc += __ldg(part + (size_t)b * stride + k);
    s[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && k < len) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += s[w][lane];
        out[k] = t;
    }
}

// ---- first layer: 1 -> 32 (CUDA cores) -------------------------------------
__global__ void __launch_bounds__(256) k_conv_in(const float *__restrict__ x, const float *__restrict__ w1,
                                                 const float *__restrict__ b1, __nv_bfloat16 *__restrict__ out,
                                                 int N, int H, int W)
{
    __shared__ float s_w[9 * CH + CH];
    for (int k = threadIdx.x; k < 9 * CH + CH; k += 256) s_w[k] = k < 9 * CH ? w1[k] : b1[k - 9 * CH];
    __syncthreads();
    const long long total = (long long)N * H * W;
    for (long long pidx = (long long)blockIdx.x * 256 + threadIdx.x; pidx < total; pidx += (long long)gridDim.x * 256) {
        const int n = (int)(pidx / ((long long)H * W));
        const int rem = (int)(pidx - (long long)n * H * W), y = rem / W, xx = rem - y * W;
        float in[9];
#pragma unroll
        for (int tap = 0; tap < 9; ++tap)
            in[tap] = __ldg(x + apix(n, y + tap / 3 - 1, xx + tap % 3 - 1, H, W));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float t = s_w[9 * CH + 8 * q + c];
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) t = fmaf(in[tap], s_w[tap * CH + 8 * q + c], t);
                v[c] = fmaxf(t, 0.f);
            }
            *(uint4 *)(out + aoff(n, y, xx, q, H, W)) = pack_bf16x8(v);
        }
    }
}

// ---- last layer: 32 -> 1 (CUDA cores), residual output, fused MSE loss -------
// out[p] = x[p] + b8 + sum_tap sum_ci a7[p + off][ci] w8[tap][ci]. With a target
// y: dout[p] = 2 (out - y) / count (padded layout) and per-block FP64 partial
// sums of (out - y)^2.
__global__ void __launch_bounds__(256) k_conv_out(const __nv_bfloat16 *__restrict__ a7,
                                                  const float *__restrict__ w8, const float *__restrict__ b8,
                                                  const float *__restrict__ x, const float *__restrict__ y,
                                                  float *__restrict__ out, float *__restrict__ dout,
                                                  double *__restrict__ loss_part, float inv_count, int N, int H,
                                                  int W)
{
    __shared__ float s_w[9 * CH];
    __shared__ double s_red[8];
    for (int k = threadIdx.x; k < 9 * CH; k += 256) s_w[k] = w8[k];
    __syncthreads();
    const float bias = __ldg(b8);
    const long long total = (long long)N * H * W;
    double lsum = 0.0;
    for (long long pidx = (long long)blockIdx.x * 256 + threadIdx.x; pidx < total; pidx += (long long)gridDim.x * 256) {
        const int n = (int)(pidx / ((long long)H * W));
        const int rem = (int)(pidx - (long long)n * H * W), yy = rem / W, xx = rem - yy * W;
        float acc = bias;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 v = __ldg((const uint4 *)(a7 + aoff(n, yy + tap / 3 - 1, xx + tap % 3 - 1, q, H, W)));
                const __nv_bfloat162 *h = (const __nv_bfloat162 *)&v;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 f = __bfloat1622float2(h[e]);
                    acc = fmaf(f.x, s_w[tap * CH + q * 8 + 2 * e], acc);
                    acc = fmaf(f.y, s_w[tap * CH + q * 8 + 2 * e + 1], acc);
                }
            }
        }
        const size_t pp = apix(n, yy, xx, H, W);
        const float o = __ldg(x + pp) + acc;
        out[(size_t)n * H * W + rem] = o;
        if (y) {
            const float r = o - __ldg(y + (size_t)n * H * W + rem);
            dout[pp] = 2.f * r * inv_count;
            lsum += (double)r * (double)r;
        }
    }
    if (!loss_part) return;
    lsum = warp_sum(lsum);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += s_red[k];
        loss_part[blockIdx.x] = t;
    }
}

// Input gradient of the last layer, masked by layer 7's activation:
// d7[p][ci] = [a7[p][ci] > 0] sum_tap w8[tap][ci] dout[p - off(tap)].
__global__ void __launch_bounds__(256) k_conv_out_bwd(const float *__restrict__ dout, const float *__restrict__ w8,
                                                      const __nv_bfloat16 *__restrict__ a7,
                                                      __nv_bfloat16 *__restrict__ d7, int N, int H, int W)
{
    __shared__ float s_w[9 * CH];
    for (int k = threadIdx.x; k < 9 * CH; k += 256) s_w[k] = w8[k];
    __syncthreads();
    const long long total = (long long)N * H * W;
    for (long long pidx = (long long)blockIdx.x * 256 + threadIdx.x; pidx < total; pidx += (long long)gridDim.x * 256) {
        const int n = (int)(pidx / ((long long)H * W));
        const int rem = (int)(pidx - (long long)n * H * W), yy = rem / W, xx = rem - yy * W;
        float g[9];
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) g[tap] = __ldg(dout + apix(n, yy - (tap / 3 - 1), xx - (tap % 3 - 1), H, W));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const size_t o = aoff(n, yy, xx, q, H, W);
            const uint4 mv = __ldg((const uint4 *)(a7 + o));
            const __nv_bfloat16 *m = (const __nv_bfloat16 *)&mv;
            float v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float t = 0.f;
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) t = fmaf(g[tap], s_w[tap * CH + 8 * q + c], t);
                v[c] = __bfloat162float(m[c]) > 0.f ? t : 0.f;
            }
            *(uint4 *)(d7 + o) = pack_bf16x8(v);
        }
    }
}

// Per-block partials of the weight / bias gradients of the 1-channel layers
// (row stride EDGE_LEN):
//   MODE 0 (first layer): part[b][tap*32 + co] = sum_p xs[p + off] d1[p][co],
//                          part[b][288 + co]   = sum_p d1[p][co]
//   MODE 1 (last layer):  part[b][tap*32 + ci] = sum_p a7[p + off][ci] dout[p],
//                          part[b][288]        = sum_p dout[p] (289 .. 319 zero)
// narrow = xs / dout: FP32 padded [N][H+2][W+2]; wide = d1 / a7: BF16 padded
// octet planes (aoff). 320 threads: warp w < 9 owns tap w (lane = channel), warp 9 the bias.
// Blocks stride over 8 x 16 output tiles staged in shared memory, the shifted
// operand with its one-pixel halo.
constexpr int EDGE_LEN = 9 * CH + CH;
template <int MODE>
__global__ void __launch_bounds__(320) k_dw_edge(const float *__restrict__ narrow,
                                                 const __nv_bfloat16 *__restrict__ wide, float *__restrict__ part,
                                                 int N, int H, int W)
{
    constexpr int HP = (TH + 2) * (TW + 2);      // halo tile pixels
    constexpr int WP = MODE == 1 ? HP : TH * TW; // pixels of the staged wide tile
    constexpr int NP = MODE == 1 ? TH * TW : HP; // pixels of the staged narrow tile
    __shared__ __align__(16) __nv_bfloat16 s_w[WP * CH];
    __shared__ float s_n[NP];
    __shared__ float s_r[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    const int n_tiles = N * tiles_x * tiles_y;
    const int ky = warp / 3, kx = warp - 3 * (warp / 3);
    float acc = 0.f;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int n = tile / (tiles_x * tiles_y), rem = tile - n * tiles_x * tiles_y;
        const int y0 = (rem / tiles_x) * TH, x0 = (rem % tiles_x) * TW;
        __syncthreads();
        for (int k = tid; k < WP * 4; k += 320) {
            const int px = k >> 2, q = k & 3;
            const int tw = MODE == 1 ? TW + 2 : TW, o = MODE == 1 ? 1 : 0;
            const int ty = px / tw, tx = px - ty * tw;
            const int gy = y0 + ty - o, gx = x0 + tx - o;
            const bool ok = MODE == 1 ? (gy <= H && gx <= W) : (gy < H && gx < W);
            uint4 v = make_uint4(0, 0, 0, 0);
            if (ok) v = *(const uint4 *)(wide + aoff(n, gy, gx, q, H, W));
            *((uint4 *)(s_w + px * CH) + q) = v;
        }
        for (int px = tid; px < NP; px += 320) {
            const int tw = MODE == 0 ? TW + 2 : TW, o = MODE == 0 ? 1 : 0;
            const int ty = px / tw, tx = px - ty * tw;
            const int gy = y0 + ty - o, gx = x0 + tx - o;
            const bool ok = MODE == 0 ? (gy <= H && gx <= W) : (gy < H && gx < W);
            s_n[px] = ok ? __ldg(narrow + apix(n, gy, gx, H, W)) : 0.f;
        }
        __syncthreads();
        if (warp < 9) {
#pragma unroll 4
            for (int p = 0; p < TH * TW; ++p) {
                const int py = p / TW, pxx = p - py * TW;
                const int hp = (py + ky) * (TW + 2) + pxx + kx; // the shifted pixel in the halo tile
                if (MODE == 1)
                    acc = fmaf(__bfloat162float(s_w[hp * CH + lane]), s_n[p], acc);
                else
                    acc = fmaf(s_n[hp], __bfloat162float(s_w[p * CH + lane]), acc);
            }
        } else if (MODE == 0) {
#pragma unroll 4
            for (int p = 0; p < TH * TW; ++p) acc += __bfloat162float(s_w[p * CH + lane]);
        } else {
            for (int p = lane; p < TH * TW; p += 32) acc += s_n[p];
        }
    }
    float *dst = part + (size_t)blockIdx.x * EDGE_LEN;
    if (warp < 9) {
        dst[warp * CH + lane] = acc;
    } else if (MODE == 0) {
        dst[9 * CH + lane] = acc;
    } else {
        s_r[lane] = acc;
        __syncwarp();
        if (lane == 0) {
            float t = 0.f;
            for (int k = 0; k < 32; ++k) t += s_r[k];
            dst[9 * CH] = t;
        } else {
            dst[9 * CH + lane] = 0.f;
        }
    }
}

// Adam step on the FP32 master parameters (bias-corrected), then the BF16 /
// rounded copies used by the kernels: wf = BF16-rounded FP32 parameters,
// wk_fwd[l][tap][co][ci] and wk_bwd[l][tap][ci][co] (flipped taps) BF16.
__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPARAM) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

__global__ void k_refresh(const float *__restrict__ w, float *__restrict__ wf, __nv_bfloat16 *__restrict__ wk_fwd,
                          __nv_bfloat16 *__restrict__ wk_bwd)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPARAM) return;
    const float r = __bfloat162float(__float2bfloat16_rn(w[k]));
    wf[k] = r;
    if (k >= OFF_MID && k < OFF_W8) {
        const int l = (k - OFF_MID) / MID_SIZE, e = (k - OFF_MID) % MID_SIZE;
        if (e < 9 * CH * CH) {
            const int tap = e / (CH * CH), ci = (e / CH) % CH, co = e % CH;
            const __nv_bfloat16 b = __float2bfloat16_rn(w[k]);
            wk_fwd[(((size_t)l * 9 + tap) * CH + co) * CH + ci] = b;
            wk_bwd[(((size_t)l * 9 + (8 - tap)) * CH + ci) * CH + co] = b;
        }
    }
}

__global__ void k_fill_f32(float *p, long long count, float v)
{
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x)
        p[k] = v;
}

// Scaled padded input: xs[n][y+1][x+1] = scale * img[n][y][x] (border untouched).
__global__ void k_scale_in(const float *__restrict__ img, float scale, float *__restrict__ xs, int N, int H, int W)
{
    const long long total = (long long)N * H * W;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(k / ((long long)H * W));
        const int rem = (int)(k - (long long)n * H * W), y = rem / W, x = rem - y * W;
        xs[apix(n, y, x, H, W)] = scale * img[k];
    }
}

__global__ void k_scale(const float *__restrict__ a, float s, float *__restrict__ b, long long count)
{
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x)
        b[k] = s * a[k];
}

} // namespace cnn
} // namespace mvct

#include "mvct_cnn_tc.cuh" // the 32 -> 32 convolutions on tcgen05 (uses CH and apix above)

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using namespace mvct;
using namespace mvct::cnn;

struct mvct_cnn_s {
    int device = 0, num_sms = 0, nmax = 0, H = 0, W = 0;
    float scale = 10.f;
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *wf = nullptr; // [NPARAM]
    __nv_bfloat16 *wk_fwd = nullptr, *wk_bwd = nullptr;                          // [6][9][32][32]
    float *xs = nullptr, *ys = nullptr, *dout = nullptr;                         // padded / plain FP32
    float *tout = nullptr;                                                         // training-pass output
    __nv_bfloat16 *act[7] = {};                                                   // a1 .. a7 (padded NHWC)
    __nv_bfloat16 *dgrad[2] = {};                                                 // ping-pong pre-activation gradients
    float *part = nullptr;                                                         // weight-gradient partials
    double *loss_part = nullptr, *h_loss = nullptr;
    int part_blocks = 0, steps = 0;
    int *tc_err = nullptr;   // set by a tensor-core convolution whose wait gave up
    int tc_grid = 0;         // persistent blocks of the tensor-core convolutions
    unsigned long long wait_ns = 1000000000ull; // longest mbarrier wait of those convolutions
    int debug_stall = 0;     // test knob: their copy warps issue nothing
};

namespace {

#define CKC(call)                                                                        \
    do {                                                                                 \
        cudaError_t _e = (call);                                                         \
        if (_e != cudaSuccess)                                                           \
            return mvct_fail(MVCT_ECUDA, "%s: %s", #call, cudaGetErrorString(_e));       \
    } while (0)

struct Dev {
    int prev = -1;
    explicit Dev(int d)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
    }
    ~Dev()
    {
        int c;
        if (prev >= 0 && cudaGetDevice(&c) == cudaSuccess && c != prev) cudaSetDevice(prev);
    }
};

void free_cnn(mvct_cnn_s *c)
{
    if (!c) return;
    void *p[] = {c->w,    c->m,    c->v,         c->g,         c->wf,        c->wk_fwd,   c->wk_bwd, c->xs,
                 c->ys,   c->dout, c->tout,      c->part,      c->loss_part, c->dgrad[0], c->dgrad[1],
                 c->tc_err};
    for (void *q : p)
        if (q) cudaFree(q);
    for (auto *a : c->act)
        if (a) cudaFree(a);
    if (c->h_loss) cudaFreeHost(c->h_loss);
    delete c;
}

int grid_for(const mvct_cnn_s *c, long long work, int per_block)
{
    const long long want = (work + per_block - 1) / per_block;
    return (int)std::max<long long>(1, std::min<long long>(want, (long long)c->num_sms * 8));
}

// forward through the network for n images already scaled into c->xs; writes the
// (scaled) output to `out` and, with a target, dout and the loss partials.
int cnn_forward(mvct_cnn_s *c, int n, float *out, bool with_target, cudaStream_t st)
{
    const int H = c->H, W = c->W;
    const long long pix = (long long)n * H * W;
    k_conv_in<<<grid_for(c, pix, 256), 256, 0, st>>>(c->xs, c->wf + OFF_W1, c->wf + OFF_B1, c->act[0], n, H, W);
    for (int l = 0; l < MID; ++l) {
        tc::k_conv32_tc<0><<<c->tc_grid, tc::THREADS, tc::SMEM_BYTES, st>>>(
            c->act[l], c->wk_fwd + (size_t)l * 9 * CH * CH, c->wf + OFF_MID + l * MID_SIZE + 9 * CH * CH, nullptr,
            c->act[l + 1], n, H, W, c->tc_err, c->wait_ns, c->debug_stall);
    }
    const int gb = grid_for(c, pix, 256);
    k_conv_out<<<gb, 256, 0, st>>>(c->act[6], c->wf + OFF_W8, c->wf + OFF_B8, c->xs, with_target ? c->ys : nullptr, out,
                                   c->dout, with_target ? c->loss_part : nullptr, 1.f / (float)pix, n, H, W);
    CKC(cudaGetLastError());
    return gb;
}

int cnn_backward(mvct_cnn_s *c, int n, cudaStream_t st)
{
    const int H = c->H, W = c->W;
    const long long pix = (long long)n * H * W;
    const int PB = c->part_blocks;
    // last layer: weight and bias gradient (W8 and b8 are contiguous in the
    // parameter vector), then the input gradient masked by a7
    k_dw_edge<1><<<PB, 320, 0, st>>>(c->dout, c->act[6], c->part, n, H, W);
    k_reduce_parts<<<(9 * CH + 1 + 31) / 32, 256, 0, st>>>(c->part, PB, 9 * CH + 1, EDGE_LEN, c->g + OFF_W8);
    k_conv_out_bwd<<<grid_for(c, pix, 256), 256, 0, st>>>(c->dout, c->wf + OFF_W8, c->act[6], c->dgrad[0], n, H, W);
    int cur = 0;
    for (int l = MID - 1; l >= 0; --l) {
        // layer l+2 (0-based mid index l): input act[l], pre-activation gradient dgrad[cur];
        // weights then bias, contiguous in the parameter vector
        k_dw32<<<PB, 288, 0, st>>>(c->act[l], c->dgrad[cur], c->part, n, H, W);
        k_reduce_parts<<<(MID_SIZE + 31) / 32, 256, 0, st>>>(c->part, PB, MID_SIZE, MID_SIZE,
                                                            c->g + OFF_MID + l * MID_SIZE);
        // input gradient, masked by the previous activation (act[l])
        tc::k_conv32_tc<1><<<c->tc_grid, tc::THREADS, tc::SMEM_BYTES, st>>>(
            c->dgrad[cur], c->wk_bwd + (size_t)l * 9 * CH * CH, nullptr, c->act[l], c->dgrad[cur ^ 1], n, H, W, c->tc_err,
            c->wait_ns, c->debug_stall);
        cur ^= 1;
    }
    // first layer: weight and bias gradient (W1 and b1 contiguous) from the scaled input
    k_dw_edge<0><<<PB, 320, 0, st>>>(c->xs, c->dgrad[cur], c->part, n, H, W);
    k_reduce_parts<<<(EDGE_LEN + 31) / 32, 256, 0, st>>>(c->part, PB, EDGE_LEN, EDGE_LEN, c->g + OFF_W1);
    CKC(cudaGetLastError());
    return MVCT_OK;
}

int check_batch(const mvct_cnn_s *c, int n)
{
    if (!c) return mvct_fail(MVCT_EINVAL, "mvct_cnn: null network");
    if (n < 1 || n > c->nmax) return mvct_fail(MVCT_EINVAL, "mvct_cnn: batch %d outside 1..%d", n, c->nmax);
    return MVCT_OK;
}

} // namespace

extern "C" int32_t mvct_cnn_param_count(void) { return NPARAM; }

extern "C" int mvct_cnn_create(int32_t nmax, int32_t h, int32_t w, double scale, const float *params, mvct_cnn *out)
{
    if (!out) return mvct_fail(MVCT_EINVAL, "mvct_cnn_create: out is NULL");
    *out = nullptr;
    if (nmax < 1 || h < 1 || w < 1 || h > 8192 || w > 8192 || !params || !(scale > 0))
        return mvct_fail(MVCT_EINVAL, "mvct_cnn_create: invalid arguments");
    mvct_cnn_s *c = new mvct_cnn_s();
    CKC(cudaGetDevice(&c->device));
    CKC(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    c->nmax = nmax;
    c->H = h;
    c->W = w;
    c->scale = (float)scale;
    c->part_blocks = c->num_sms * 2;
    const size_t padpix = (size_t)nmax * (h + 2) * (w + 2);
    bool ok = true;
    auto alloc = [&](void **p, size_t bytes) { ok = ok && cudaMalloc(p, bytes) == cudaSuccess; };
    alloc((void **)&c->w, sizeof(float) * NPARAM);
    alloc((void **)&c->m, sizeof(float) * NPARAM);
    alloc((void **)&c->v, sizeof(float) * NPARAM);
    alloc((void **)&c->g, sizeof(float) * NPARAM);
    alloc((void **)&c->wf, sizeof(float) * NPARAM);
    alloc((void **)&c->wk_fwd, sizeof(__nv_bfloat16) * MID * 9 * CH * CH);
    alloc((void **)&c->wk_bwd, sizeof(__nv_bfloat16) * MID * 9 * CH * CH);
    alloc((void **)&c->xs, sizeof(float) * padpix);
    alloc((void **)&c->ys, sizeof(float) * (size_t)nmax * h * w);
    alloc((void **)&c->tout, sizeof(float) * (size_t)nmax * h * w);
    alloc((void **)&c->dout, sizeof(float) * padpix);
    for (auto &a : c->act) alloc((void **)&a, sizeof(__nv_bfloat16) * padpix * CH);
    for (auto &d : c->dgrad) alloc((void **)&d, sizeof(__nv_bfloat16) * padpix * CH);
    alloc((void **)&c->part, sizeof(float) * (size_t)c->part_blocks * MID_SIZE);
    alloc((void **)&c->loss_part, sizeof(double) * c->num_sms * 8);
    alloc((void **)&c->tc_err, sizeof(int));
    c->tc_grid = c->num_sms * 2; // 2 blocks of 93.5 KB shared memory per SM
    ok = ok && cudaFuncSetAttribute(tc::k_conv32_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tc::SMEM_BYTES) == cudaSuccess &&
         cudaFuncSetAttribute(tc::k_conv32_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES) ==
             cudaSuccess;
    ok = ok && cudaMallocHost((void **)&c->h_loss, sizeof(double) * c->num_sms * 8) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_cnn(c);
        return mvct_fail(MVCT_ENOMEM, "mvct_cnn_create: allocation failed (batch %d, %d x %d)", nmax, h, w);
    }
    // zero borders (never written), moments, and the parameters
    cudaError_t e = cudaMemset(c->xs, 0, sizeof(float) * padpix);
    if (e == cudaSuccess) e = cudaMemset(c->dout, 0, sizeof(float) * padpix);
    for (auto &a : c->act)
        if (e == cudaSuccess) e = cudaMemset(a, 0, sizeof(__nv_bfloat16) * padpix * CH);
    for (auto &d : c->dgrad)
        if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(__nv_bfloat16) * padpix * CH);
    if (e == cudaSuccess) e = cudaMemset(c->m, 0, sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = cudaMemset(c->v, 0, sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = cudaMemset(c->tc_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(c->w, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_refresh<<<(NPARAM + 255) / 256, 256>>>(c->w, c->wf, c->wk_fwd, c->wk_bwd);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        free_cnn(c);
        return mvct_fail(MVCT_ECUDA, "mvct_cnn_create: %s", cudaGetErrorString(e));
    }
    *out = c;
    return MVCT_OK;
}

extern "C" void mvct_cnn_destroy(mvct_cnn c)
{
    if (!c) return;
    Dev d(c->device);
    cudaDeviceSynchronize();
    free_cnn(c);
}

extern "C" int mvct_cnn_get_params(mvct_cnn c, float *params_out)
{
    if (!c || !params_out) return mvct_fail(MVCT_EINVAL, "mvct_cnn_get_params: null argument");
    Dev d(c->device);
    CKC(cudaMemcpy(params_out, c->w, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    return MVCT_OK;
}

extern "C" int mvct_cnn_set_wait(mvct_cnn c, double timeout_ms, int32_t debug_stall)
{
    if (!c) return mvct_fail(MVCT_EINVAL, "mvct_cnn_set_wait: null network");
    if (!(timeout_ms > 0) || timeout_ms > 60000.0)
        return mvct_fail(MVCT_EINVAL, "mvct_cnn_set_wait: timeout_ms must be in (0, 60000]");
    if (debug_stall != 0 && debug_stall != 1) return mvct_fail(MVCT_EINVAL, "mvct_cnn_set_wait: debug_stall must be 0 or 1");
    c->wait_ns = (unsigned long long)(timeout_ms * 1e6);
    c->debug_stall = debug_stall;
    return MVCT_OK;
}

extern "C" int mvct_cnn_status(mvct_cnn c, void *stream)
{
    if (!c) return mvct_fail(MVCT_EINVAL, "mvct_cnn_status: null network");
    int rc = mvct_check_ptrs(c->device, stream, "mvct_cnn_status", {});
    if (rc) return rc;
    Dev d(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    int terr = 0;
    CKC(cudaMemcpyAsync(&terr, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    if (terr) {
        CKC(cudaMemsetAsync(c->tc_err, 0, sizeof(int), st));
        CKC(cudaStreamSynchronize(st));
        return mvct_fail(MVCT_ETIMEOUT, "mvct_cnn: a tensor-core convolution gave up waiting (its output is invalid)");
    }
    return MVCT_OK;
}

extern "C" int mvct_cnn_forward(mvct_cnn c, const float *d_in, int32_t n, float *d_out, void *stream)
{
    int rc = check_batch(c, n);
    if (rc) return rc;
    rc = mvct_check_ptrs(c->device, stream, "mvct_cnn_forward", {d_in, d_out});
    if (rc) return rc;
    Dev d(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const long long pix = (long long)n * c->H * c->W;
    k_scale_in<<<grid_for(c, pix, 256), 256, 0, st>>>(d_in, c->scale, c->xs, n, c->H, c->W);
    rc = cnn_forward(c, n, d_out, false, st);
    if (rc < 0) return rc;
    k_scale<<<grid_for(c, pix, 256), 256, 0, st>>>(d_out, 1.f / c->scale, d_out, pix);
    CKC(cudaGetLastError());
    return MVCT_OK;
}

// Loss and parameter gradient for a batch (d_grad: device NPARAM floats or NULL).
static int loss_and_grad(mvct_cnn_s *c, const float *d_in, const float *d_target, int n, double *loss,
                         cudaStream_t st)
{
    const long long pix = (long long)n * c->H * c->W;
    k_scale_in<<<grid_for(c, pix, 256), 256, 0, st>>>(d_in, c->scale, c->xs, n, c->H, c->W);
    k_scale<<<grid_for(c, pix, 256), 256, 0, st>>>(d_target, c->scale, c->ys, pix);
    // the output of the training pass is not returned (the loss and dout are used)
    const int gb = cnn_forward(c, n, c->tout, true, st);
    if (gb < 0) return gb;
    int rc = cnn_backward(c, n, st);
    if (rc) return rc;
    CKC(cudaMemcpyAsync(c->h_loss, c->loss_part, sizeof(double) * gb, cudaMemcpyDeviceToHost, st));
    int terr = 0;
    CKC(cudaMemcpyAsync(&terr, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    if (terr) {
        cudaMemsetAsync(c->tc_err, 0, sizeof(int), st);
        return mvct_fail(MVCT_ETIMEOUT, "mvct_cnn: a tensor-core convolution gave up waiting for its MMAs");
    }
    double s = 0.0;
    for (int b = 0; b < gb; ++b) s += c->h_loss[b];
    if (loss) *loss = s / (double)pix;
    return MVCT_OK;
}

extern "C" int mvct_cnn_grad(mvct_cnn c, const float *d_in, const float *d_target, int32_t n, float *d_grad,
                             double *loss, void *stream)
{
    int rc = check_batch(c, n);
    if (rc) return rc;
    rc = mvct_check_ptrs(c->device, stream, "mvct_cnn_grad", {d_in, d_target});
    if (rc == MVCT_OK && d_grad) rc = mvct_check_ptrs(c->device, stream, "mvct_cnn_grad", {d_grad});
    if (rc) return rc;
    Dev d(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    rc = loss_and_grad(c, d_in, d_target, n, loss, st);
    if (rc) return rc;
    if (d_grad) CKC(cudaMemcpyAsync(d_grad, c->g, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, st));
    return MVCT_OK;
}

extern "C" int mvct_cnn_train_step(mvct_cnn c, const float *d_in, const float *d_target, int32_t n, double lr,
                                   double *loss, void *stream)
{
    int rc = check_batch(c, n);
    if (rc) return rc;
    if (!(lr > 0)) return mvct_fail(MVCT_EINVAL, "mvct_cnn_train_step: lr must be > 0");
    rc = mvct_check_ptrs(c->device, stream, "mvct_cnn_train_step", {d_in, d_target});
    if (rc) return rc;
    Dev d(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    rc = loss_and_grad(c, d_in, d_target, n, loss, st);
    if (rc) return rc;
    c->steps += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)c->steps), c2 = 1.f - std::pow(b2, (float)c->steps);
    k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(c->w, c->m, c->v, c->g, (float)lr, b1, b2, 1e-8f, c1, c2);
    k_refresh<<<(NPARAM + 255) / 256, 256, 0, st>>>(c->w, c->wf, c->wk_fwd, c->wk_bwd);
    CKC(cudaGetLastError());
    return MVCT_OK;
}
