// 32 -> 32 convolution of the warm-start network on the 5th-generation tensor
// cores (tcgen05, sm_100a / sm_103a), included by mvct_cnn.cu.
//
// Implicit GEMM, one tile = 128 consecutive output pixels of one image row:
//   D[128 pixels][32 co] = sum over 9 taps and 2 K-steps of 16 input channels
//                          A_tap[128][16] x B_tap[16][32]        (BF16, FP32 accumulate)
// A_tap is the tile's input strip shifted by the tap offset, B_tap the tap's
// weights. One elected thread issues the 18 tcgen05.mma (M = 128, N = 32,
// K = 16) into a 32-column TMEM accumulator and commits them to an mbarrier;
// the four warps then read their 32 TMEM lanes (tcgen05.ld 32x32b) and write
// bias + ReLU (forward) or the activation mask (input gradient) as BF16.
//
// Shared-memory operands use the K-major layout without swizzle: a core matrix
// is 8 rows (pixels or output channels) x 16 bytes (8 channels of K) stored
// contiguously (128 B); core matrices 8 rows further along M/N are SBO = 128 B
// apart, the next 8 channels along K are LBO bytes apart.
//   A strip: [3 rows][4 channel octets][130 pixels][8] BF16 (24,960 B);
//            tap (ky, kx), K-step kk starts at ((ky*4 + 2kk)*130 + kx)*16 B,
//            LBO = 130*16 B (the next channel octet of the same pixels).
//   B:       [9 taps][4 input-channel octets][32 co][8] BF16 (18,432 B);
//            tap, kk starts at (tap*4 + 2kk)*32*16 B, LBO = 32*16 B.
// Each persistent block loads its layer's weights once and walks tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...; every wait on the mbarrier is
// bounded (global timer), after which the block records an error, frees its
// TMEM and leaves.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace mvct {
namespace cnn {
namespace tc {

constexpr int M = 128;                        // output pixels per tile
constexpr int PIX = M + 2;                    // strip pixels per row (one halo pixel each side)
constexpr int A_BYTES = 3 * 4 * PIX * 16;     // 24,960
constexpr int B_BYTES = 9 * 4 * 32 * 16;      // 18,432
constexpr int BAR_OFF = A_BYTES + B_BYTES;    // 8-byte aligned
constexpr int SMEM_BYTES = BAR_OFF + 16;      // mbarrier + TMEM address slot
constexpr int THREADS = 128;
constexpr uint32_t TMEM_COLS = 32;            // 128 lanes x 32 FP32 columns
// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A and
// B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((uint32_t)(M >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, LBO and SBO in 16-byte units
// (bits 0-13, 16-29, 32-45), descriptor version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
                 "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return done != 0;
}

// Wait for phase `parity` of the mbarrier, at most timeout_ns of global time.
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity, unsigned long long timeout_ns)
{
    if (try_wait(bar, parity)) return true;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (try_wait(bar, parity)) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > timeout_ns) return false;
    }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes into v.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                   "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                   "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// MODE 0 (forward): out = relu(conv(in, wk) + bias).
// MODE 1 (input gradient): out = conv(in, wk) * [mask > 0].
// in / mask / out: padded NHWC [N][H+2][W+2][32] BF16; wk: [9][32 n][32 k] BF16.
// err: set to 1 if a wait for the tensor cores gave up (the block then leaves).
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_conv32_tc(const __nv_bfloat16 *__restrict__ in,
                                                       const __nv_bfloat16 *__restrict__ wk,
                                                       const float *__restrict__ bias,
                                                       const __nv_bfloat16 *__restrict__ mask,
                                                       __nv_bfloat16 *__restrict__ out, int N, int H, int W,
                                                       int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sA = smem, *sB = smem + A_BYTES;
    uint64_t *bar = (uint64_t *)(smem + BAR_OFF);
    uint32_t *tslot = (uint32_t *)(smem + BAR_OFF + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_a = smem_u32(bar), sA_a = smem_u32(sA), sB_a = smem_u32(sB);

    // weights [tap][co][ci] -> [tap][ci octet][co][8 ci]
    for (int k = tid; k < 9 * CH * 4; k += THREADS) {
        const int row = k >> 2, q = k & 3, tap = row >> 5, co = row & 31;
        const uint4 v = __ldg((const uint4 *)(wk + (size_t)row * CH) + q);
        *(uint4 *)(sB + ((tap * 4 + q) * CH + co) * 16) = v;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    const int segs = (W + M - 1) / M;
    const long long tiles = (long long)N * H * segs;
    uint32_t parity = 0;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int n = (int)(t / ((long long)H * segs));
        const int rem = (int)(t - (long long)n * H * segs);
        const int y = rem / segs, x0 = (rem - y * segs) * M;
        // input strip: image rows y-1 .. y+1, pixels x0-1 .. x0+M (padded coordinates are valid up to W)
        for (int k = tid; k < 3 * PIX * 4; k += THREADS) {
            const int q = k & 3, pr = k >> 2, r = pr / PIX, px = pr - r * PIX;
            const int gx = x0 - 1 + px, gy = y - 1 + r;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gx <= W) v = __ldg((const uint4 *)(in + apix(n, gy, gx, H, W) * CH) + q);
            *(uint4 *)(sA + ((r * 4 + q) * PIX + px) * 16) = v;
        }
        fence_async_smem(); // the strip's generic stores, seen by the tensor cores' async proxy
        fence_before();
        __syncthreads();
        if (tid == 0) {
            fence_after();
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int ky = tap / 3, kx = tap - 3 * ky;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const uint64_t ad = smem_desc(sA_a + ((ky * 4 + 2 * kk) * PIX + kx) * 16, PIX * 16, 128);
                    const uint64_t bd = smem_desc(sB_a + (tap * 4 + 2 * kk) * CH * 16, CH * 16, 128);
                    mma_f16(tmem, ad, bd, (tap | kk) != 0 ? 1u : 0u);
                }
            }
            commit(bar_a);
        }
        __syncwarp();
        // every thread waits; the block leaves together if any wait gave up
        const bool ok = __syncthreads_and(wait_bounded(bar_a, parity, 1000000000ull)) != 0;
        parity ^= 1u;
        if (!ok) {
            if (tid == 0) atomicExch(err, 1);
            break;
        }
        fence_after();
        float acc[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), acc);
        const int x = x0 + warp * 32 + lane;
        if (x < W) {
            const size_t base = apix(n, y, x, H, W) * CH;
            uint4 o[4];
            __nv_bfloat162 *ob = (__nv_bfloat162 *)o;
            if (MODE == 0) {
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    ob[c] = __floats2bfloat162_rn(fmaxf(acc[2 * c] + __ldg(bias + 2 * c), 0.f),
                                                  fmaxf(acc[2 * c + 1] + __ldg(bias + 2 * c + 1), 0.f));
            } else {
                uint4 mv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) mv[q] = __ldg((const uint4 *)(mask + base) + q);
                const __nv_bfloat162 *mb = (const __nv_bfloat162 *)mv;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float2 m = __bfloat1622float2(mb[c]);
                    ob[c] = __floats2bfloat162_rn(m.x > 0.f ? acc[2 * c] : 0.f, m.y > 0.f ? acc[2 * c + 1] : 0.f);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) *((uint4 *)(out + base) + q) = o[q];
        }
        fence_before(); // this tile's TMEM reads come before the next tile's MMAs
    }
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

} // namespace tc
} // namespace cnn
} // namespace mvct
