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
//   A strip (a ring of STAGES): [3 rows][4 channel octets][130 pixels][8]
//            BF16 (24,960 B). Each (row, octet) line of the strip is one
//            contiguous run of the padded octet-plane activations (130 pixels x
//            16 B), so the strip arrives as 12 bulk asynchronous copies
//            (cp.async.bulk, the tensor memory accelerator's untiled form)
//            completed on a per-stage mbarrier; at a ragged row end the copies
//            are shortened to the pixels that exist, and the stale rest of the
//            line only reaches accumulator rows of pixels past the row end,
//            which are not written. Tap (ky, kx), K-step kk starts at
//            ((ky*4 + 2kk)*130 + kx)*16 B, LBO = 130*16 B (the next octet).
//   B:       [9 taps][4 input-channel octets][32 co][8] BF16 (18,432 B);
//            tap, kk starts at (tap*4 + 2kk)*32*16 B, LBO = 32*16 B.
// Each persistent block loads its layer's weights once and walks tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...; the strip of the next tile is
// fetched while the current tile's MMAs and epilogue run. Every wait on an
// mbarrier is bounded (global timer), after which the block records an error,
// waits (bounded) for its copy in flight, frees its TMEM and leaves.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace mvct {
namespace cnn {
namespace tc {

constexpr int M = 128;                        // output pixels per tile
constexpr int PIX = M + 2;                    // strip pixels per row (one halo pixel each side)
constexpr int PLANE = PIX * 16;               // one row of one channel octet of the strip (2,080 B)
constexpr int A_BYTES = 3 * 4 * PLANE;        // one strip per stage (24,960 B, a multiple of 128 B)
constexpr int STAGES = 3;                     // strips in flight
constexpr int ACCS = 2;                       // TMEM accumulators (the epilogue of one tile overlaps the next MMAs)
constexpr int B_BYTES = 9 * 4 * 32 * 16;      // 18,432
constexpr int B_OFF = STAGES * A_BYTES;
constexpr int BAR_OFF = B_OFF + B_BYTES;      // full[STAGES], empty[STAGES], tfull[ACCS], tempty[ACCS]
constexpr int NBARS = 2 * STAGES + 2 * ACCS;
constexpr int SMEM_BYTES = BAR_OFF + 8 * NBARS + 16; // + TMEM address slot and the failure flag
constexpr int THREADS = 192;                  // warp 0: copies, warp 1: MMAs, warps 2-5: epilogue
constexpr uint32_t TMEM_COLS = 32 * ACCS;     // 128 lanes x 32 FP32 columns per accumulator
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

__device__ __forceinline__ void arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One contiguous run of `bytes` bytes (a multiple of 16, both addresses 16-byte
// aligned) from global into shared memory, completing on bar.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

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
// in / mask / out: padded octet planes [N][H+2][4][W+2][8] BF16 (aoff);
// wk: [9][32 n][32 k] BF16.
// Warp-specialised pipeline over the block's tiles i = 0, 1, ... (tile
// blockIdx.x + i*gridDim.x): warp 0 fetches strip i into stage i mod STAGES once
// the MMAs of tile i - STAGES have released it (empty); warp 1 waits for the
// strip (full) and for accumulator i mod ACCS to be drained (tempty), issues the
// 18 MMAs and commits them to empty and tfull; warps 2-5 wait for tfull, read
// their TMEM lane quarter (warp w reads lanes 32 (w mod 4) ..), release the
// accumulator (tempty) and write the tile.
// err: set to 1 if a wait gave up (every role then leaves its loop, bounded);
// kLimit: the longest wait on one mbarrier phase, in ns of global time.
// stall (test knob): the copy warp issues nothing.
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_conv32_tc(const __nv_bfloat16 *__restrict__ in,
                                                       const __nv_bfloat16 *__restrict__ wk,
                                                       const float *__restrict__ bias,
                                                       const __nv_bfloat16 *__restrict__ mask,
                                                       __nv_bfloat16 *__restrict__ out, int N, int H, int W,
                                                       int *__restrict__ err, unsigned long long kLimit,
                                                       int stall)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sB = smem + B_OFF;
    uint64_t *bars = (uint64_t *)(smem + BAR_OFF);
    uint32_t *tslot = (uint32_t *)(smem + BAR_OFF + 8 * NBARS);
    volatile int *fail = (volatile int *)(smem + BAR_OFF + 8 * NBARS + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sA_a = smem_u32(smem), sB_a = smem_u32(sB), bar0 = smem_u32(bars);
    auto full_b = [bar0](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty_b = [bar0](int s) { return bar0 + 8u * (uint32_t)(STAGES + s); };
    auto tfull_b = [bar0](int a) { return bar0 + 8u * (uint32_t)(2 * STAGES + a); };
    auto tempty_b = [bar0](int a) { return bar0 + 8u * (uint32_t)(2 * STAGES + ACCS + a); };

    // weights [tap][co][ci] -> [tap][ci octet][co][8 ci]
    for (int k = tid; k < 9 * CH * 4; k += THREADS) {
        const int row = k >> 2, q = k & 3, tap = row >> 5, co = row & 31;
        const uint4 v = __ldg((const uint4 *)(wk + (size_t)row * CH) + q);
        *(uint4 *)(sB + ((tap * 4 + q) * CH + co) * 16) = v;
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full_b(s)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty_b(s)) : "memory");
        }
        for (int a = 0; a < ACCS; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tfull_b(a)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(tempty_b(a)) : "memory"); // 4 epilogue warps
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *fail = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem(); // the weights' generic stores, seen by the tensor cores' async proxy
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    const int segs = (W + M - 1) / M;
    const long long tiles = (long long)N * H * segs;
    const int my_tiles = (long long)blockIdx.x < tiles ? (int)((tiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;
    auto tile_at = [&](int i, int &n, int &y, int &x0) {
        const long long t = blockIdx.x + (long long)i * gridDim.x;
        n = (int)(t / ((long long)H * segs));
        const int rem = (int)(t - (long long)n * H * segs);
        y = rem / segs;
        x0 = (rem - y * segs) * M;
    };
    auto give_up = [&]() {
        *fail = 1;
        atomicExch(err, 1);
    };

    if (warp == 0) {
        // copies: the strip of tile i into stage i mod STAGES (none with the stall
        // test knob: the MMA warp's first wait then runs out)
        if (lane == 0 && !stall) {
            int issued = 0;
            for (int i = 0; i < my_tiles && !*fail; ++i, ++issued) {
                const int s = i % STAGES;
                if (i >= STAGES && !wait_bounded(empty_b(s), (uint32_t)(((i / STAGES) + 1) & 1), kLimit)) {
                    give_up();
                    break;
                }
                int n, y, x0;
                tile_at(i, n, y, x0);
                const uint32_t bytes = (uint32_t)min(PIX, W + 2 - x0) * 16u;
                expect_tx(full_b(s), 12u * bytes);
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        bulk_load(sA_a + s * A_BYTES + (r * 4 + q) * PLANE, in + aoff(n, y - 1 + r, x0 - 1, q, H, W),
                                  bytes, full_b(s));
            }
            // after a failure, copies still in flight land before the block's shared
            // memory is released (a stage's last phase is pending or complete)
            if (*fail)
                for (int i = issued > STAGES ? issued - STAGES : 0; i < issued; ++i)
                    wait_bounded(full_b(i % STAGES), (uint32_t)((i / STAGES) & 1), kLimit);
        }
    } else if (warp == 1) {
        // MMAs of tile i into accumulator i mod ACCS
        if (lane == 0) {
            for (int i = 0; i < my_tiles && !*fail; ++i) {
                const int s = i % STAGES, a = i % ACCS;
                if (!wait_bounded(full_b(s), (uint32_t)((i / STAGES) & 1), kLimit) ||
                    (i >= ACCS && !wait_bounded(tempty_b(a), (uint32_t)(((i / ACCS) + 1) & 1), kLimit))) {
                    give_up();
                    break;
                }
                fence_after();
                const uint32_t a0 = sA_a + s * A_BYTES, d = tmem + (uint32_t)(a * 32);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap - 3 * ky;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint64_t ad = smem_desc(a0 + ((ky * 4 + 2 * kk) * PIX + kx) * 16, PLANE, 128);
                        const uint64_t bd = smem_desc(sB_a + (tap * 4 + 2 * kk) * CH * 16, CH * 16, 128);
                        mma_f16(d, ad, bd, (tap | kk) != 0 ? 1u : 0u);
                    }
                }
                commit(empty_b(s)); // the strip may be refilled once these MMAs are done
                commit(tfull_b(a)); // and the accumulator read
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31, one pixel per thread
        const int quarter = warp & 3;
        for (int i = 0; i < my_tiles; ++i) {
            const int a = i % ACCS;
            const bool ok = wait_bounded(tfull_b(a), (uint32_t)((i / ACCS) & 1), kLimit) && !*fail;
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) give_up();
                break;
            }
            fence_after();
            float acc[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * 32), acc);
            fence_before();
            __syncwarp();
            if (lane == 0) arrive(tempty_b(a)); // the accumulator may take the next MMAs
            int n, y, x0;
            tile_at(i, n, y, x0);
            const int x = x0 + quarter * 32 + lane;
            if (x < W) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const size_t o = aoff(n, y, x, q, H, W);
                    float v[8];
                    if (MODE == 0) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) v[c] = fmaxf(acc[8 * q + c] + __ldg(bias + 8 * q + c), 0.f);
                    } else {
                        const uint4 mv = __ldg((const uint4 *)(mask + o));
                        const __nv_bfloat16 *m = (const __nv_bfloat16 *)&mv;
#pragma unroll
                        for (int c = 0; c < 8; ++c) v[c] = __bfloat162float(m[c]) > 0.f ? acc[8 * q + c] : 0.f;
                    }
                    *(uint4 *)(out + o) = pack_bf16x8(v);
                }
            }
        }
    }
    __syncwarp();
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

} // namespace tc
} // namespace cnn
} // namespace mvct
