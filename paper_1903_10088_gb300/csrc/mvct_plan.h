// Host-side plan object and the internal launchers shared by the C-ABI entry
// points (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <vector>

#include "mvct.h"
#include "mvct_device.cuh"

namespace mvct {

// One slice of a loop launch (device copy read by the loop kernel).
struct SliceDesc {
    Geo g;
    const float4 *rays;
    const int *ray_range;     // [V*C] p_lo | (p_hi + 1) << 16 (see joseph_warp)
    const float4 *views;
    const float *p;           // measured log projections [V][C]
    const float *w;           // statistical weights [V][C]
    const float *D;           // surrogate diagonal [n][n]
    float *mu0, *mu1;         // row 0 of the padded ping-pong images
    float *muT0, *muT1;       // and of their transposes
    // 16-bit storage (mvct_recon_opts.storage): row 0 of the padded 16-bit copies
    // of the ping-pong images and transposes that the reprojection reads, and the
    // 16-bit p and w (unused with FP32 storage)
    void *hm0, *hm1, *hmT0, *hmT1;
    const void *hp, *hw;
    float4 *e4;               // [Vs][C] per-ray (u_c, m, prescaled residual, flag)
    float *tile_part;         // [n_tiles][groups-1][32*32] partial tiles
    unsigned int *tile_flag;  // [n_tiles][groups-1] publication stamps
    float *best;              // best iterate (or null)
    double *phi_hist;         // [n_iter]
    double *lam_hist;         // [n_iter]
    const double *sched;      // lambda replay schedule (or null)
    const int *sorder;        // [S] subset visiting order (or null: 0, 1, ..., S-1)
    mvct_recon_state *st;     // loop state (resume in, final out)
    int tiles_x, n_tiles, groups;
    // balanced phase-B plan (or null: every tile in `groups` groups): per block
    // of the group (tile, view group h, view groups of the tile, first partial
    // slot of the tile), tile -1 for a block without an item
    const int4 *bitems;
    int reducer;              // block that reduces and publishes Phi_n (-1: every block)
    float beta;
};

// A group of consecutive blocks that reconstructs a list of slices in turn.
// Each block group owns kGroupSyncWords words of device memory, two 128-byte
// lines: its barrier counter (word 0 of the first line) and the publication of
// Phi_n by the group's reducer block (PhiPub, the second line).
constexpr int kGroupSyncWords = 64;
struct PhiPub {
    unsigned int stamp;       // barrier count after which the values below are valid
    unsigned int pad;
    double phi;               // Phi_n
    double pass;              // Phi_{n-S+1} + ... + Phi_n
    double phi_old;           // Phi_{n-S} (0 for n < S)
    double pass_last;         // Phi_{n-S} + ... + Phi_{n-1}, the last complete pass (n >= S)
};
static_assert(sizeof(PhiPub) <= 128, "PhiPub fits one line");
inline __host__ __device__ PhiPub *phi_pub(unsigned int *count)
{
    return reinterpret_cast<PhiPub *>(count + 32);
}

struct GroupDesc {
    int block0, nblocks;      // blocks [block0, block0 + nblocks)
    int slice0, nslices;      // slices [slice0, slice0 + nslices) of the slice array
    unsigned int *count;      // the group's barrier counter and PhiPub (kGroupSyncWords words)
    double *partials;         // [nblocks] FP64 partial sums of Phi
};

struct LoopArgs {
    SliceDesc one;            // one-slice launches: the slice
    GroupDesc one_group;      // one-slice launches: all blocks
    const SliceDesc *slices;  // batch launches
    const GroupDesc *groups;
    const int *block_group;   // [grid] group of each block
    Barrier *gbar;            // err (any wait gave up) and data_err (set-up input check)
    unsigned long long *phase_ns; // [2] block 0's time in the two phases (first slice)
    int n_iter;
    double lambda0, dup, ddown, lmin, kappa;
    float eps;
    unsigned long long timeout_ns, spin_cap;
    int debug_unreachable;
    int poisson;              // 1: Poisson data term, e = w - exp(-q)
    int lambda_rule;          // MVCT_LAMBDA_*: which square differences Eq. 4-5 compare
    // One-slice launches of place_per_sm blocks on each of place_sms SMs (0: off):
    // a block takes the index slot * place_sms + (its SM), slot = its arrival
    // order on that SM (counted in sm_slots, zeroed before the launch), so that
    // index b runs on SM b mod place_sms, as the balanced phase-B plan and the
    // phase-F ray deal assume (the hardware, not the block index, picks the SM).
    int *sm_slots;
    int place_sms, place_per_sm;
};

// Batches of up to kParamSlices slices pass their descriptors in the kernel
// parameters (a __grid_constant__ argument read through the constant cache)
// instead of global memory copied to shared memory.
constexpr int kParamSlices = 96;
struct BatchParams {
    SliceDesc sl[kParamSlices];
    GroupDesc gr[kParamSlices];
};

} // namespace mvct

struct mvct_plan_s {
    mvct_geometry g;
    int device = 0;
    int num_sms = 0;
    mvct::Geo geo{};

    float4 *rays = nullptr;     // [V*C] ray table (see mvct_device.cuh)
    int *ray_range = nullptr;   // [V*C] samples walked by each ray: p_lo | (p_hi + 1) << 16
    float4 *views = nullptr;    // [V] source point and central direction
    float *a1t = nullptr;       // [n*n] A^T 1 over all views (support mask = a1t > 0)
    float *a1 = nullptr;        // [V*C] A 1 (projection of the all-ones image), geometry only
    // Zero-row-padded images ((n + 2*kPadRows) rows of n floats; the pointers
    // below address the allocation, row 0 of the image is at + kPadRows*n):
    // pad[0], pad[1] the loop's ping-pong image, pad[2], pad[3] their transposes;
    // pad[0] and pad[2] double as the stand-alone projector's copies.
    float *pad[4] = {nullptr, nullptr, nullptr, nullptr};
    float *pad_ones = nullptr;  // padded all-ones image (its own transpose)
    float *sino_tmp = nullptr;  // [V*C] set-up scratch
    float *D = nullptr;         // [n*n] surrogate diagonal (0 off the support)
    float4 *e4 = nullptr;       // [Vs*C] (u_c, m, prescaled weighted residual, flag) of one subset
    float *tile_part = nullptr; // [n_tiles][groups][32*32] partial tiles of the loop's phase B
    float *back_part = nullptr; // [n_tiles][8][32*32] partial tiles of the stand-alone backprojection
    unsigned int *tile_flag = nullptr; // [n_tiles][groups] publication stamps
    int tiles_x = 0, n_tiles = 0;  // phase-B decomposition of the loop kernel: 32x32 tiles,
    int groups = 1;                // each tile's views dealt to `groups` blocks (one-slice launches)
    int groups_cap = 1;            // partial-tile buffers allocated for this many groups
    int tuned_groups = 0;          // > 0: view groups chosen by the autotuner (overrides `groups`)
    int grid = 0;                  // blocks of one-slice loop launches (<= recon_grid; autotuner)
    int4 *bitems = nullptr;        // [recon_grid] balanced phase-B plan of the default shape (or null)
    int bitems_reducer = -1;       // its block without an item
    double *partials = nullptr; // [partials_cap] per-block FP64 partial sums
    double *partials2 = nullptr;
    int partials_cap = 0;
    double *tv_sum = nullptr;   // [1] scratch scalar
    mvct::Barrier *bar = nullptr;
    unsigned long long *phase_ns = nullptr; // [2] loop phase timers
    void *loop_state = nullptr; // device copy of the resume state
    mvct::SliceDesc *d_slice = nullptr; // the one-slice launch description
    mvct::GroupDesc *d_group = nullptr;
    int *d_block_group = nullptr;       // [recon_grid] zeros
    int *sm_slots = nullptr;            // [num_sms] blocks of the loop launch seen on each SM
    unsigned int *d_count = nullptr;    // group barrier counter and PhiPub (kGroupSyncWords words)
    bool in_batch = false;              // owned by a batch (its scratch is in use there)
    // 16-bit storage buffers (allocated on first use): padded ping-pong image
    // copies and transposes, p and w
    void *pad16[4] = {nullptr, nullptr, nullptr, nullptr};
    void *p16 = nullptr, *w16 = nullptr;
    float *fbp_g = nullptr;             // [2C-1] fan-beam ramp g(k a)
    float *fbp_cos = nullptr;           // [C] D cos(gamma_c)
    float *fbp_q = nullptr;             // [V][C+4] filtered rows, channel c at c + 2, zero ends
    float fbp_a = 0.f;                  // channel pitch (rad)
    double *hist = nullptr;     // [2*hist_cap] phi and lambda per sub-iteration
    double *sched = nullptr;    // [hist_cap] lambda schedule
    int *sorder = nullptr;      // [S] subset visiting order of one-slice launches
    int hist_cap = 0;
    int recon_grid = 0;         // co-resident blocks of the loop kernel
    int reduce_grid = 0;        // grid of the grid-stride reduction kernels
};

namespace mvct {

constexpr int kThreads = 256;        // threads per block of every kernel
constexpr int kWarps = kThreads / 32;

// Stand-alone launchers (mvct_kernels.cu). All enqueue on `st` and return the
// launch status.
cudaError_t launch_pad_transpose(const float *src, float *dst, float *dstT, int n, cudaStream_t st);
cudaError_t launch_forward(const mvct_plan_s *P, const float *img, const float *imgT, float *out,
                           int subset, const float *mul, const float *check_p, int *data_err,
                           cudaStream_t st);
cudaError_t launch_back(const mvct_plan_s *P, const float *sino, float *img, int subset,
                        cudaStream_t st);
cudaError_t launch_tv(const mvct_plan_s *P, const float *img, float eps, float *grad,
                      double *partials, cudaStream_t st);
cudaError_t launch_tv_grid(int n, const float *img, float eps, float *grad, double *partials, int grid,
                           cudaStream_t st);
cudaError_t launch_weight_a1(const mvct_plan_s *P, const float *w, const float *p, float *out, int *data_err,
                             cudaStream_t st);
cudaError_t launch_residual(const mvct_plan_s *P, const float *img, const float *imgT,
                            const float *p, const float *w, double *partials, float *e_out, cudaStream_t st);
cudaError_t launch_axpy(const mvct_plan_s *P, float *y, const float *x, float a, size_t count, cudaStream_t st);
cudaError_t launch_final_sum(const double *a, int na, double ca, const double *b, int nb, double cb,
                             double *out, cudaStream_t st);
cudaError_t launch_setup_back(const mvct_plan_s *P, const float *wa1, float cb, float mu0,
                              int init_from_input, const float *init, float *mu, float *muT,
                              cudaStream_t st);
cudaError_t launch_fill(float *dst, size_t count, float value, cudaStream_t st);

// Row 0 of a zero-row-padded image buffer.
inline float *pad_row0(float *buf, int n) { return buf + (size_t)kPadRows * n; }
inline size_t pad_floats(int n) { return (size_t)(n + 2 * kPadRows) * n; }

// Persistent loop (mvct_recon.cu).
// Largest persistent grid (8 co-resident blocks on each of up to 160 SMs).
#define MVCT_MAX_RECON_GRID 1280
int recon_occupancy(mvct_plan_s *P);
// View groups per tile for a group of nblocks blocks; `override_h` > 0 forces
// that count (autotuner), clamped to the plan's buffers and its views per subset.
int slice_groups(const mvct_plan_s *P, int nblocks, int override_h = 0);

// Balanced phase-B plan of a one-slice launch of `grid` blocks on num_sms SMs
// (block b assumed on SM b mod num_sms): every SM gets r - 1 items of half a
// tile's views (r = grid / num_sms blocks per SM) and one small item of a tile
// split into 2..groups_cap groups; one block stays without an item. False (and
// nothing written) when the sizes do not allow it. The placement is only an
// assumption (the hardware decides it); the results do not depend on it.
bool balanced_items(int n_tiles, int Vs, int groups_cap, int grid, int num_sms, std::vector<int4> &items,
                    int &idle_block);

} // namespace mvct

// FBP tables of a plan (mvct_fbp.cu).
int mvct_fbp_tables(mvct_plan_s *P);

// The TV smoothing eps is applied in FP32 (inside the square root of every
// pixel term): it must be finite, > 0 and stay a normal float when rounded,
// otherwise a flat region gives 0 * rsqrt(0) = NaN gradients.
inline bool mvct_eps_ok(double eps)
{
    return eps > 0 && std::isfinite(eps) && (float)eps >= FLT_MIN && std::isfinite((float)eps);
}

// Error reporting shared by the translation units (mvct_api.cu).
int mvct_fail(int code, const char *fmt, ...);

// Every pointer must be non-null device (or managed) memory of `device`:
// otherwise MVCT_EINVAL naming `who`, before anything is launched. While
// `stream` is being captured into a CUDA graph only the null test is made.
int mvct_check_ptrs(int device, void *stream, const char *who, std::initializer_list<const void *> ptrs);
