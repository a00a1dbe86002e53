// Host-side plan object and the internal launchers shared by the C-ABI entry
// points (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include "mvct.h"
#include "mvct_device.cuh"

struct mvct_plan_s {
    mvct_geometry g;
    int device = 0;
    int num_sms = 0;
    mvct::Geo geo{};

    float4 *rays = nullptr;     // [V*C] ray table (see mvct_device.cuh)
    float4 *views = nullptr;    // [V] source point and central direction
    float *a1t = nullptr;       // [n*n] A^T 1 over all views (support mask = a1t > 0)
    float *ones_img = nullptr;  // [n*n] all ones (its own transpose)
    float *imgT = nullptr;      // [n*n] transpose scratch of the stand-alone projector
    float *sino_tmp = nullptr;  // [V*C] set-up scratch
    float *mu1 = nullptr;       // [n*n] second image buffer of the loop
    float *muT0 = nullptr;      // [n*n] transposes of the two loop buffers
    float *muT1 = nullptr;
    float *D = nullptr;         // [n*n] surrogate diagonal (0 off the support)
    float4 *e4 = nullptr;       // [Vs*C] (u_c, m, prescaled weighted residual, flag) of one subset
    float *tile_part = nullptr; // [n_tiles][groups-1][32*32] partial tile backprojections
    unsigned int *tile_flag = nullptr; // [n_tiles][groups-1] publication stamps
    int tiles_x = 0, n_tiles = 0, groups = 1; // phase-B decomposition of the loop kernel
    double *partials = nullptr; // [partials_cap] per-block FP64 partial sums
    double *partials2 = nullptr;
    int partials_cap = 0;
    double *tv_sum = nullptr;   // [1] scratch scalar
    mvct::Barrier *bar = nullptr;
    void *loop_state = nullptr; // device copy of the resume state
    double *hist = nullptr;     // [2*hist_cap] phi and lambda per sub-iteration
    double *sched = nullptr;    // [hist_cap] lambda schedule
    int hist_cap = 0;
    int recon_grid = 0;         // co-resident blocks of the loop kernel
    int reduce_grid = 0;        // grid of the grid-stride reduction kernels
};

namespace mvct {

constexpr int kThreads = 256;        // threads per block of every kernel
constexpr int kWarps = kThreads / 32;

// Stand-alone launchers (mvct_kernels.cu). All enqueue on `st` and return the
// launch status.
cudaError_t launch_transpose(const float *src, float *dst, int n, cudaStream_t st);
cudaError_t launch_forward(const mvct_plan_s *P, const float *img, const float *imgT, float *out,
                           int subset, const float *mul, const float *check_p, int *data_err,
                           cudaStream_t st);
cudaError_t launch_back(const mvct_plan_s *P, const float *sino, float *img, int subset,
                        cudaStream_t st);
cudaError_t launch_tv(const mvct_plan_s *P, const float *img, float eps, float *grad,
                      double *partials, cudaStream_t st);
cudaError_t launch_tv_grid(int n, const float *img, float eps, float *grad, double *partials, int grid,
                           cudaStream_t st);
cudaError_t launch_residual(const mvct_plan_s *P, const float *img, const float *imgT,
                            const float *p, const float *w, double *partials, cudaStream_t st);
cudaError_t launch_final_sum(const double *a, int na, double ca, const double *b, int nb, double cb,
                             double *out, cudaStream_t st);
cudaError_t launch_setup_back(const mvct_plan_s *P, const float *wa1, float cb, float mu0,
                              int init_from_input, float *mu, float *muT, cudaStream_t st);
cudaError_t launch_fill(float *dst, size_t count, float value, cudaStream_t st);

// Persistent loop (mvct_recon.cu).
int recon_occupancy(mvct_plan_s *P);

} // namespace mvct

// Error reporting shared by the translation units (mvct_api.cu).
int mvct_fail(int code, const char *fmt, ...);
