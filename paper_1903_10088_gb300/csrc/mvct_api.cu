// C-ABI entry points: plan construction, argument validation and the
// stand-alone operators (mvct_forward, mvct_back, mvct_tv_grad, mvct_objective).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mvct_plan.h"

using namespace mvct;

static thread_local char g_err[512] = "";

int mvct_fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

extern "C" const char *mvct_last_error(void) { return g_err; }

int mvct_check_ptrs(int device, void *stream, const char *who, std::initializer_list<const void *> ptrs)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusNone;
    }
    for (const void *p : ptrs) {
        if (!p) return mvct_fail(MVCT_EINVAL, "%s: null device pointer", who);
        if (cs != cudaStreamCaptureStatusNone) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return mvct_fail(MVCT_EINVAL, "%s: %p is not CUDA memory", who, p);
        }
        if (a.type == cudaMemoryTypeManaged) continue;
        if (a.type != cudaMemoryTypeDevice || a.device != device)
            return mvct_fail(MVCT_EINVAL, "%s: %p is not device memory of device %d", who, p, device);
    }
    return MVCT_OK;
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t _e = (call);                                                         \
        if (_e != cudaSuccess)                                                           \
            return mvct_fail(MVCT_ECUDA, "%s: %s", #call, cudaGetErrorString(_e));       \
    } while (0)

const double kPi = 3.14159265358979323846;

double fan_of(const mvct_geometry &g)
{
    return g.fan_angle_rad > 0 ? g.fan_angle_rad : 2.0 * std::asin((g.fov_cm / 2.0) / g.sad_cm);
}

int validate(const mvct_geometry *g, int S)
{
    if (!g) return mvct_fail(MVCT_EINVAL, "geometry is NULL");
    if (g->n < 1 || g->n > MVCT_MAX_N) return mvct_fail(MVCT_EINVAL, "n = %d outside 1..%d", g->n, MVCT_MAX_N);
    if (g->n_views < 1 || g->n_channels < 1 || g->n_views > 65536 || g->n_channels > 65536 ||
        (long long)g->n_views * g->n_channels > (1ll << 28))
        return mvct_fail(MVCT_EINVAL, "views/channels out of range (%d x %d)", g->n_views, g->n_channels);
    if (!std::isfinite(g->fov_cm) || !(g->fov_cm > 0)) return mvct_fail(MVCT_EINVAL, "fov_cm must be > 0");
    if (!std::isfinite(g->sad_cm) || !(g->sad_cm > g->fov_cm * std::sqrt(2.0) / 2.0))
        return mvct_fail(MVCT_EINVAL, "sad_cm must exceed fov_cm*sqrt(2)/2 (source outside the image)");
    if (!std::isfinite(g->view0_rad) || !std::isfinite(g->channel_offset) || !std::isfinite(g->fan_angle_rad))
        return mvct_fail(MVCT_EINVAL, "non-finite geometry field");
    if (g->fan_angle_rad >= kPi) return mvct_fail(MVCT_EINVAL, "fan_angle_rad must be < pi");
    if (S < 1 || S > MVCT_MAX_SUBSETS || S > g->n_views || g->n_views % S != 0)
        return mvct_fail(MVCT_EINVAL, "n_subsets = %d must divide n_views = %d (and be <= %d)", S,
                         g->n_views, MVCT_MAX_SUBSETS);
    return MVCT_OK;
}

// Ray and view tables in FP64, stored as FP32 (layout in mvct_device.cuh).
void build_tables(const mvct_geometry &g, int S, std::vector<float4> &rays, std::vector<float4> &views,
                  std::vector<int> &ranges, Geo &geo)
{
    const int n = g.n, V = g.n_views, C = g.n_channels;
    const double delta = g.fov_cm / n, pc = (n - 1) / 2.0;
    const double dg = fan_of(g) / C;
    rays.resize((size_t)V * C);
    ranges.resize((size_t)V * C);
    views.resize(V);
    for (int v = 0; v < V; ++v) {
        const double b = g.view0_rad + 2.0 * kPi * v / V;
        const double sx = g.sad_cm * std::cos(b), sy = g.sad_cm * std::sin(b);
        const double ex = -std::cos(b), ey = -std::sin(b);
        views[v] = make_float4((float)sx, (float)sy, (float)ex, (float)ey);
        for (int c = 0; c < C; ++c) {
            const double gm = (c - (C - 1) / 2.0 + g.channel_offset) * dg;
            const double dx = std::cos(gm) * ex - std::sin(gm) * ey;
            const double dy = std::sin(gm) * ex + std::cos(gm) * ey;
            float4 r;
            if (std::fabs(dx) >= std::fabs(dy)) { // x-driven: walk columns, interpolate rows
                const double m = dy / dx;
                r = make_float4((float)((sy - sx * m) / delta + pc), (float)m, (float)(delta / std::fabs(dx)), 1.f);
            } else {                              // y-driven: walk rows, interpolate columns
                const double m = dx / dy;
                r = make_float4((float)((sx - sy * m) / delta + pc), (float)m, (float)(delta / std::fabs(dy)), 0.f);
            }
            rays[(size_t)v * C + c] = r;
            // samples whose taps can fall inside the image, u(p) in (-1, n), from the
            // stored FP32 u_c and m, widened by one sample on each side (a superset:
            // taps outside land on the zero rows)
            const double uc = r.x, mm = r.y;
            int p_lo = 0, p_hi = n - 1;
            if (mm != 0.0) {
                const double a = (-1.0 - uc) / mm, bb = ((double)n - uc) / mm;
                const double lo = std::max(std::min(a, bb) + pc, -2.0), hi = std::min(std::max(a, bb) + pc, n + 1.0);
                p_lo = std::max(0, (int)std::floor(lo) - 1);
                p_hi = std::min(n - 1, (int)std::ceil(hi) + 1);
            } else if (!(uc > -1.0 && uc < (double)n)) {
                p_hi = -1;
            }
            if (p_hi < p_lo) p_lo = 0, p_hi = -1;
            ranges[(size_t)v * C + c] = p_lo | ((p_hi + 1) << 16);
        }
    }
    geo.n = n;
    geo.V = V;
    geo.C = C;
    geo.S = S;
    geo.Vs = V / S;
    geo.pc = (float)pc;
    geo.delta = (float)delta;
    geo.inv_dgamma = (float)(1.0 / dg);
    geo.c_mid = (float)((C - 1) / 2.0 - g.channel_offset);
}

void free_plan(mvct_plan_s *P)
{
    if (!P) return;
    void *ptrs[] = {P->rays, P->ray_range, P->views, P->a1t, P->a1, P->pad[0], P->pad[1], P->pad[2], P->pad[3],
                    P->pad_ones, P->sino_tmp, P->D, P->e4, P->tile_part, P->back_part, P->tile_flag, P->partials, P->partials2,
                    P->tv_sum, P->bar, P->phase_ns, P->loop_state, P->hist, P->sched,
                    P->d_slice, P->d_group, P->d_block_group, P->d_count, P->sm_slots, P->fbp_g, P->fbp_cos, P->fbp_q, P->sorder,
                    P->pad16[0], P->pad16[1], P->pad16[2], P->pad16[3], P->p16, P->w16, P->bitems};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete P;
}

int check_plan_subset(mvct_plan P, int subset, const char *who)
{
    if (!P) return mvct_fail(MVCT_EINVAL, "%s: null plan", who);
    if (subset < -1 || subset >= P->geo.S)
        return mvct_fail(MVCT_EINVAL, "%s: subset %d outside -1..%d", who, subset, P->geo.S - 1);
    return MVCT_OK;
}

} // namespace

extern "C" int mvct_plan_create(const mvct_geometry *g, int32_t n_subsets, mvct_plan *out)
{
    if (!out) return mvct_fail(MVCT_EINVAL, "mvct_plan_create: out is NULL");
    *out = nullptr;
    int rc = validate(g, n_subsets);
    if (rc) return rc;
    mvct_plan_s *P = new mvct_plan_s();
    P->g = *g;
    CK(cudaGetDevice(&P->device));
    CK(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device));

    std::vector<float4> rays, views;
    std::vector<int> ranges;
    build_tables(*g, n_subsets, rays, views, ranges, P->geo);
    const size_t nn = (size_t)g->n * g->n, R = (size_t)g->n_views * g->n_channels;
    const size_t Rs = (size_t)P->geo.Vs * g->n_channels;
    P->reduce_grid = P->num_sms * 8;
    P->recon_grid = recon_occupancy(P);
    P->partials_cap = std::max(P->reduce_grid, P->recon_grid);
    // phase B of the loop: 32x32 tiles, each tile's views dealt round-robin to
    // `groups` blocks so that tiles x groups fills the grid
    P->tiles_x = (g->n + kTile - 1) / kTile;
    P->n_tiles = P->tiles_x * P->tiles_x;
    P->groups_cap = std::max(1, std::min(kMaxGroups, P->geo.Vs));
    P->groups = std::max(1, std::min(P->groups_cap, P->recon_grid / P->n_tiles));
    P->grid = P->recon_grid;
    std::vector<int4> bitems;
    const bool balanced = balanced_items(P->n_tiles, P->geo.Vs, P->groups_cap, P->recon_grid, P->num_sms, bitems,
                                         P->bitems_reducer);
    const size_t part_floats = (size_t)P->n_tiles * P->groups_cap * kTile * kTile;
    const size_t n_flags = (size_t)P->n_tiles * P->groups_cap;

    bool ok = cudaMalloc(&P->rays, R * sizeof(float4)) == cudaSuccess &&
              cudaMalloc(&P->ray_range, R * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&P->views, g->n_views * sizeof(float4)) == cudaSuccess &&
              cudaMalloc(&P->a1t, nn * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&P->a1, R * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&P->pad[0], pad_floats(g->n) * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&P->pad[1], pad_floats(g->n) * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&P->pad[2], pad_floats(g->n) * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&P->pad[3], pad_floats(g->n) * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&P->pad_ones, pad_floats(g->n) * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&P->sino_tmp, R * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&P->D, nn * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&P->e4, Rs * sizeof(float4)) == cudaSuccess &&
              cudaMalloc(&P->back_part, (size_t)P->n_tiles * 8 * kTile * kTile * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&P->tile_part, part_floats * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&P->tile_flag, n_flags * sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc(&P->partials, P->partials_cap * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&P->partials2, P->partials_cap * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&P->tv_sum, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&P->bar, sizeof(Barrier)) == cudaSuccess &&
              cudaMalloc(&P->phase_ns, 2 * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&P->loop_state, sizeof(mvct_recon_state)) == cudaSuccess &&
              cudaMalloc(&P->d_slice, sizeof(SliceDesc)) == cudaSuccess &&
              cudaMalloc(&P->d_group, sizeof(GroupDesc)) == cudaSuccess &&
              cudaMalloc(&P->d_block_group, sizeof(int) * std::max(1, P->recon_grid)) == cudaSuccess &&
              cudaMalloc(&P->d_count, sizeof(unsigned int) * kGroupSyncWords) == cudaSuccess &&
              cudaMalloc(&P->sm_slots, sizeof(int) * std::max(1, P->num_sms)) == cudaSuccess &&
              cudaMalloc(&P->sorder, sizeof(int) * std::max(1, n_subsets)) == cudaSuccess &&
              (!balanced || cudaMalloc(&P->bitems, sizeof(int4) * P->recon_grid) == cudaSuccess);
    if (!ok) {
        cudaGetLastError();
        free_plan(P);
        return mvct_fail(MVCT_ENOMEM, "mvct_plan_create: device allocation failed (n=%d, %d x %d rays)",
                         g->n, g->n_views, g->n_channels);
    }
    cudaStream_t st = 0;
    cudaError_t e = cudaMemcpy(P->rays, rays.data(), R * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->ray_range, ranges.data(), R * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->views, views.data(), g->n_views * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && balanced)
        e = cudaMemcpy(P->bitems, bitems.data(), sizeof(int4) * P->recon_grid, cudaMemcpyHostToDevice);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaMemset(P->pad[k], 0, pad_floats(g->n) * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(P->pad_ones, 0, pad_floats(g->n) * sizeof(float));
    if (e == cudaSuccess) e = launch_fill(pad_row0(P->pad_ones, g->n), nn, 1.f, st);
    if (e == cudaSuccess) e = launch_fill(P->sino_tmp, R, 1.f, st);
    if (e == cudaSuccess) e = launch_back(P, P->sino_tmp, P->a1t, -1, st); // A^T 1
    if (e == cudaSuccess) {
        const float *ones = pad_row0(P->pad_ones, g->n);
        e = launch_forward(P, ones, ones, P->a1, -1, nullptr, nullptr, nullptr, st); // A 1
    }
    if (e == cudaSuccess) e = cudaMemset(P->bar, 0, sizeof(Barrier));
    if (e == cudaSuccess) e = cudaMemset(P->d_block_group, 0, sizeof(int) * std::max(1, P->recon_grid));
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_plan(P);
        return mvct_fail(MVCT_ECUDA, "mvct_plan_create: %s", cudaGetErrorString(e));
    }
    rc = mvct_fbp_tables(P);
    if (rc) {
        free_plan(P);
        return rc;
    }
    *out = P;
    return MVCT_OK;
}

extern "C" void mvct_plan_destroy(mvct_plan P)
{
    if (!P) return;
    DeviceGuard dg(P->device);
    cudaDeviceSynchronize();
    free_plan(P);
}

extern "C" int mvct_forward(mvct_plan P, const float *d_img, float *d_sino, int32_t subset, void *stream)
{
    int rc = check_plan_subset(P, subset, "mvct_forward");
    if (rc) return rc;
    rc = mvct_check_ptrs(P->device, stream, "mvct_forward", {d_img, d_sino});
    if (rc) return rc;
    DeviceGuard dg(P->device);
    cudaStream_t st = (cudaStream_t)stream;
    float *img = pad_row0(P->pad[0], P->geo.n), *imgT = pad_row0(P->pad[2], P->geo.n);
    CK(launch_pad_transpose(d_img, img, imgT, P->geo.n, st));
    CK(launch_forward(P, img, imgT, d_sino, subset, nullptr, nullptr, nullptr, st));
    return MVCT_OK;
}

extern "C" int mvct_back(mvct_plan P, const float *d_sino, float *d_img, int32_t subset, void *stream)
{
    int rc = check_plan_subset(P, subset, "mvct_back");
    if (rc) return rc;
    rc = mvct_check_ptrs(P->device, stream, "mvct_back", {d_img, d_sino});
    if (rc) return rc;
    DeviceGuard dg(P->device);
    CK(launch_back(P, d_sino, d_img, subset, (cudaStream_t)stream));
    return MVCT_OK;
}

extern "C" int mvct_tv_grad(mvct_plan P, const float *d_img, double eps, float *d_grad,
                            double *d_tv_or_null, void *stream)
{
    if (!P) return mvct_fail(MVCT_EINVAL, "mvct_tv_grad: null plan");
    int rc = mvct_check_ptrs(P->device, stream, "mvct_tv_grad", {d_img, d_grad});
    if (rc == MVCT_OK && d_tv_or_null) rc = mvct_check_ptrs(P->device, stream, "mvct_tv_grad", {d_tv_or_null});
    if (rc) return rc;
    if (!mvct_eps_ok(eps))
        return mvct_fail(MVCT_EINVAL, "mvct_tv_grad: eps must be > 0 and a normal float (>= FLT_MIN)");
    DeviceGuard dg(P->device);
    cudaStream_t st = (cudaStream_t)stream;
    CK(launch_tv(P, d_img, (float)eps, d_grad, P->partials, st));
    if (d_tv_or_null)
        CK(launch_final_sum(P->partials, P->reduce_grid, 1.0, nullptr, 0, 0.0, d_tv_or_null, st));
    return MVCT_OK;
}

extern "C" int mvct_objective(mvct_plan P, const float *d_img, const float *d_sino, const float *d_weights,
                              double beta, double eps, double *d_out, void *stream)
{
    if (!P) return mvct_fail(MVCT_EINVAL, "mvct_objective: null plan");
    int rc = mvct_check_ptrs(P->device, stream, "mvct_objective", {d_img, d_sino, d_weights, d_out});
    if (rc) return rc;
    if (!mvct_eps_ok(eps) || !std::isfinite(beta))
        return mvct_fail(MVCT_EINVAL, "mvct_objective: invalid beta/eps");
    DeviceGuard dg(P->device);
    cudaStream_t st = (cudaStream_t)stream;
    float *img = pad_row0(P->pad[0], P->geo.n), *imgT = pad_row0(P->pad[2], P->geo.n);
    CK(launch_pad_transpose(d_img, img, imgT, P->geo.n, st));
    CK(launch_residual(P, img, imgT, d_sino, d_weights, P->partials, nullptr, st));
    CK(launch_tv(P, d_img, (float)eps, nullptr, P->partials2, st));
    CK(launch_final_sum(P->partials, P->reduce_grid, 0.5, P->partials2, P->reduce_grid, beta, d_out, st));
    return MVCT_OK;
}

extern "C" int mvct_objective_grad(mvct_plan P, const float *d_img, const float *d_sino, const float *d_weights,
                                   double beta, double eps, float *d_grad, double *d_out_or_null, void *stream)
{
    if (!P) return mvct_fail(MVCT_EINVAL, "mvct_objective_grad: null plan");
    int rc = mvct_check_ptrs(P->device, stream, "mvct_objective_grad", {d_img, d_sino, d_weights, d_grad});
    if (rc == MVCT_OK && d_out_or_null) rc = mvct_check_ptrs(P->device, stream, "mvct_objective_grad", {d_out_or_null});
    if (rc) return rc;
    if (!mvct_eps_ok(eps) || !std::isfinite(beta))
        return mvct_fail(MVCT_EINVAL, "mvct_objective_grad: invalid beta/eps");
    if (d_grad == d_img) return mvct_fail(MVCT_EINVAL, "mvct_objective_grad: d_grad must not alias d_img");
    DeviceGuard dg(P->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = P->geo.n;
    float *img = pad_row0(P->pad[0], n), *imgT = pad_row0(P->pad[2], n);
    float *tvg = pad_row0(P->pad[1], n); // scratch outside mvct_recon
    CK(launch_pad_transpose(d_img, img, imgT, n, st));
    // e = w .* (A img - p) over all views, and sum w r^2 (FP64)
    CK(launch_residual(P, img, imgT, d_sino, d_weights, P->partials, P->sino_tmp, st));
    CK(launch_back(P, P->sino_tmp, d_grad, -1, st));                 // A^T e
    CK(launch_tv(P, d_img, (float)eps, tvg, P->partials2, st));      // grad TV_eps
    CK(launch_axpy(P, d_grad, tvg, (float)beta, (size_t)n * n, st));
    if (d_out_or_null)
        CK(launch_final_sum(P->partials, P->reduce_grid, 0.5, P->partials2, P->reduce_grid, beta, d_out_or_null,
                            st));
    return MVCT_OK;
}

extern "C" int mvct_phase_b_plan(int32_t n_tiles, int32_t views_per_subset, int32_t groups_cap, int32_t grid,
                                 int32_t num_sms, int32_t *items, int32_t *idle_block)
{
    if (!items || !idle_block) return mvct_fail(MVCT_EINVAL, "mvct_phase_b_plan: null output");
    if (n_tiles < 1 || views_per_subset < 1 || groups_cap < 1 || grid < 1 || num_sms < 1)
        return mvct_fail(MVCT_EINVAL, "mvct_phase_b_plan: sizes must be >= 1");
    std::vector<int4> plan;
    int idle = -1;
    if (!balanced_items(n_tiles, views_per_subset, groups_cap, grid, num_sms, plan, idle)) return 0;
    for (int b = 0; b < grid; ++b) {
        items[4 * b + 0] = plan[b].x;
        items[4 * b + 1] = plan[b].y;
        items[4 * b + 2] = plan[b].z;
        items[4 * b + 3] = plan[b].w;
    }
    *idle_block = idle;
    return 1;
}
