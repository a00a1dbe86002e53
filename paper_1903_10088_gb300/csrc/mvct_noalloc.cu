// mvct_tv_grad_noalloc: the TV gradient and value without a plan and without any
// device allocation.
//
// Who needs it: callers that may not allocate device memory -- applications
// whose GPU memory is handed out up front by their own allocator (nothing else
// may call cudaMalloc), and latency-critical paths where cudaMalloc/cudaFree are
// off limits because they can synchronise the device and stall other streams.
//
// The only scratch the TV reduction needs -- one FP64 partial sum per block --
// lives in the file-scope array below, in the library's static device memory.
// Every GPU that loads the library holds these 16 KiB until the process exits.
#include <cmath>
#include <mutex>

#include "mvct_plan.h"

namespace {

static __device__ __align__(256) double g_tv_partials[MVCT_NOALLOC_MAX_BLOCKS];

constexpr int kMaxDevices = 64;

struct DeviceScratch {
    double *partials = nullptr; // device address of g_tv_partials on this device
    int blocks = 0;             // grid used by the reduction on this device
};

std::mutex g_mutex;
DeviceScratch g_scratch[kMaxDevices];

// Once per device, with that device current: look up the device address of the
// static array (host code may not use the symbol itself: on the host it names a
// shadow variable, not device memory).
int device_scratch(int dev, DeviceScratch *out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceScratch &d = g_scratch[dev];
    if (!d.partials) {
        double *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_tv_partials);
        if (e != cudaSuccess)
            return mvct_fail(MVCT_ECUDA, "mvct_tv_grad_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return mvct_fail(MVCT_ECUDA, "mvct_tv_grad_noalloc: %s", cudaGetErrorString(e));
        d.blocks = sms * 8 < MVCT_NOALLOC_MAX_BLOCKS ? sms * 8 : MVCT_NOALLOC_MAX_BLOCKS;
        d.partials = ptr;
    }
    *out = d;
    return MVCT_OK;
}

} // namespace

extern "C" int mvct_tv_grad_noalloc(const float *d_img, int32_t n, double eps, float *d_grad,
                                    double *d_tv_or_null, void *stream)
{
    if (!d_img || !d_grad) return mvct_fail(MVCT_EINVAL, "mvct_tv_grad_noalloc: null device pointer");
    if (n < 1 || n > MVCT_MAX_N)
        return mvct_fail(MVCT_EINVAL, "mvct_tv_grad_noalloc: n = %d outside 1..%d (the static scratch "
                         "serves images up to %d x %d)", n, MVCT_MAX_N, MVCT_MAX_N, MVCT_MAX_N);
    if (!mvct_eps_ok(eps))
        return mvct_fail(MVCT_EINVAL, "mvct_tv_grad_noalloc: eps must be > 0 and a normal float (>= FLT_MIN)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mvct_fail(MVCT_ECUDA, "mvct_tv_grad_noalloc: %s", cudaGetErrorString(e));
    {
        int rc = mvct_check_ptrs(dev, stream, "mvct_tv_grad_noalloc", {d_img, d_grad});
        if (rc == MVCT_OK && d_tv_or_null) rc = mvct_check_ptrs(dev, stream, "mvct_tv_grad_noalloc", {d_tv_or_null});
        if (rc) return rc;
    }
    if (dev < 0 || dev >= kMaxDevices)
        return mvct_fail(MVCT_EINVAL, "mvct_tv_grad_noalloc: device ordinal %d >= %d", dev, kMaxDevices);
    DeviceScratch s;
    int rc = device_scratch(dev, &s);
    if (rc) return rc;
    const long long want = ((long long)n * n + mvct::kThreads - 1) / mvct::kThreads;
    const int grid = (int)(want < s.blocks ? want : s.blocks);
    cudaStream_t st = (cudaStream_t)stream;
    // Every block writes its own partial before the final sum reads exactly
    // `grid` of them, so no slot has to be cleared between calls.
    e = mvct::launch_tv_grid(n, d_img, (float)eps, d_grad, s.partials, grid, st);
    if (e == cudaSuccess && d_tv_or_null)
        e = mvct::launch_final_sum(s.partials, grid, 1.0, nullptr, 0, 0.0, d_tv_or_null, st);
    if (e != cudaSuccess) return mvct_fail(MVCT_ECUDA, "mvct_tv_grad_noalloc: launch: %s", cudaGetErrorString(e));
    return MVCT_OK;
}
