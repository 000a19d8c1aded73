// sky_noalloc.cu -- sky_skyline_noalloc: the skyline of a small point set
// without any device or host memory allocation.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they need a skyline: for example a host process that has already handed
// all device memory to its own arena allocator, or a latency-critical loop
// in which an allocation's implicit device-wide synchronisation is not
// allowed. For them this entry point runs the same kernels as sky_skyline,
// but takes all of its scratch memory from one fixed-size array in device
// global memory that the library reserves when it is loaded (a file-scope
// static __device__ array). The caller still passes the input points and the
// output buffer.
//
// Limits: n <= SKY_NOALLOC_MAX_POINTS (65,536) points and a grid of at most
// 2^20 cells (log2_g * d <= 20); anything larger is rejected with
// SKY_ERR_TOO_LARGE. The array (12 MiB) stays reserved on every GPU that
// loads the library until the process exits.
//
// Sharing: every call, on every stream and thread, uses the same array, and
// it keeps the previous call's contents. The kernels clear what must start at
// zero at the start of each call. Calls that overlap on the GPU (two streams,
// or two host threads on one device) race on the array and give wrong results:
// serialise them.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress while that device is current (host code cannot use
// the array's name as a device address). That first call should come before
// any stream capture is started on the device.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/sky.h"
#include "sky_common.cuh"
#include "sky_internal.h"

using namespace sky;

namespace {

constexpr int64_t kMaxPoints = SKY_NOALLOC_MAX_POINTS;
constexpr int kMaxGridBits = 20;
constexpr size_t kScratchBytes = size_t(12) << 20;  // 12 MiB; the worst case (65,536 x 16 at 2^16 cells) needs less

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};

thread_local char t_msg[256];

// The message goes to both sky_noalloc_last_error() and sky_last_error().
sky_status noalloc_fail(sky_status s, const char* msg)
{
    snprintf(t_msg, sizeof(t_msg), "%s", msg);
    sky::set_last_error(msg);
    return s;
}

// Device address of the scratch array on the current device (looked up once).
sky_status scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(SKY_ERR_NO_DEVICE, "no CUDA device");
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(SKY_ERR_NO_DEVICE, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return noalloc_fail(SKY_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed");
        g_scratch_dev[dev] = ptr;
    }
    *out = g_scratch_dev[dev];
    return SKY_OK;
}

}  // namespace

extern "C" SKY_API const char* sky_noalloc_last_error(void) { return t_msg; }

extern "C" sky_status sky_skyline_noalloc(const float* d_pts, int64_t n, int32_t d, int64_t ld,
                                          const sky_options* opt, int32_t* d_out_idx, int64_t out_capacity,
                                          int64_t* h_out_count, void* stream)
{
    t_msg[0] = 0;
    sky::set_last_error("");
    if (!h_out_count) return noalloc_fail(SKY_ERR_INVALID_ARGUMENT, "NULL count pointer");
    if (d < 1 || d > kMaxDim) return noalloc_fail(SKY_ERR_INVALID_ARGUMENT, "d outside [1, 16]");
    if (ld < d) return noalloc_fail(SKY_ERR_INVALID_ARGUMENT, "ld < d");
    if (n < 0) return noalloc_fail(SKY_ERR_INVALID_ARGUMENT, "n < 0");
    if (n > kMaxPoints) return noalloc_fail(SKY_ERR_TOO_LARGE, "n above SKY_NOALLOC_MAX_POINTS (65536)");
    if (n > 0 && !d_pts) return noalloc_fail(SKY_ERR_INVALID_ARGUMENT, "NULL points pointer");
    if (reinterpret_cast<uintptr_t>(d_pts) & 3u) return noalloc_fail(SKY_ERR_INVALID_ARGUMENT, "points not 4-byte aligned");
    if (out_capacity < 0 || (out_capacity > 0 && !d_out_idx))
        return noalloc_fail(SKY_ERR_INVALID_ARGUMENT, "bad output buffer");
    if (opt && (opt->n_filter < 0 || opt->n_filter > 16 || (opt->n_filter > 0 && !opt->d_filter_pts)))
        return noalloc_fail(SKY_ERR_INVALID_ARGUMENT, "bad filter proposals");
    // the call reads the count back (one synchronisation): a stream that is
    // being captured cannot run it, and is left untouched
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap) != cudaSuccess ||
        cap != cudaStreamCaptureStatusNone)
        return noalloc_fail(SKY_ERR_INVALID_ARGUMENT, "stream is being captured: the call synchronises its stream "
                                                      "and cannot be recorded in a graph");
    if (n == 0) { *h_out_count = 0; return SKY_OK; }

    Plan p;
    p.pts = d_pts;
    p.n = n;
    p.d = d;
    p.ld = ld;
    const int au = opt ? opt->assume_unit : 0;
    if (au < 0 || au > 2) return noalloc_fail(SKY_ERR_INVALID_ARGUMENT, "assume_unit outside {0, 1, 2}");
    p.map_mode = au == 1 ? kMapUnit : (au == 2 ? kMapMinMax : kMapAuto);
    int lg = (opt && opt->log2_g >= 0) ? opt->log2_g : auto_log2g(n, d);
    while (lg > 0 && lg * d > kMaxGridBits && !(opt && opt->log2_g >= 0)) --lg;
    if (lg * d > kMaxGridBits) return noalloc_fail(SKY_ERR_TOO_LARGE, "grid above 2^20 cells (log2_g * d > 20)");
    p.log2g = lg;
    p.morton_bits = morton_bits_for(n, d);
    p.tma_ok = (ld == d) && ((reinterpret_cast<uintptr_t>(d_pts) & 15u) == 0);
    if (opt && (opt->survivors_only < 0 || opt->survivors_only > 1))
        return noalloc_fail(SKY_ERR_INVALID_ARGUMENT, "survivors_only outside {0, 1}");
    p.survivors_only = opt && opt->survivors_only == 1;
    if (plan_workspace_bytes(n, d, lg, false) > kScratchBytes)
        return noalloc_fail(SKY_ERR_TOO_LARGE, "workspace exceeds the fixed scratch array");

    void* scratch = nullptr;
    sky_status st = scratch_address(&scratch);
    if (st != SKY_OK) return st;
    plan_carve(p, scratch, false);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n_prop = opt ? opt->n_filter : 0;
    cudaError_t e = cudaMemsetAsync(p.res, 0, sizeof(DevResult), s);
    if (e == cudaSuccess) e = launch_build(p, s);
    if (e == cudaSuccess) e = launch_snap(p, n_prop ? opt->d_filter_pts : nullptr, n_prop, s);
    if (e == cudaSuccess) e = launch_prefix_or(p, s);
    if (e == cudaSuccess) e = launch_survivors(p, n_prop, s);
    if (p.survivors_only) {
        if (e == cudaSuccess) e = launch_copy_survivors(p, d_out_idx, out_capacity, s);
    } else {
        if (e == cudaSuccess) e = launch_sort(p, s);
        if (e == cudaSuccess) e = launch_gather(p, s);
        if (e == cudaSuccess) e = launch_refine(p, s);
        if (e == cudaSuccess) e = launch_emit(p, d_out_idx, out_capacity, s);
    }
    DevResult r{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, p.res, sizeof(DevResult), cudaMemcpyDeviceToHost, s);
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e != cudaSuccess || es != cudaSuccess) return noalloc_fail(SKY_ERR_CUDA, "kernel launch or copy failed");
    if (r.err & SKY_DEV_ERR_NONFINITE) return noalloc_fail(SKY_ERR_NONFINITE, "input holds NaN or infinity");
    if (r.err & SKY_DEV_ERR_TIMEOUT) return noalloc_fail(SKY_ERR_TIMEOUT, "a bounded device wait ran out");
    *h_out_count = r.count;
    if ((int64_t)r.count > out_capacity) return noalloc_fail(SKY_ERR_CAPACITY, "output capacity too small");
    return SKY_OK;
}
