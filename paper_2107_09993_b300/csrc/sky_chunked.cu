// sky_chunked.cu -- sky_skyline_chunked: the skyline of a point set that one
// in-core call cannot take, because it has more than 2^31 - 1 rows or because
// it lives in host memory (possibly larger than device memory).
//
// The rows are processed in chunks with the kernels of steps (a)-(c) and a
// single occupancy bitmap for the whole set, so that cell pruning sees every
// row [Eq. 1, Definition 3, Corollary 4]:
//   pass 1  every chunk is mapped and its cells are marked in the bitmap
//   prefix  the prefix-OR of the bitmap (once)
//   pass 2  every chunk is mapped again (keys only); the rows whose cell is
//           not dominated are appended, coordinates and 64-bit row ids, to a
//           candidate buffer
//   refine  one in-core skyline call on the candidates [Definition 1]; its
//           indices are translated back to row ids
// The value map is decided once for the whole set: the automatic rule on
// rows 0, t, 2t, ... (t = ceil(n / 4096)) of all n rows, or the min / max of
// all rows (one more pass), or the unit cube. Host input is copied through a
// double-buffered staging area on a second stream, so the copy of the next
// chunk overlaps the kernels of the current one; both passes read the input
// once each.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sky.h"
#include "sky_common.cuh"
#include "sky_internal.h"

using namespace sky;

namespace {

sky_status cfail(sky_status s, const char* msg, cudaError_t e = cudaSuccess)
{
    char buf[320];
    snprintf(buf, sizeof(buf), "%s%s%s", msg, e != cudaSuccess ? ": " : "",
             e != cudaSuccess ? cudaGetErrorString(e) : "");
    set_last_error(buf);
    return s;
}

constexpr int kT = 256;
constexpr int64_t kSampleRows = 4096;

// rows 0, t, 2t, ... of a device array, packed into `out` (rows x d)
__global__ void k_gather_sample(const float* __restrict__ pts, int64_t n, int d, int64_t ld, float* out)
{
    int64_t t = (n + kSampleRows - 1) / kSampleRows;
    if (t < 1) t = 1;
    const int64_t rows = (n + t - 1) / t;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * d;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / d;
        const int k = (int)(i % d);
        out[i] = pts[r * t * ld + k];
    }
}

// Appends one chunk's survivors (ascending local rows) to the candidates.
// Nothing is written past `cap`; the count still advances (k_advance), so the
// caller learns how many candidates there were.
__global__ void k_append(const float* __restrict__ pts, int64_t ld, int d, const uint32_t* __restrict__ surv_idx,
                         const DevResult* res, int64_t chunk_base, const unsigned long long* count, float* cand_x,
                         int64_t* cand_ids, int64_t cap)
{
    const uint32_t m = res->survivors;
    const unsigned long long base = *count;
    if ((int64_t)(base + m) > cap) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)m * d;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / d;
        const int k = (int)(i % d);
        const int64_t row = surv_idx[j];
        cand_x[(base + j) * d + k] = pts[row * ld + k];
        if (k == 0) cand_ids[base + j] = chunk_base + row;
    }
}

__global__ void k_advance(const DevResult* res, unsigned long long* count)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *count += res->survivors;
}

// out[i] = ids[idx[i]]: skyline indices into the candidates -> row ids
__global__ void k_translate(const int32_t* __restrict__ idx, const int64_t* __restrict__ ids, int64_t count,
                            int64_t* out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = ids[idx[i]];
}

int blocks_for(int64_t work)
{
    int64_t b = (work + kT - 1) / kT;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 148 * 16));
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// The arrays of steps (a)-(c) for chunks of up to `rows` rows, carved from
// one allocation (no refinement arrays: the candidates go to sky_skyline).
size_t carve_chunk_plan(Plan& p, int64_t rows, char* base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* q = base ? base + off : nullptr;
        off += a256(bytes + 16);
        return q;
    };
    const int64_t r = std::max<int64_t>(rows, 1);
    p.words = std::max<int64_t>(1, (1ll << (p.log2g * p.d)) / 32);
    p.params = reinterpret_cast<float*>(take(64 * sizeof(float)));
    p.res = reinterpret_cast<DevResult*>(take(sizeof(DevResult)));
    p.mm_min = reinterpret_cast<uint32_t*>(take(kMaxDim * 4));
    p.mm_max = reinterpret_cast<uint32_t*>(take(kMaxDim * 4));
    p.occ = reinterpret_cast<uint32_t*>(take((size_t)p.words * 4));
    p.pre = reinterpret_cast<uint32_t*>(take((size_t)p.words * 4));
    p.occ_stage = p.words <= kPrivWords ? reinterpret_cast<uint32_t*>(take((size_t)map_blocks_bound(r) * p.words * 4))
                                        : nullptr;
    if (!base && p.words > kPrivWords) p.occ_stage = nullptr;
    p.ckey = reinterpret_cast<uint32_t*>(take((size_t)r * 4));
    p.mkey = reinterpret_cast<uint32_t*>(take((size_t)r * 4));
    p.sflags = reinterpret_cast<uint32_t*>(take((size_t)((r + 31) / 32) * 4));
    p.scount = reinterpret_cast<uint32_t*>(take((size_t)kSurvMaxBlocks * 4));
    p.surv_key = reinterpret_cast<uint32_t*>(take((size_t)r * 4));
    p.surv_idx = reinterpret_cast<uint32_t*>(take((size_t)r * 4));
    p.filt = reinterpret_cast<float*>(take(16 * kMaxDim * sizeof(float)));
    return off;
}

// Device memory released on every exit path.
struct DevBuffers {
    std::vector<void*> ptrs;
    cudaStream_t s = nullptr;
    ~DevBuffers()
    {
        for (void* q : ptrs)
            if (q) cudaFreeAsync(q, s);
    }
    template <class T>
    cudaError_t alloc(T** out, size_t bytes)
    {
        void* q = nullptr;
        const cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(bytes, 256), s);
        if (e == cudaSuccess) ptrs.push_back(q);
        *out = static_cast<T*>(q);
        return e;
    }
};

struct HostStaging {
    float* host = nullptr;          // pinned sample rows
    cudaStream_t copy = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
    ~HostStaging()
    {
        if (copy) cudaStreamSynchronize(copy);
        for (int i = 0; i < 2; ++i) {
            if (copied[i]) cudaEventDestroy(copied[i]);
            if (done[i]) cudaEventDestroy(done[i]);
        }
        if (copy) cudaStreamDestroy(copy);
        if (host) cudaFreeHost(host);
    }
};

}  // namespace

extern "C" {

sky_status sky_skyline_chunked(const float* pts, int32_t host_pts, int64_t n, int32_t d, int64_t ld,
                               const sky_options* opt, int64_t chunk_rows, int64_t max_candidates,
                               int64_t* d_out_ids, int64_t capacity, int64_t* h_count, void* stream)
{
    if (!h_count) return cfail(SKY_ERR_INVALID_ARGUMENT, "h_count is NULL");
    *h_count = 0;
    if (d < 1 || d > kMaxDim) return cfail(SKY_ERR_INVALID_ARGUMENT, "d outside [1, 16]");
    if (n < 0 || n > (int64_t(1) << 40)) return cfail(SKY_ERR_INVALID_ARGUMENT, "n outside [0, 2^40]");
    if (ld < d) return cfail(SKY_ERR_INVALID_ARGUMENT, "ld < d");
    if (n > 0 && !pts) return cfail(SKY_ERR_INVALID_ARGUMENT, "points pointer is NULL");
    if (reinterpret_cast<uintptr_t>(pts) & 3u) return cfail(SKY_ERR_INVALID_ARGUMENT, "points not 4-byte aligned");
    if (host_pts != 0 && host_pts != 1) return cfail(SKY_ERR_INVALID_ARGUMENT, "host_pts outside {0, 1}");
    if (chunk_rows < 0 || chunk_rows > (int64_t(1) << 30)) return cfail(SKY_ERR_INVALID_ARGUMENT, "chunk_rows outside [0, 2^30]");
    if (max_candidates < 0 || max_candidates > 0x7fffffffll)
        return cfail(SKY_ERR_INVALID_ARGUMENT, "max_candidates outside [0, 2^31 - 1]");
    if (capacity < 0 || (capacity > 0 && !d_out_ids)) return cfail(SKY_ERR_INVALID_ARGUMENT, "bad output buffer");
    if (opt && opt->n_filter != 0) return cfail(SKY_ERR_INVALID_ARGUMENT, "filter proposals are not supported here");
    const int au = opt ? opt->assume_unit : 0;
    if (au < 0 || au > 2) return cfail(SKY_ERR_INVALID_ARGUMENT, "assume_unit outside {0, 1, 2}");
    const bool surv_only = opt && opt->survivors_only == 1;
    if (n == 0) return SKY_OK;

    Plan p;
    p.d = d;
    p.map_mode = au == 1 ? kMapUnit : (au == 2 ? kMapMinMax : kMapAuto);
    p.log2g = (opt && opt->log2_g >= 0) ? opt->log2_g : auto_log2g(n, d);
    if (opt && opt->log2_g > 16) return cfail(SKY_ERR_TOO_LARGE, "log2_g above 16");
    if (p.log2g * d > 27) return cfail(SKY_ERR_TOO_LARGE, "grid above the dense limit 2^27");
    const int64_t crows = std::min<int64_t>(n, chunk_rows > 0 ? chunk_rows : (host_pts ? (1ll << 26) : (1ll << 28)));
    p.morton_bits = morton_bits_for(crows, d);
    const int64_t cand_cap = max_candidates > 0 ? max_candidates : std::min<int64_t>(n, 1ll << 28);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuffers buf;
    buf.s = s;
    char* ws = nullptr;
    cudaError_t e = buf.alloc(&ws, carve_chunk_plan(p, crows, nullptr));
    if (e != cudaSuccess) return cfail(SKY_ERR_OUT_OF_MEMORY, "chunk workspace", e);
    carve_chunk_plan(p, crows, ws);
    float* stage[2] = {nullptr, nullptr};
    float* sample = nullptr;
    float* cand_x = nullptr;
    int64_t* cand_ids = nullptr;
    unsigned long long* cand_count = nullptr;
    if (host_pts) {
        for (int i = 0; i < 2; ++i)
            if ((e = buf.alloc(&stage[i], (size_t)crows * d * sizeof(float))) != cudaSuccess)
                return cfail(SKY_ERR_OUT_OF_MEMORY, "staging buffers", e);
    }
    if ((e = buf.alloc(&sample, (size_t)kSampleRows * d * sizeof(float))) != cudaSuccess ||
        (e = buf.alloc(&cand_x, (size_t)cand_cap * d * sizeof(float))) != cudaSuccess ||
        (e = buf.alloc(&cand_ids, (size_t)cand_cap * sizeof(int64_t))) != cudaSuccess ||
        (e = buf.alloc(&cand_count, sizeof(unsigned long long))) != cudaSuccess)
        return cfail(SKY_ERR_OUT_OF_MEMORY, "candidate buffers", e);
    cudaMemsetAsync(p.res, 0, sizeof(DevResult), s);
    cudaMemsetAsync(p.occ, 0, sizeof(uint32_t) * p.words, s);
    cudaMemsetAsync(cand_count, 0, sizeof(unsigned long long), s);

    HostStaging hs;
    if (host_pts) {
        if ((e = cudaStreamCreateWithFlags(&hs.copy, cudaStreamNonBlocking)) != cudaSuccess)
            return cfail(SKY_ERR_CUDA, "copy stream", e);
        for (int i = 0; i < 2; ++i) {
            if ((e = cudaEventCreateWithFlags(&hs.copied[i], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&hs.done[i], cudaEventDisableTiming)) != cudaSuccess)
                return cfail(SKY_ERR_CUDA, "events", e);
            cudaEventRecord(hs.done[i], s);
        }
    }
    const int64_t nchunks = (n + crows - 1) / crows;

    // Makes chunk c's rows visible on `s`: a pointer into device input, or the
    // staging buffer its copy went to (the copy waits until the kernels that
    // read that buffer two chunks ago are done).
    auto chunk = [&](int64_t c, Plan& q) -> cudaError_t {
        const int64_t r0 = c * crows;
        const int64_t rows = std::min<int64_t>(crows, n - r0);
        q = p;
        q.n = rows;
        if (!host_pts) {
            q.pts = pts + r0 * ld;
            q.ld = ld;
        } else {
            const int b = (int)(c & 1);
            cudaError_t ee = cudaStreamWaitEvent(hs.copy, hs.done[b], 0);
            if (ee == cudaSuccess) {
                if (ld == d)
                    ee = cudaMemcpyAsync(stage[b], pts + r0 * ld, (size_t)rows * d * sizeof(float),
                                         cudaMemcpyHostToDevice, hs.copy);
                else
                    ee = cudaMemcpy2DAsync(stage[b], (size_t)d * sizeof(float), pts + r0 * ld, (size_t)ld * sizeof(float),
                                           (size_t)d * sizeof(float), (size_t)rows, cudaMemcpyHostToDevice, hs.copy);
            }
            if (ee == cudaSuccess) ee = cudaEventRecord(hs.copied[b], hs.copy);
            if (ee == cudaSuccess) ee = cudaStreamWaitEvent(s, hs.copied[b], 0);
            if (ee != cudaSuccess) return ee;
            q.pts = stage[b];
            q.ld = d;
        }
        q.tma_ok = (q.ld == d) && ((reinterpret_cast<uintptr_t>(q.pts) & 15u) == 0);
        return cudaSuccess;
    };
    auto chunk_done = [&](int64_t c) {
        if (host_pts) cudaEventRecord(hs.done[c & 1], s);
    };

    // ---- value map
    if (p.map_mode == kMapMinMax) {
        launch_mm_reset(p, s);
        for (int64_t c = 0; c < nchunks; ++c) {
            Plan q;
            if ((e = chunk(c, q)) != cudaSuccess) return cfail(SKY_ERR_CUDA, "chunk copy", e);
            launch_minmax_accumulate(q, s);
            chunk_done(c);
        }
        launch_params(p, s);
    } else if (p.map_mode == kMapUnit) {
        launch_params(p, s);
    } else {
        int64_t t = (n + kSampleRows - 1) / kSampleRows;
        const int64_t rows = (n + t - 1) / t;
        if (!host_pts) {
            k_gather_sample<<<blocks_for(rows * d), kT, 0, s>>>(pts, n, d, ld, sample);
        } else {
            if ((e = cudaMallocHost(&hs.host, (size_t)rows * d * sizeof(float))) != cudaSuccess)
                return cfail(SKY_ERR_OUT_OF_MEMORY, "pinned sample", e);
            for (int64_t r = 0; r < rows; ++r) memcpy(hs.host + r * d, pts + r * t * ld, (size_t)d * sizeof(float));
            cudaMemcpyAsync(sample, hs.host, (size_t)rows * d * sizeof(float), cudaMemcpyHostToDevice, s);
        }
        Plan q = p;
        q.pts = sample;
        q.n = rows;
        q.ld = d;
        launch_params(q, s);   // rows 0, t, 2t, ... of the whole set: the automatic rule
    }

    // ---- pass 1: mark every chunk's cells
    for (int64_t c = 0; c < nchunks; ++c) {
        Plan q;
        if ((e = chunk(c, q)) != cudaSuccess) return cfail(SKY_ERR_CUDA, "chunk copy", e);
        q.ckey = q.mkey = nullptr;   // this pass only marks: no keys are written
        if ((e = launch_map_pass(q, true, s)) != cudaSuccess) return cfail(SKY_ERR_CUDA, "map pass", e);
        chunk_done(c);
    }
    if ((e = launch_prefix_or(p, s)) != cudaSuccess) return cfail(SKY_ERR_CUDA, "prefix-OR", e);

    // ---- pass 2: keys again, survivors appended as candidates
    for (int64_t c = 0; c < nchunks; ++c) {
        Plan q;
        if ((e = chunk(c, q)) != cudaSuccess) return cfail(SKY_ERR_CUDA, "chunk copy", e);
        launch_map_pass(q, false, s);
        launch_survivors(q, 0, s);
        k_append<<<blocks_for(q.n * d), kT, 0, s>>>(q.pts, q.ld, d, q.surv_idx, q.res, c * crows, cand_count, cand_x,
                                                     cand_ids, cand_cap);
        k_advance<<<1, 32, 0, s>>>(q.res, cand_count);
        chunk_done(c);
        if ((e = cudaGetLastError()) != cudaSuccess) return cfail(SKY_ERR_CUDA, "survivor pass", e);
    }
    unsigned long long m = 0;
    uint32_t err = 0;
    if ((e = cudaMemcpyAsync(&m, cand_count, sizeof(m), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&err, &p.res->err, sizeof(err), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cfail(SKY_ERR_CUDA, "candidate count", e);
    if (err & SKY_DEV_ERR_NONFINITE) return cfail(SKY_ERR_NONFINITE, "input holds NaN or infinity");
    if (err & SKY_DEV_ERR_TIMEOUT) return cfail(SKY_ERR_TIMEOUT, "a bounded device wait ran out");
    if ((int64_t)m > cand_cap) {
        char msg[128];
        snprintf(msg, sizeof(msg), "%llu candidates after step (c), max_candidates %lld", m, (long long)cand_cap);
        return cfail(SKY_ERR_CAPACITY, msg);
    }

    // ---- refinement of the candidates (or the candidates themselves)
    if (surv_only) {
        *h_count = (int64_t)m;
        if ((int64_t)m > capacity) return cfail(SKY_ERR_CAPACITY, "output capacity below the candidate count");
        if (m) cudaMemcpyAsync(d_out_ids, cand_ids, (size_t)m * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
        e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? SKY_OK : cfail(SKY_ERR_CUDA, "copy out", e);
    }
    if (m == 0) return SKY_OK;
    int32_t* idx = nullptr;
    if ((e = buf.alloc(&idx, (size_t)m * sizeof(int32_t))) != cudaSuccess)
        return cfail(SKY_ERR_OUT_OF_MEMORY, "refinement output", e);
    sky_options o{};
    o.log2_g = -1;
    o.assume_unit = 0;
    int64_t cnt = 0;
    sky_status st = sky_skyline(cand_x, (int64_t)m, d, d, &o, idx, (int64_t)m, &cnt, stream);
    if (st != SKY_OK) {
        const std::string inner = sky_last_error();
        return cfail(st, inner.c_str());
    }
    *h_count = cnt;
    if (cnt > capacity) return cfail(SKY_ERR_CAPACITY, "output capacity below the skyline size");
    if (cnt) k_translate<<<blocks_for(cnt), kT, 0, s>>>(idx, cand_ids, cnt, d_out_ids);
    e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? SKY_OK : cfail(SKY_ERR_CUDA, "translate", e);
}

}  // extern "C"
