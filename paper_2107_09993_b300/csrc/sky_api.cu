// sky_api.cu -- the C ABI of libsky (include/sky.h): argument checks, workspace
// layout, and the order in which the kernels of steps (a)-(d) are enqueued.
#include <algorithm>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "../../include/sky.h"
#include "sky_common.cuh"
#include "sky_internal.h"

using namespace sky;

namespace {

constexpr int kTournamentMaxBits = 27;   // layers of up to 2^27 cells (the dense limit)
// Grids above kPrivWords words with at least half as many rows as cells are
// marked in a byte-per-cell map (plain byte stores, packed into the bitmap
// afterwards) instead of by global atomicOr on the bitmap, in the single-set
// path (sky_skyline, the sets calls, the witness mode); the grid API, the
// chunked path and the no-allocation entry point keep the atomic marking.
// Measured on B300: 10^7 x 12 independent (2^24 cells) pruning call 226 ->
// 216 us; at 10^6 rows on 2^24 cells the byte map lost 15-50 us.
#ifndef SKY_BYTEMAP_MARKING
#define SKY_BYTEMAP_MARKING 1
#endif
constexpr bool kByteMapMarking = SKY_BYTEMAP_MARKING != 0;
thread_local std::string t_err;
thread_local sky_run_stats t_stats = {};
thread_local sky_phase_times t_phase = {};
// 0: off; 1: events between the phases (direct launches, no graph);
// 2: events around the whole kernel sequence of the call (graph replay kept)
thread_local int t_timing = 0;
thread_local cudaEvent_t t_ev[9] = {};

// Optional per-phase events on the call's stream.
struct PhaseClock {
    cudaStream_t s;
    bool on;
    int next = 0;
    explicit PhaseClock(cudaStream_t st, bool allow = true) : s(st), on(allow && t_timing == 1)
    {
        if (!on) return;
        for (auto& e : t_ev)
            if (!e && cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
        mark();
    }
    void mark()
    {
        if (on && next < 9) cudaEventRecord(t_ev[next++], s);
    }
    void collect()
    {
        if (!on) return;
        float ms[8] = {};
        for (int i = 0; i + 1 < next; ++i)
            if (cudaEventElapsedTime(&ms[i], t_ev[i], t_ev[i + 1]) != cudaSuccess) ms[i] = 0.0f;
        cudaGetLastError();   // leave no error behind for the caller
        t_phase = {ms[0], ms[1], ms[2], ms[3], ms[4], ms[5], ms[6], ms[7], 0.0f};
    }
};

// Whole-call timing (mode 2): two events per thread and a bounded delay
// kernel (it sleeps until the global timer has advanced by `ns`).
thread_local cudaEvent_t t_span[2] = {};
constexpr uint32_t kSpanDelayNs = 50000;

bool span_events()
{
    for (auto& e : t_span)
        if (!e && cudaEventCreate(&e) != cudaSuccess) return false;
    return true;
}

__global__ void k_delay(uint32_t ns)
{
    uint64_t t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    do {
        __nanosleep(1000);
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    } while (t - t0 < ns);
}

int count_kernels(const Plan& p, int n_prop, int64_t capacity)
{
    const int passes = (p.morton_bits * p.d + 7) / 8;
    const int through_c =
        build_kernel_count(p) + (n_prop > 0 ? 2 : 0) + (prefix_trivial(p) ? 0 : prefix_kernel_count(p)) + 2;
    if (p.survivors_only) return through_c + (capacity >= p.n ? 0 : 1);   // + the id copy
    return through_c + 3 * passes + 1 + 3 + 1 +   // sort, gather, cost + order + refine, emit
           (refine_prepass(p) ? 3 : 0);          // the refinement's pre-pass, compaction, second gather
}

sky_status fail(sky_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
sky_status fail(sky_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

sky_status cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(SKY_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
        return fail(SKY_ERR_NO_DEVICE, "%s: %s", what, cudaGetErrorString(e));
    return fail(SKY_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SKY_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Carver {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t count)
    {
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += align256(count * sizeof(T) + 16);
        return p;
    }
};

// One layout function serves both sizing (base == nullptr) and carving.
size_t layout(Plan& p, char* base, bool grid_api)
{
    Carver c{base};
    const int64_t n = p.n > 0 ? p.n : 1;
    const int dp = pad4(p.d);
    const int64_t n_pad = ((n + kRefineTile - 1) / kRefineTile) * kRefineTile;
    const int64_t tiles = n_pad / kRefineTile;
    p.words = std::max<int64_t>(1, (1ll << (p.log2g * p.d)) / 32);
    p.lb_tiles = (n + kScanTile - 1) / kScanTile;
    p.sort_blocks = (n + kSortTile - 1) / kSortTile;
    p.mm_min = c.take<uint32_t>(kMaxDim);
    p.mm_max = c.take<uint32_t>(kMaxDim);
    p.params = c.take<float>(64);
    p.res = c.take<DevResult>(1);
    p.filt = c.take<float>(16 * kMaxDim);
    p.snap = c.take<unsigned long long>(16);
    p.lb_counter = c.take<uint32_t>(4);
    p.lb_states = c.take<unsigned long long>(p.lb_tiles);
    p.occ = c.take<uint32_t>(p.words);
    p.occ_stage = p.words <= kPrivWords ? c.take<uint32_t>((size_t)map_blocks_bound(n) * p.words) : nullptr;
    // the byte map pays when the rows at least half fill the grid (clearing
    // and packing 2^(log2g d) bytes then costs less than the atomics saved)
    p.occb = (p.bytemap && p.words > kPrivWords && n >= p.words * 16) ? c.take<uint8_t>((size_t)p.words * 32)
                                                                       : nullptr;
    p.pre = c.take<uint32_t>(p.words);
    p.dom = grid_api ? c.take<uint32_t>(p.words) : nullptr;
    p.ckey = c.take<uint32_t>(n);
    p.mkey = c.take<uint32_t>(n);
    p.sflags = c.take<uint32_t>((n + 31) / 32);
    p.scount = c.take<uint32_t>(kSurvMaxBlocks);
    p.surv_key = c.take<uint32_t>(n);
    p.surv_idx = c.take<uint32_t>(n);
    p.sort_key2 = c.take<uint32_t>(n);
    p.sort_val2 = c.take<uint32_t>(n);
    p.hist = c.take<uint32_t>(256 * p.sort_blocks);
    p.digit_total = c.take<uint32_t>(4 * 256);
    p.X = c.take<float>(n_pad * dp);
    p.C = c.take<uint32_t>(n_pad * (dp / 4));
    p.ids = c.take<int32_t>(n_pad);
    p.tmax = c.take<uint32_t>(tiles * (dp / 4));
    p.tile_cost = c.take<uint32_t>(tiles);
    p.tile_order = c.take<uint32_t>(tiles + kSplitExtra);
    p.tile_part = c.take<uint32_t>(tiles + kSplitExtra);
    p.split_state = c.take<uint32_t>(size_t(kSplitSlots) * 5 + 1);
    p.subcode = c.take<uint32_t>(tiles * 5 * (dp / 4));
    p.tile_end = c.take<uint32_t>(tiles);
    p.supmin = c.take<uint32_t>(((tiles + 31) / 32) * (dp / 4));
    p.cidx = c.take<uint32_t>(size_t(2) << (p.d > 0 ? p.d : 1));
    p.tend_pre = c.take<uint32_t>(tiles);
    p.tmask = refine_mask_probe(p.d) ? c.take<uint32_t>(tiles * kMaskWords) : nullptr;
    p.pre_states = c.take<unsigned long long>(p.lb_tiles);
    p.keep = c.take<uint8_t>(n + 16);
    return c.off;
}

void enable_pool_cache()
{
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

sky_status check_points(const float* pts, int64_t n, int32_t d, int64_t ld)
{
    if (d < 1 || d > kMaxDim) return fail(SKY_ERR_INVALID_ARGUMENT, "d = %d outside [1, 16]", d);
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(SKY_ERR_INVALID_ARGUMENT, "n = %lld outside [0, 2^31)", (long long)n);
    if (ld < d) return fail(SKY_ERR_INVALID_ARGUMENT, "ld = %lld < d = %d", (long long)ld, d);
    if (n > 0 && !pts) return fail(SKY_ERR_INVALID_ARGUMENT, "points pointer is NULL");
    if (reinterpret_cast<uintptr_t>(pts) & 3u) return fail(SKY_ERR_INVALID_ARGUMENT, "points pointer not 4-byte aligned");
    return SKY_OK;
}

sky_status make_plan(Plan& p, const float* pts, int64_t n, int32_t d, int64_t ld, const sky_options* opt)
{
    p.pts = pts;
    p.n = n;
    p.d = d;
    p.ld = ld;
    const int au = opt ? opt->assume_unit : 0;
    if (au < 0 || au > 2) return fail(SKY_ERR_INVALID_ARGUMENT, "assume_unit = %d outside {0, 1, 2}", au);
    p.map_mode = au == 1 ? kMapUnit : (au == 2 ? kMapMinMax : kMapAuto);
    int lg = (opt && opt->log2_g >= 0) ? opt->log2_g : auto_log2g(n, d);
    if (opt && opt->log2_g > 16) return fail(SKY_ERR_TOO_LARGE, "log2_g = %d above 16", opt->log2_g);
    if (lg * d > 27) return fail(SKY_ERR_TOO_LARGE, "grid of 2^%d cells exceeds the dense limit 2^27", lg * d);
    p.log2g = lg;
    p.morton_bits = morton_bits_for(n, d);
    p.tma_ok = (ld == d) && ((reinterpret_cast<uintptr_t>(pts) & 15u) == 0);
    if (opt && (opt->survivors_only < 0 || opt->survivors_only > 1))
        return fail(SKY_ERR_INVALID_ARGUMENT, "survivors_only = %d outside {0, 1}", opt->survivors_only);
    p.survivors_only = opt && opt->survivors_only == 1;
    if (opt && (opt->n_filter < 0 || opt->n_filter > 16))
        return fail(SKY_ERR_INVALID_ARGUMENT, "n_filter = %d outside [0, 16]", opt->n_filter);
    if (opt && opt->n_filter > 0 && !opt->d_filter_pts)
        return fail(SKY_ERR_INVALID_ARGUMENT, "n_filter > 0 with a NULL proposal pointer");
    return SKY_OK;
}

// Steps (a)+(b): normalisation (optional), parameters, map + mark.
sky_status run_build(Plan& p, cudaStream_t s)
{
    SKY_CUDA(cudaMemsetAsync(p.res, 0, sizeof(DevResult), s));
    SKY_CUDA(launch_build(p, s));
    return SKY_OK;
}

// Step (c) (+ the optional proposal filter).
sky_status run_prune(Plan& p, const float* prop, int n_prop, cudaStream_t s, bool grid_api)
{
    SKY_CUDA(launch_snap(p, prop, n_prop, s));
    SKY_CUDA(launch_prefix_or(p, s));
    if (grid_api) {
        SKY_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(p.res) + offsetof(DevResult, occupied_cells), 0,
                                 2 * sizeof(uint32_t), s));
        SKY_CUDA(launch_dominated(p, s));
    }
    SKY_CUDA(launch_survivors(p, n_prop, s));
    return SKY_OK;
}

sky_status status_from_flags(uint32_t err)
{
    if (err & SKY_DEV_ERR_NONFINITE) return fail(SKY_ERR_NONFINITE, "input holds NaN or infinity");
    if (err & SKY_DEV_ERR_TIMEOUT) return fail(SKY_ERR_TIMEOUT, "a bounded device wait ran out");
    if (err & SKY_DEV_ERR_LAYOUT) return fail(SKY_ERR_CUDA, "refinement shared memory not 256-byte aligned");
    return SKY_OK;
}

DevResult* host_result()
{
    thread_local DevResult* h = nullptr;
    if (!h) {
        if (cudaMallocHost(&h, sizeof(DevResult)) != cudaSuccess) h = nullptr;
    }
    return h;
}

// Enqueues steps (a)-(d) on `s` (directly, or into a graph under capture).
// Witness mode (p.witness set; never captured): `wit_rep` is the cell scratch
// of launch_witness_cells, run after the survivor pass.
cudaError_t enqueue_pipeline(Plan& p, const float* prop, int n_prop, int32_t* out, int64_t capacity,
                             cudaStream_t s, PhaseClock& clk, int32_t* wit_rep = nullptr)
{
    cudaError_t e = launch_build_params(p, s);   // clears the result block first
    clk.mark();
    if (e == cudaSuccess) e = launch_map_pass(p, true, s);
    clk.mark();
    // without proposals the snap is skipped: n_filter_used stays 0 from the
    // cleared result block, and the survivor pass then reads no filter
    if (e == cudaSuccess && n_prop > 0) e = launch_snap(p, prop, n_prop, s);
    if (prefix_trivial(p)) p.pre = p.occ;   // the survivor pass reads the bitmap itself
    else if (e == cudaSuccess) e = launch_prefix_or(p, s);
    clk.mark();
    // a survivors-only call whose buffer holds n ids receives them directly
    const bool direct = p.survivors_only && capacity >= p.n;
    if (e == cudaSuccess) e = launch_survivors(p, n_prop, s, direct ? reinterpret_cast<uint32_t*>(out) : nullptr);
    if (e == cudaSuccess && p.witness) e = launch_witness_cells(p, wit_rep, n_prop, s);
    clk.mark();
    if (p.survivors_only) {
        if (e == cudaSuccess && !direct) e = launch_copy_survivors(p, out, capacity, s);
        clk.mark();
        return e;
    }
    if (e == cudaSuccess) e = launch_sort(p, s);
    clk.mark();
    if (e == cudaSuccess) e = launch_gather(p, s);
    clk.mark();
    if (e == cudaSuccess) e = launch_refine(p, s);
    clk.mark();
    if (e == cudaSuccess) e = launch_emit(p, out, capacity, s);
    clk.mark();
    return e;
}

// Per-thread cache of workspaces and CUDA graphs. A call whose arguments
// (device, buffers, sizes, options) repeat a recent call reuses that call's
// workspace; from the second repeat on, the whole kernel sequence is replayed
// as one CUDA graph instead of ~30 separate launches. Every replay runs every
// kernel on the current contents of the buffers.
struct CacheKey {
    int dev = -1;
    const float* pts = nullptr;
    int64_t n = 0, ld = 0, cap = 0;
    int d = 0, log2g = 0, mode = 0, n_prop = 0, timing = 0, surv_only = 0;
    const float* prop = nullptr;
    int32_t* out = nullptr;
    bool operator==(const CacheKey& o) const
    {
        return dev == o.dev && pts == o.pts && n == o.n && ld == o.ld && cap == o.cap && d == o.d &&
               log2g == o.log2g && mode == o.mode && n_prop == o.n_prop && timing == o.timing &&
               surv_only == o.surv_only &&
               prop == o.prop && out == o.out;
    }
};

struct CacheEntry {
    CacheKey key;
    bool used = false;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    cudaGraphExec_t exec = nullptr;
    int calls = 0;
    uint64_t tick = 0;
};

constexpr int kCacheSlots = 8;
thread_local CacheEntry t_cache[kCacheSlots];
thread_local uint64_t t_tick = 0;
thread_local cudaStream_t t_stream = nullptr;   // library-internal stream of this thread
thread_local cudaEvent_t t_join = nullptr;
thread_local int t_stream_dev = -1;

CacheEntry* cache_lookup(const CacheKey& k, size_t bytes, cudaStream_t s, sky_status* st)
{
    CacheEntry* lru = &t_cache[0];
    for (auto& e : t_cache) {
        if (e.used && e.key == k) {
            e.tick = ++t_tick;
            return &e;
        }
        if (!e.used || e.tick < lru->tick) lru = &e;
    }
    if (lru->used) {
        if (lru->exec) cudaGraphExecDestroy(lru->exec);
        if (lru->ws) cudaFree(lru->ws);
        *lru = CacheEntry{};
    }
    void* ws = nullptr;
    const cudaError_t e = cudaMallocAsync(&ws, bytes, s);
    if (e != cudaSuccess) {
        *st = cuda_fail(e, "cudaMallocAsync(workspace)");
        return nullptr;
    }
    lru->key = k;
    lru->used = true;
    lru->ws = ws;
    lru->ws_bytes = bytes;
    lru->tick = ++t_tick;
    return lru;
}

// One call between its enqueue and the read of its result block.
struct Inflight {
    Plan p;
    int64_t capacity = 0;
    int n_prop = 0;
    DevResult* h = nullptr;   // page-locked copy of the result block (NULL: `local`)
    DevResult local{};
    bool span = false;
    bool empty = false;       // n == 0: nothing enqueued
};

// Enqueues steps (a)-(d) of one point set on `s` and the copy of its result
// block to the host; returns without waiting. From the second repeat of the
// same arguments the kernel sequence is one CUDA-graph replay.
sky_status skyline_enqueue(const float* pts, int64_t n, int32_t d, int64_t ld, const sky_options* opt,
                           int32_t* out, int64_t capacity, cudaStream_t s, DevResult* hres, int timing,
                           PhaseClock& clk, Inflight& f)
{
    Plan& p = f.p;
    sky_status st = make_plan(p, pts, n, d, ld, opt);
    if (st != SKY_OK) return st;
    f.capacity = capacity;
    f.h = hres;
    if (n == 0) {
        f.empty = true;
        return SKY_OK;
    }
    enable_pool_cache();
    int dev = 0;
    SKY_CUDA(cudaGetDevice(&dev));
    const int n_prop = opt ? opt->n_filter : 0;
    const float* prop = n_prop ? opt->d_filter_pts : nullptr;
    f.n_prop = n_prop;
    p.bytemap = kByteMapMarking;
    CacheKey key;
    key.dev = dev; key.pts = pts; key.n = n; key.ld = ld; key.cap = capacity; key.d = d;
    key.log2g = p.log2g; key.mode = p.map_mode; key.n_prop = n_prop; key.timing = timing == 1 ? 1 : 0;
    key.surv_only = p.survivors_only ? 1 : 0;
    key.prop = prop; key.out = out;
    const size_t bytes = layout(p, nullptr, false);
    CacheEntry* ce = cache_lookup(key, bytes, s, &st);
    if (!ce) return st;
    layout(p, static_cast<char*>(ce->ws), false);
    ++ce->calls;

    cudaError_t e = cudaSuccess;
    // graphs only when no phase events are requested (the events time the
    // direct launches)
    if (ce->calls >= 2 && !ce->exec && timing != 1) {
        // second call with these arguments: capture the sequence once
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            PhaseClock cap_clk(s, false);
            const cudaError_t e1 = enqueue_pipeline(p, prop, n_prop, out, capacity, s, cap_clk);
            const cudaError_t e2 = cudaStreamEndCapture(s, &g);
            if (e1 == cudaSuccess && e2 == cudaSuccess && g) {
                if (cudaGraphInstantiate(&ce->exec, g, 0) != cudaSuccess) ce->exec = nullptr;
            }
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();   // a failed capture falls back to direct launches
        e = cudaSuccess;
    }
    // whole-call timing: a short device-side delay first, so that the host
    // has enqueued the start event and the kernel sequence before the device
    // reaches them; the two events then bracket device work only
    f.span = timing == 2 && span_events();
    if (f.span) {
        k_delay<<<1, 32, 0, s>>>(kSpanDelayNs);
        cudaEventRecord(t_span[0], s);
    }
    if (ce->exec && timing != 1) {
        e = cudaGraphLaunch(ce->exec, s);
    } else {
        e = enqueue_pipeline(p, prop, n_prop, out, capacity, s, clk);
    }
    if (f.span) cudaEventRecord(t_span[1], s);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    e = cudaMemcpyAsync(f.h ? f.h : &f.local, p.res, sizeof(DevResult), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
    return SKY_OK;
}

// Reads the result block of an enqueued call whose stream has completed.
sky_status skyline_finish(Inflight& f, int64_t* count, sky_run_stats& rs)
{
    rs = {};
    rs.n = f.p.n;
    rs.d = f.p.d;
    rs.log2_g = f.p.log2g;
    if (f.empty) {
        *count = 0;
        return SKY_OK;
    }
    rs.kernels = count_kernels(f.p, f.n_prop, f.capacity);
    const DevResult r = f.h ? *f.h : f.local;
    if (f.span) {
        float ms = 0.0f;
        t_phase = {};
        if (cudaEventElapsedTime(&ms, t_span[0], t_span[1]) == cudaSuccess) t_phase.call_ms = ms;
        cudaGetLastError();
    }
    rs.survivors = r.survivors;
    rs.skyline = r.count;
    rs.pairs = (int64_t)r.pairs;
    rs.n_filter_used = (int32_t)r.n_filter_used;
    rs.tiles = (int64_t)r.tiles;
    rs.group_scans = (int64_t)r.groups;
    rs.code_hits = (int64_t)r.hits;
    rs.exact_tests = (int64_t)r.exact;
    const sky_status st = status_from_flags(r.err);
    if (st != SKY_OK) return st;
    if (f.p.survivors_only && f.capacity >= f.p.n) {   // ids written by the survivor pass itself
        rs.skyline = r.survivors;
        *count = r.survivors;
        return SKY_OK;
    }
    *count = r.count;
    if ((int64_t)r.count > f.capacity)
        return fail(SKY_ERR_CAPACITY, "skyline has %u points, capacity %lld", r.count, (long long)f.capacity);
    return SKY_OK;
}

// The library-internal stream of this thread, ordered after `user_s`.
sky_status internal_stream(cudaStream_t user_s, cudaStream_t* s)
{
    int dev = 0;
    SKY_CUDA(cudaGetDevice(&dev));
    if (!t_stream || t_stream_dev != dev) {
        SKY_CUDA(cudaStreamCreateWithFlags(&t_stream, cudaStreamNonBlocking));
        SKY_CUDA(cudaEventCreateWithFlags(&t_join, cudaEventDisableTiming));
        t_stream_dev = dev;
    }
    SKY_CUDA(cudaEventRecord(t_join, user_s));
    SKY_CUDA(cudaStreamWaitEvent(t_stream, t_join, 0));
    *s = t_stream;
    return SKY_OK;
}

// Whole path on device-resident points. The work runs on a library-internal
// stream that first waits for the caller's stream; the call returns after it
// completes, so the caller sees the usual stream order.
sky_status skyline_device(const float* pts, int64_t n, int32_t d, int64_t ld, const sky_options* opt,
                          int32_t* out, int64_t capacity, int64_t* count, cudaStream_t user_s)
{
    t_stats = {};
    cudaStream_t s = nullptr;
    sky_status st = internal_stream(user_s, &s);
    if (st != SKY_OK) return st;
    Inflight f;
    PhaseClock clk(s);
    st = skyline_enqueue(pts, n, d, ld, opt, out, capacity, s, host_result(), t_timing, clk, f);
    const cudaError_t e = f.empty ? cudaSuccess : cudaStreamSynchronize(s);
    if (st != SKY_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    clk.collect();
    return skyline_finish(f, count, t_stats);
}

// ---------------------------------------------------------------- many sets
// Sets of one sky_skyline_sets / sky_skyline_host_sets call run on up to
// kSetSlots internal streams at once; set i takes slot i % kSetSlots, after
// set i - kSetSlots has completed there.
constexpr int kSetSlots = 4;

struct SetSlots {
    int dev = -1;
    cudaStream_t s[kSetSlots] = {};
    cudaStream_t h2d = nullptr;              // host sets: the input copies, in set order
    cudaEvent_t join = nullptr;
    cudaEvent_t copied[kSetSlots] = {};
    DevResult* res = nullptr;                // page-locked [kSetSlots]
    float* in[kSetSlots] = {};               // host sets: device staging (grow-only)
    int32_t* out[kSetSlots] = {};
    size_t in_cap[kSetSlots] = {}, out_cap[kSetSlots] = {};
};
thread_local SetSlots t_slots;

sky_status set_slots(cudaStream_t user_s, bool host)
{
    SetSlots& S = t_slots;
    int dev = 0;
    SKY_CUDA(cudaGetDevice(&dev));
    if (S.dev != dev) {
        S = SetSlots{};   // streams of another device are abandoned, not reused
        for (int i = 0; i < kSetSlots; ++i) {
            SKY_CUDA(cudaStreamCreateWithFlags(&S.s[i], cudaStreamNonBlocking));
            SKY_CUDA(cudaEventCreateWithFlags(&S.copied[i], cudaEventDisableTiming));
        }
        SKY_CUDA(cudaStreamCreateWithFlags(&S.h2d, cudaStreamNonBlocking));
        SKY_CUDA(cudaEventCreateWithFlags(&S.join, cudaEventDisableTiming));
        SKY_CUDA(cudaMallocHost(&S.res, sizeof(DevResult) * kSetSlots));
        S.dev = dev;
    }
    SKY_CUDA(cudaEventRecord(S.join, user_s));
    for (int i = 0; i < kSetSlots; ++i) SKY_CUDA(cudaStreamWaitEvent(S.s[i], S.join, 0));
    if (host) SKY_CUDA(cudaStreamWaitEvent(S.h2d, S.join, 0));
    return SKY_OK;
}

sky_status grow(void** p, size_t* cap, size_t bytes)
{
    if (bytes <= *cap) return SKY_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    SKY_CUDA(cudaMalloc(p, align256(bytes)));
    *cap = align256(bytes);
    return SKY_OK;
}

sky_status check_sets(const sky_set* sets, int32_t count, const sky_options* opt)
{
    if (count < 0 || (count > 0 && !sets)) return fail(SKY_ERR_INVALID_ARGUMENT, "bad set array");
    if (opt && opt->n_filter != 0)
        return fail(SKY_ERR_INVALID_ARGUMENT, "proposals (n_filter) belong to one set; not accepted here");
    for (int32_t i = 0; i < count; ++i) {
        const sky_set& q = sets[i];
        if (q.capacity < 0 || (q.capacity > 0 && !q.out_idx))
            return fail(SKY_ERR_INVALID_ARGUMENT, "set %d: bad output buffer", i);
        const sky_status st = check_points(q.pts, q.n, q.d, q.ld);
        if (st != SKY_OK) return fail(st, "set %d: %s", i, t_err.c_str());
        Plan p;
        const sky_status sp = make_plan(p, q.pts, q.n, q.d, q.ld, opt);
        if (sp != SKY_OK) return fail(sp, "set %d: %s", i, t_err.c_str());
    }
    return SKY_OK;
}

// Device or host sets. For host sets every input goes to a per-slot device
// staging buffer by one copy on the copy stream (in set order, so the copy
// of set i+1 overlaps the kernels of set i), and the ids come back by one
// copy of `count` entries once the set's count is known.
sky_status run_sets(sky_set* sets, int32_t count, const sky_options* opt, cudaStream_t user_s, bool host)
{
    t_stats = {};
    sky_status st = check_sets(sets, count, opt);
    if (st != SKY_OK) return st;
    for (int32_t i = 0; i < count; ++i) {
        sets[i].count = -1;
        sets[i].status = SKY_OK;
    }
    if (count == 0) return SKY_OK;
    st = set_slots(user_s, host);
    if (st != SKY_OK) return st;
    SetSlots& S = t_slots;
    Inflight fl[kSetSlots];
    int32_t at[kSetSlots];   // set held by each slot, -1: none
    for (int k = 0; k < kSetSlots; ++k) at[k] = -1;
    sky_status first = SKY_OK;
    std::string first_err;
    auto note = [&](int32_t i, sky_status s) {
        sets[i].status = s;
        if (s != SKY_OK && first == SKY_OK) {
            first = s;
            first_err = "set " + std::to_string(i) + ": " + t_err;
        }
    };
    // completes the set that holds slot k (its stream is synchronised)
    auto complete = [&](int k) {
        const int32_t i = at[k];
        if (i < 0) return;
        at[k] = -1;
        const cudaError_t e = cudaStreamSynchronize(S.s[k]);
        if (sets[i].status != SKY_OK) return;   // failed while enqueueing
        if (e != cudaSuccess) { note(i, cuda_fail(e, "stream synchronize")); return; }
        int64_t cnt = -1;   // stays -1 when the set fails before its count is known
        sky_run_stats rs;
        const sky_status fs = skyline_finish(fl[k], &cnt, rs);
        sets[i].count = cnt;
        t_stats.n += rs.n;
        t_stats.d = rs.d;
        t_stats.log2_g = rs.log2_g;
        t_stats.survivors += rs.survivors;
        t_stats.skyline += rs.skyline;
        t_stats.pairs += rs.pairs;
        t_stats.n_filter_used += rs.n_filter_used;
        t_stats.kernels += rs.kernels;
        t_stats.tiles += rs.tiles;
        t_stats.group_scans += rs.group_scans;
        t_stats.code_hits += rs.code_hits;
        t_stats.exact_tests += rs.exact_tests;
        if (fs != SKY_OK || !host) { note(i, fs); return; }
        // host set: the staging buffer holds all cnt ids; the caller's
        // buffer receives at most its capacity
        const int64_t ncopy = std::min(cnt, sets[i].capacity);
        if (ncopy > 0) {
            const cudaError_t ec = cudaMemcpyAsync(sets[i].out_idx, S.out[k], sizeof(int32_t) * (size_t)ncopy,
                                                   cudaMemcpyDeviceToHost, S.s[k]);
            if (ec != cudaSuccess) { note(i, cuda_fail(ec, "device-to-host copy")); return; }
        }
        if (cnt > sets[i].capacity) {
            note(i, fail(SKY_ERR_CAPACITY, "skyline has %lld points, capacity %lld", (long long)cnt,
                         (long long)sets[i].capacity));
            return;
        }
        note(i, SKY_OK);
    };
    for (int32_t i = 0; i < count; ++i) {
        const int k = i % kSetSlots;
        complete(k);   // set i - kSetSlots
        sky_set& q = sets[i];
        fl[k] = Inflight{};
        at[k] = i;
        const float* pts = q.pts;
        int32_t* out = q.out_idx;
        int64_t cap = q.capacity;
        if (host && q.n > 0) {
            // the device buffers hold all n ids, so the count is always known
            const size_t in_bytes = (size_t)((q.n - 1) * q.ld + q.d) * sizeof(float);
            sky_status gs = grow(reinterpret_cast<void**>(&S.in[k]), &S.in_cap[k], in_bytes);
            if (gs == SKY_OK)
                gs = grow(reinterpret_cast<void**>(&S.out[k]), &S.out_cap[k], sizeof(int32_t) * (size_t)q.n);
            if (gs != SKY_OK) { note(i, gs); continue; }
            cudaError_t e = cudaMemcpyAsync(S.in[k], q.pts, in_bytes, cudaMemcpyHostToDevice, S.h2d);
            if (e == cudaSuccess) e = cudaEventRecord(S.copied[k], S.h2d);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(S.s[k], S.copied[k], 0);
            if (e != cudaSuccess) { note(i, cuda_fail(e, "host-to-device copy")); continue; }
            pts = S.in[k];
            out = S.out[k];
            cap = q.n;
        }
        PhaseClock clk(S.s[k], false);   // sets take no phase times
        const sky_status es =
            skyline_enqueue(pts, q.n, q.d, q.ld, opt, out, cap, S.s[k], S.res + k, 0, clk, fl[k]);
        if (es != SKY_OK) note(i, es);
    }
    for (int32_t j = 0; j < kSetSlots; ++j) complete((count + j) % kSetSlots);
    // drain every slot (host sets: the copies of the ids)
    for (int k = 0; k < kSetSlots; ++k) {
        const cudaError_t e = cudaStreamSynchronize(S.s[k]);
        if (e != cudaSuccess && first == SKY_OK) {
            first = cuda_fail(e, "stream synchronize");
            first_err = t_err;
        }
    }
    if (first != SKY_OK) t_err = first_err;
    return first;
}

}  // namespace

namespace sky {

size_t plan_workspace_bytes(int64_t n, int d, int log2g, bool grid_api)
{
    Plan p;
    p.n = n;
    p.d = d;
    p.log2g = log2g;
    return layout(p, nullptr, grid_api);
}

void plan_carve(Plan& p, void* ws, bool grid_api)
{
    layout(p, static_cast<char*>(ws), grid_api);
}

void set_last_error(const char* msg) { t_err = msg ? msg : ""; }

// Setters of every translation unit's wait-limit constant (registered by
// static initialisers, so the table is a function-local static).
struct WaitLimitTable {
    WaitLimitSetter f[32];
    int n = 0;
};
WaitLimitTable& wait_limit_table()
{
    static WaitLimitTable t;
    return t;
}

void register_wait_limit_setter(WaitLimitSetter f)
{
    WaitLimitTable& t = wait_limit_table();
    if (t.n < 32) t.f[t.n++] = f;
}

}  // namespace sky

// ===========================================================================
struct sky_grid {
    Plan plan;
    void* ws = nullptr;
    cudaStream_t stream = nullptr;
    bool pruned = false;
};

extern "C" {

const char* sky_status_string(sky_status s)
{
    switch (s) {
        case SKY_OK: return "ok";
        case SKY_ERR_INVALID_ARGUMENT: return "invalid argument";
        case SKY_ERR_NONFINITE: return "non-finite input";
        case SKY_ERR_CAPACITY: return "output capacity too small";
        case SKY_ERR_OUT_OF_MEMORY: return "out of device memory";
        case SKY_ERR_CUDA: return "CUDA error";
        case SKY_ERR_TOO_LARGE: return "grid too large";
        case SKY_ERR_TIMEOUT: return "device wait timed out";
        case SKY_ERR_NO_DEVICE: return "no usable CUDA device";
    }
    return "unknown status";
}

const char* sky_last_error(void) { return t_err.c_str(); }

const char* sky_version(void) { return "libsky 0.1 (sm_103a)"; }

sky_status sky_set_wait_limit(uint32_t polls)
{
    const WaitLimitTable& t = wait_limit_table();
    for (int i = 0; i < t.n; ++i) SKY_CUDA(t.f[i](polls));
    SKY_CUDA(cudaDeviceSynchronize());
    return SKY_OK;
}

sky_status sky_last_run_stats(sky_run_stats* out)
{
    if (!out) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL stats pointer");
    *out = t_stats;
    return SKY_OK;
}

sky_status sky_set_phase_timing(int32_t enable)
{
    if (enable < 0 || enable > 2) return fail(SKY_ERR_INVALID_ARGUMENT, "timing mode %d outside {0, 1, 2}", enable);
    t_timing = enable;
    return SKY_OK;
}

sky_status sky_last_phase_times(sky_phase_times* out)
{
    if (!out) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL pointer");
    *out = t_phase;
    return SKY_OK;
}

sky_status sky_build_grid(const float* d_pts, int64_t n, int32_t d, int64_t ld, const sky_options* opt,
                          void* stream, sky_grid** out)
{
    if (!out) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL handle pointer");
    *out = nullptr;
    sky_status st = check_points(d_pts, n, d, ld);
    if (st != SKY_OK) return st;
    sky_grid* g = new (std::nothrow) sky_grid();
    if (!g) return fail(SKY_ERR_OUT_OF_MEMORY, "host allocation failed");
    st = make_plan(g->plan, d_pts, n, d, ld, opt);
    if (st != SKY_OK) { delete g; return st; }
    g->stream = static_cast<cudaStream_t>(stream);
    const size_t bytes = layout(g->plan, nullptr, true);
    cudaError_t e = cudaMalloc(&g->ws, bytes);
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "cudaMalloc(grid workspace)"); }
    layout(g->plan, static_cast<char*>(g->ws), true);
    st = run_build(g->plan, g->stream);
    if (st != SKY_OK) { cudaFree(g->ws); delete g; return st; }
    *out = g;
    return SKY_OK;
}

sky_status sky_prune_cells(sky_grid* g, const float* d_filter_pts, int32_t n_filter, void* stream)
{
    if (!g) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL grid");
    if (n_filter < 0 || n_filter > 16) return fail(SKY_ERR_INVALID_ARGUMENT, "n_filter = %d outside [0, 16]", n_filter);
    if (n_filter > 0 && !d_filter_pts) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL proposal pointer");
    if (stream) g->stream = static_cast<cudaStream_t>(stream);
    if (g->plan.n == 0) { g->pruned = true; return SKY_OK; }
    sky_status st = run_prune(g->plan, d_filter_pts, n_filter, g->stream, true);
    if (st == SKY_OK) g->pruned = true;
    return st;
}

sky_status sky_grid_stats(const sky_grid* g, sky_grid_stats_t* out)
{
    if (!g || !out) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->log2_g = g->plan.log2g;
    out->d = g->plan.d;
    out->n = g->plan.n;
    if (g->plan.n == 0) return SKY_OK;
    DevResult r{};
    SKY_CUDA(cudaMemcpyAsync(&r, g->plan.res, sizeof(r), cudaMemcpyDeviceToHost, g->stream));
    SKY_CUDA(cudaStreamSynchronize(g->stream));
    out->occupied_cells = g->pruned ? (int64_t)r.occupied_cells : -1;
    out->surviving_cells = g->pruned ? (int64_t)r.surviving_cells : -1;
    out->surviving_points = g->pruned ? (int64_t)r.survivors : -1;
    out->n_filter_used = (int32_t)r.n_filter_used;
    out->error_flags = (int32_t)r.err;
    return status_from_flags(r.err);
}

sky_status sky_grid_get_view(const sky_grid* g, sky_grid_view* out)
{
    if (!g || !out) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL argument");
    out->cell_key = g->plan.ckey;
    out->occupied = g->plan.occ;
    out->dominated = g->plan.dom;
    out->survivors = reinterpret_cast<const int32_t*>(g->plan.surv_idx);
    out->cell_offset = g->plan.params;
    out->cell_scale = g->plan.params + 16;
    out->words = g->plan.words;
    return SKY_OK;
}

sky_status sky_grid_copy_out(const sky_grid* g, sky_grid_array which, void* d_dst, size_t bytes)
{
    if (!g || (!d_dst && bytes)) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL argument");
    const Plan& p = g->plan;
    const void* src = nullptr;
    size_t need = 0;
    switch (which) {
        case SKY_GRID_CELL_KEY: src = p.ckey; need = sizeof(uint32_t) * (size_t)p.n; break;
        case SKY_GRID_OCCUPIED: src = p.occ; need = sizeof(uint32_t) * (size_t)p.words; break;
        case SKY_GRID_DOMINATED:
            if (!g->pruned) return fail(SKY_ERR_INVALID_ARGUMENT, "grid not pruned yet");
            src = p.dom; need = sizeof(uint32_t) * (size_t)p.words; break;
        case SKY_GRID_SURVIVORS: {
            if (!g->pruned) return fail(SKY_ERR_INVALID_ARGUMENT, "grid not pruned yet");
            DevResult r{};
            if (p.n > 0) {
                SKY_CUDA(cudaMemcpyAsync(&r, p.res, sizeof(r), cudaMemcpyDeviceToHost, g->stream));
                SKY_CUDA(cudaStreamSynchronize(g->stream));
            }
            src = p.surv_idx; need = sizeof(int32_t) * (size_t)r.survivors; break;
        }
        case SKY_GRID_CELL_MAP: src = p.params; need = sizeof(float) * 32; break;
        case SKY_GRID_SNAP:
            if (!g->pruned) return fail(SKY_ERR_INVALID_ARGUMENT, "grid not pruned yet");
            src = p.snap; need = sizeof(unsigned long long) * 16; break;
        default: return fail(SKY_ERR_INVALID_ARGUMENT, "unknown array %d", (int)which);
    }
    if (bytes < need) return fail(SKY_ERR_CAPACITY, "array needs %zu bytes, got %zu", need, bytes);
    if (need) SKY_CUDA(cudaMemcpyAsync(d_dst, src, need, cudaMemcpyDeviceToDevice, g->stream));
    SKY_CUDA(cudaStreamSynchronize(g->stream));
    return SKY_OK;
}

void sky_grid_destroy(sky_grid* g)
{
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    cudaFree(g->ws);
    delete g;
}

sky_status sky_skyline(const float* d_pts, int64_t n, int32_t d, int64_t ld, const sky_options* opt,
                       int32_t* d_out_idx, int64_t out_capacity, int64_t* h_out_count, void* stream)
{
    if (!h_out_count) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL count pointer");
    if (out_capacity < 0 || (out_capacity > 0 && !d_out_idx))
        return fail(SKY_ERR_INVALID_ARGUMENT, "bad output buffer");
    sky_status st = check_points(d_pts, n, d, ld);
    if (st != SKY_OK) return st;
    return skyline_device(d_pts, n, d, ld, opt, d_out_idx, out_capacity, h_out_count,
                          static_cast<cudaStream_t>(stream));
}

sky_status sky_skyline_witness(const float* d_pts, int64_t n, int32_t d, int64_t ld, const sky_options* opt,
                               int32_t* d_out_idx, int64_t out_capacity, int64_t* h_out_count, int32_t* d_witness,
                               void* stream)
{
    t_stats = {};
    if (!h_out_count) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL count pointer");
    if (out_capacity < 0 || (out_capacity > 0 && !d_out_idx))
        return fail(SKY_ERR_INVALID_ARGUMENT, "bad output buffer");
    if (n > 0 && !d_witness) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL witness buffer");
    if (reinterpret_cast<uintptr_t>(d_witness) & 3u) return fail(SKY_ERR_INVALID_ARGUMENT, "witness buffer not 4-byte aligned");
    if (opt && opt->survivors_only != 0)
        return fail(SKY_ERR_INVALID_ARGUMENT, "witnesses are defined for the skyline (survivors_only = 0)");
    sky_status st = check_points(d_pts, n, d, ld);
    if (st != SKY_OK) return st;
    Inflight f;
    st = make_plan(f.p, d_pts, n, d, ld, opt);
    if (st != SKY_OK) return st;
    if (n == 0) { *h_out_count = 0; return SKY_OK; }
    Plan& p = f.p;
    f.capacity = out_capacity;
    f.n_prop = opt ? opt->n_filter : 0;
    const float* prop = f.n_prop ? opt->d_filter_pts : nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    enable_pool_cache();
    void* ws = nullptr;
    int32_t* rep = nullptr;
    p.bytemap = kByteMapMarking;
    const size_t bytes = layout(p, nullptr, false);
    SKY_CUDA(cudaMallocAsync(&ws, bytes, s));
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&rep), sizeof(int32_t) << (p.log2g * p.d), s);
    if (e != cudaSuccess) {
        cudaFreeAsync(ws, s);
        return cuda_fail(e, "cudaMallocAsync(witness cells)");
    }
    layout(p, static_cast<char*>(ws), false);
    p.witness = d_witness;
    e = cudaMemsetAsync(d_witness, 0xff, sizeof(int32_t) * (size_t)n, s);   // -1: kept
    PhaseClock clk(s, false);
    if (e == cudaSuccess) e = enqueue_pipeline(p, prop, f.n_prop, d_out_idx, out_capacity, s, clk, rep);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&f.local, p.res, sizeof(DevResult), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(rep, s);
    cudaFreeAsync(ws, s);
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "witness-mode launch");
    if (es != cudaSuccess) return cuda_fail(es, "stream synchronize");
    return skyline_finish(f, h_out_count, t_stats);
}

size_t sky_tournament_workspace_size(int32_t d, int32_t log2_g)
{
    if (d < 1 || d > kMaxDim || log2_g < 0 || log2_g * d > kTournamentMaxBits) return 0;
    return tournament_workspace_bytes(d, log2_g);
}

sky_status sky_tournament_cells(const uint32_t* d_occupied, int32_t d, int32_t log2_g, uint8_t* d_classes, void* d_ws,
                                size_t ws_bytes, void* stream)
{
    if (d < 1 || d > kMaxDim) return fail(SKY_ERR_INVALID_ARGUMENT, "d = %d outside [1, 16]", d);
    if (log2_g < 0) return fail(SKY_ERR_INVALID_ARGUMENT, "log2_g = %d < 0", log2_g);
    if (log2_g * d > kTournamentMaxBits)
        return fail(SKY_ERR_TOO_LARGE, "layer of 2^%d cells above the tournament limit 2^%d", log2_g * d,
                    kTournamentMaxBits);
    if (!d_occupied || !d_classes) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL bitmap or class buffer");
    const size_t need = tournament_workspace_bytes(d, log2_g);
    if (!d_ws || ws_bytes < need) return fail(SKY_ERR_CAPACITY, "workspace needs %zu bytes", need);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255u) return fail(SKY_ERR_INVALID_ARGUMENT, "workspace not 256-byte aligned");
    SKY_CUDA(launch_tournament(d_occupied, d, log2_g, d_classes, d_ws, static_cast<cudaStream_t>(stream)));
    return SKY_OK;
}

sky_status sky_skyline_sets(sky_set* sets, int32_t count, const sky_options* opt, void* stream)
{
    return run_sets(sets, count, opt, static_cast<cudaStream_t>(stream), false);
}

sky_status sky_skyline_host_sets(sky_set* sets, int32_t count, const sky_options* opt, void* stream)
{
    return run_sets(sets, count, opt, static_cast<cudaStream_t>(stream), true);
}

sky_status sky_skyline_host(const float* h_pts, int64_t n, int32_t d, int64_t ld, const sky_options* opt,
                            int32_t* h_out_idx, int64_t out_capacity, int64_t* h_out_count, void* stream)
{
    if (!h_out_count) return fail(SKY_ERR_INVALID_ARGUMENT, "NULL count pointer");
    if (out_capacity < 0 || (out_capacity > 0 && !h_out_idx))
        return fail(SKY_ERR_INVALID_ARGUMENT, "bad output buffer");
    sky_status st = check_points(h_pts, n, d, ld);
    if (st != SKY_OK) return st;
    if (n == 0) { *h_out_count = 0; return SKY_OK; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    enable_pool_cache();
    // per-thread device staging buffers (grow-only), so that repeated calls
    // hand the same device pointers to the cached path
    thread_local float* t_in = nullptr;
    thread_local int32_t* t_out = nullptr;
    thread_local size_t t_in_cap = 0, t_out_cap = 0;
    const size_t in_bytes = (size_t)((n - 1) * ld + d) * sizeof(float);
    const size_t out_bytes = sizeof(int32_t) * (size_t)n;
    if (in_bytes > t_in_cap) {
        if (t_in) cudaFree(t_in);
        t_in = nullptr;
        t_in_cap = 0;
        SKY_CUDA(cudaMalloc(&t_in, align256(in_bytes)));
        t_in_cap = align256(in_bytes);
    }
    if (out_bytes > t_out_cap) {
        if (t_out) cudaFree(t_out);
        t_out = nullptr;
        t_out_cap = 0;
        SKY_CUDA(cudaMalloc(&t_out, align256(out_bytes)));
        t_out_cap = align256(out_bytes);
    }
    cudaError_t e = cudaMemcpyAsync(t_in, h_pts, in_bytes, cudaMemcpyHostToDevice, s);
    int64_t cnt = 0;
    if (e == cudaSuccess) st = skyline_device(t_in, n, d, ld, opt, t_out, n, &cnt, s);
    else st = cuda_fail(e, "host-to-device copy");
    if (st == SKY_OK) {
        *h_out_count = cnt;
        const int64_t ncopy = cnt < out_capacity ? cnt : out_capacity;
        if (ncopy > 0) {
            e = cudaMemcpyAsync(h_out_idx, t_out, sizeof(int32_t) * (size_t)ncopy, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) st = cuda_fail(e, "device-to-host copy");
        }
        if (st == SKY_OK && cnt > out_capacity)
            st = fail(SKY_ERR_CAPACITY, "skyline has %lld points, capacity %lld", (long long)cnt,
                      (long long)out_capacity);
    }
    e = cudaStreamSynchronize(s);
    if (st == SKY_OK && e != cudaSuccess) st = cuda_fail(e, "stream synchronize");
    return st;
}

}  // extern "C"
