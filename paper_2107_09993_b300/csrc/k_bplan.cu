// k_bplan.cu -- a batch of skyline queries planned on the device: the queries
// live in device memory, the workspace is sized from bounds (queries, total
// rows, columns), and the plan the host batch API builds on the host (per-
// query workspace offsets, work-item prefixes, refinement items grouped by
// padded-dimension class, largest queries first) is built here by kernels,
// so that the whole batch is enqueued without a host round trip and can be
// captured in a CUDA graph. The batched kernels (k_batched.cu) then run with
// grids sized by the bounds, reading the actual counts from the plan.
#include <cstdint>

#include "../../include/sky.h"
#include "sky_common.cuh"
#include "sky_internal.h"

namespace sky {
namespace bplan {

constexpr int kPT = 1024;                 // planner threads (one CTA)
constexpr int kMaxBatchBits = 18;         // batched grids: at most 2^18 cells
constexpr int64_t kMaxWords = int64_t(1) << (kMaxBatchBits - 5);

__host__ __device__ inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// The automatic layer and sort-key bits of a batched query (the rules of
// auto_log2g and morton_bits_for, with the batched 2^18-cell cap).
__device__ inline int plan_log2g(int64_t n, int d)
{
    int r = 24 / d;
    if (r < 1) r = 1;
    if (r > kMaxAutoLayer) r = kMaxAutoLayer;
    const double cap = 32.0 * (double)(n > 1 ? n : 1);
    while (r > 1 && (double)(1ull << (r * d)) > cap) --r;
    while (r > 1 && r * d > kMaxBatchBits) --r;
    return r;
}

__device__ inline int plan_mbits(int64_t n, int d)
{
    int lg = 0;
    while ((1ll << (lg + 1)) <= (n > 1 ? n : 1)) ++lg;
    int target = lg + 6;
    if (target < 16) target = 16;
    if (target > 32) target = 32;
    int b = (target + d / 2) / d;
    if (b < 1) b = 1;
    while (b > 1 && b * d > 32) --b;
    if (b > 16) b = 16;
    return b;
}

// Bytes of one query's arrays, in the order they are carved (the same arrays
// and sizes as the host planner's layout). `zero` receives the bytes of the
// leading arrays that must start at zero (result block, bitmap, look-back
// states, keep bytes, digit totals).
__host__ __device__ inline size_t query_bytes(int64_t n_in, int d, int dp, int64_t words, int64_t chunks,
                                              int64_t tiles, size_t* zero)
{
    const size_t n = (size_t)(n_in > 0 ? n_in : 1);
    const size_t ch = (size_t)(chunks > 0 ? chunks : 1);
    const size_t tl = (size_t)(tiles > 0 ? tiles : 1);
    const size_t npad = tl * kRefineTile;
    size_t at = 0;
    at += a256(sizeof(DevResult));
    at += a256(4 * (size_t)words);
    at += a256(8 * ch);
    at += a256(8 * ch);
    at += a256(n + 16);
    at += a256(4 * 256 * 4);
    at += a256(8 * ((size_t)1 << d));    // layer-1 cell index
    if (zero) *zero = at;
    at += a256(8 * n);                    // keys
    at += a256(4 * (size_t)words);        // prefix-OR
    at += 4 * a256(4 * n);                // sort keys, ids, ping-pong
    at += a256(4 * 256 * ch);             // histograms
    at += a256(4 * npad * (size_t)dp);    // coordinates
    at += a256(npad * (size_t)dp);        // codes
    at += a256(4 * npad);                 // ids
    at += a256(4 * tl * 5 * (size_t)(dp / 4) + 16);
    at += a256(4 * tl);
    at += a256(4 * ((tl + 31) / 32) * (size_t)(dp / 4));
    at += a256(4 * n);                    // stage
    if (dp >= 12) at += a256(16 * npad);  // threshold masks (mask probe)
    return at;
}

// Header of a device-planned workspace: offsets from its base.
struct DevLayout {
    size_t qps, pchunk, ptile, items, cls, qoff, itemoff, claims, data, total;
    int64_t max_items, max_chunks;
};

__host__ inline DevLayout dev_layout(int nq, int n_cols, int64_t max_total_rows)
{
    DevLayout L{};
    const int64_t nqq = nq > 0 ? nq : 1;
    L.max_items = max_total_rows / kRefineTile + nqq + 1;
    L.max_chunks = max_total_rows / kScanTile + nqq + 1;
    size_t at = 0;
    L.qps = at;     at += a256(sizeof(QueryPlan) * (size_t)nqq);
    L.pchunk = at;  at += a256(8 * (size_t)(nqq + 1));
    L.ptile = at;   at += a256(8 * (size_t)(nqq + 1));
    L.items = at;   at += a256(sizeof(int2) * (size_t)L.max_items);
    L.cls = at;     at += a256(sizeof(int) * 8);
    L.qoff = at;    at += a256(8 * (size_t)nqq);
    L.itemoff = at; at += a256(8 * (size_t)nqq);
    L.claims = at;  at += a256(sizeof(uint32_t) * 8);
    L.data = at;
    // per query: the arrays of a zero-row query of the widest class, plus
    // per row the growth of query_bytes with n (rounded up)
    const int cols = n_cols < kMaxDim ? n_cols : kMaxDim;
    const int dpmax = pad4(cols > 0 ? cols : 1);
    const size_t fixed = query_bytes(0, cols > 0 ? cols : 1, dpmax, kMaxWords, 1, 1, nullptr) + 24 * 256;
    const size_t per_row = 35 + 5 * (size_t)dpmax + 1 + (dpmax >= 12 ? 16 : 0);
    at += fixed * (size_t)nqq + per_row * (size_t)(max_total_rows > 0 ? max_total_rows : 0);
    L.total = at;
    return L;
}

// Order key of a query's refinement items: its class, then larger tile
// counts first (by floor(log2 tiles)).
__device__ inline int item_key(int dpclass, int64_t tiles)
{
    const int lg = 63 - __clzll((long long)tiles);
    return dpclass * 32 + (31 - (lg < 31 ? lg : 31));
}

// Block-wide exclusive scan of one int64 per thread (kPT threads).
__device__ inline int64_t block_scan64(int64_t v, int64_t* s_warp, int64_t& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    total = s_warp[31];
    const int64_t before = warp > 0 ? s_warp[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

// One CTA plans every query: validation, layer and key bits, sizes, the
// exclusive prefixes of workspace bytes, chunks and tiles, the pointers into
// the workspace, and each query's first refinement item (class-major, then
// larger queries first by power-of-two buckets of their tile count).
__global__ void __launch_bounds__(kPT) kb_plan(const sky_query* __restrict__ Q, int nq, const float* table,
                                               int64_t n_rows, int n_cols, int64_t rs, int64_t cs, char* data,
                                               size_t data_bytes, int64_t max_rows, int64_t max_chunks,
                                               int64_t max_tiles, QueryPlan* qps, int64_t* pchunk, int64_t* ptile,
                                               int* cls, int64_t* qoff, int64_t* itemoff)
{
    __shared__ int64_t s_warp[32];
    __shared__ unsigned long long s_hist[128], s_cur[128];
    __shared__ int64_t s_carry[4];
    __shared__ int s_over;
    const int tid = threadIdx.x;
    if (tid < 128) s_hist[tid] = 0ull;
    if (tid < 4) s_carry[tid] = 0;
    if (tid == 0) s_over = 0;
    __syncthreads();
    const uint32_t allowed = n_cols >= 32 ? 0xffffffffu : ((1u << n_cols) - 1u);
    // 1. per-query plan (without pointers) and its sizes
    for (int q0 = 0; q0 < nq; q0 += kPT) {
        const int q = q0 + tid;
        int64_t bytes = 0, chunks = 0, tiles = 0, rows = 0;
        if (q < nq) {
            const sky_query R = Q[q];
            QueryPlan p;
            memset(&p, 0, sizeof(p));
            const int d = __popc(R.dim_mask);
            const bool bad = (R.flags & ~SKY_QUERY_QUADRANT) != 0u || R.row_begin < 0 || R.row_count < 0 ||
                             R.row_begin > n_rows - R.row_count || R.dim_mask == 0u ||
                             (R.dim_mask & ~allowed) != 0u || d > kMaxDim;
            p.rs = rs;
            p.cs = cs;
            if (bad) {
                p.invalid = 1;
                p.d = 1;
                p.dp = 4;
                p.log2g = 1;
                p.mbits = 1;
                p.words = 1;
            } else {
                p.n = R.row_count;
                p.row_begin = R.row_begin;
                p.d = d;
                p.dp = pad4(d);
                int c = 0;
                for (int k = 0; k < 32; ++k)
                    if ((R.dim_mask >> k) & 1u) p.col[c++] = k;
                p.quadrant = (R.flags & SKY_QUERY_QUADRANT) ? 1 : 0;
                for (int k = 0; k < kMaxDim; ++k) p.origin[k] = (p.quadrant && k < d) ? R.origin[k] : 0.0f;
                p.log2g = plan_log2g(p.n, d);
                p.mbits = plan_mbits(p.n, d);
                p.words = (1ll << (p.log2g * d)) / 32 > 1 ? (1ll << (p.log2g * d)) / 32 : 1;
            }
            p.passes = (p.mbits * p.d + 7) / 8;
            p.dpclass = p.dp / 4 - 1;
            p.chunks = (p.n + kScanTile - 1) / kScanTile;
            p.tiles = (p.n + kRefineTile - 1) / kRefineTile;
            chunks = p.chunks;
            tiles = p.tiles;
            rows = p.n;
            bytes = (int64_t)query_bytes(p.n, p.d, p.dp, p.words, p.chunks, p.tiles, nullptr);
            qps[q] = p;
        }
        int64_t tb, tc, tt, tr;
        const int64_t ob = block_scan64(bytes, s_warp, tb);
        const int64_t oc = block_scan64(chunks, s_warp, tc);
        const int64_t ot = block_scan64(tiles, s_warp, tt);
        block_scan64(rows, s_warp, tr);
        if (q < nq) {
            qoff[q] = s_carry[0] + ob;
            pchunk[q] = s_carry[1] + oc;
            ptile[q] = s_carry[2] + ot;
        }
        __syncthreads();
        if (tid == 0) {
            s_carry[0] += tb;
            s_carry[1] += tc;
            s_carry[2] += tt;
            s_carry[3] += tr;
        }
        __syncthreads();
    }
    if (tid == 0) {
        pchunk[nq] = s_carry[1];
        ptile[nq] = s_carry[2];
        // every grid of the batched kernels is sized by these bounds
        s_over = ((size_t)s_carry[0] > data_bytes || s_carry[3] > max_rows || s_carry[1] > max_chunks ||
                  s_carry[2] > max_tiles) ? 1 : 0;
    }
    __syncthreads();
    // 2. beyond the workspace bound (more rows than max_total_rows): no query runs
    if (s_over) {
        for (int q = tid; q < nq; q += kPT) {
            qps[q].n = 0;
            qps[q].chunks = 0;
            qps[q].tiles = 0;
            if (!qps[q].invalid) qps[q].invalid = 2;
            qoff[q] = 0;
        }
        for (int q = tid; q <= nq; q += kPT) {
            pchunk[q] = 0;
            ptile[q] = 0;
        }
        __syncthreads();
    }
    // 3. pointers into the workspace (query q's arrays start at data + qoff[q])
    for (int q = tid; q < nq; q += kPT) {
        QueryPlan& p = qps[q];
        char* b = data + qoff[q];
        const size_t n = (size_t)(p.n > 0 ? p.n : 1);
        const size_t ch = (size_t)(p.chunks > 0 ? p.chunks : 1);
        const size_t tl = (size_t)(p.tiles > 0 ? p.tiles : 1);
        const size_t npad = tl * kRefineTile;
        size_t at = 0;
        auto take = [&](size_t sz) { char* r = b + at; at += a256(sz); return r; };
        p.base = table + (n_rows > 0 ? p.row_begin * rs : 0);
        p.res = reinterpret_cast<DevResult*>(take(sizeof(DevResult)));
        p.occ = reinterpret_cast<uint32_t*>(take(4 * (size_t)p.words));
        p.lb_a = reinterpret_cast<unsigned long long*>(take(8 * ch));
        p.lb_b = reinterpret_cast<unsigned long long*>(take(8 * ch));
        p.keep = reinterpret_cast<uint8_t*>(take(n + 16));
        p.digit_total = reinterpret_cast<uint32_t*>(take(4 * 256 * 4));
        p.cidx = reinterpret_cast<uint32_t*>(take(8 * ((size_t)1 << p.d)));
        p.keys = reinterpret_cast<uint2*>(take(8 * n));
        p.pre = reinterpret_cast<uint32_t*>(take(4 * (size_t)p.words));
        p.surv_key = reinterpret_cast<uint32_t*>(take(4 * n));
        p.surv_idx = reinterpret_cast<uint32_t*>(take(4 * n));
        p.key2 = reinterpret_cast<uint32_t*>(take(4 * n));
        p.val2 = reinterpret_cast<uint32_t*>(take(4 * n));
        p.hist = reinterpret_cast<uint32_t*>(take(4 * 256 * ch));
        p.X = reinterpret_cast<float*>(take(4 * npad * (size_t)p.dp));
        p.C = reinterpret_cast<uint32_t*>(take(npad * (size_t)p.dp));
        p.ids = reinterpret_cast<int32_t*>(take(4 * npad));
        p.sub = reinterpret_cast<uint32_t*>(take(4 * tl * 5 * (size_t)(p.dp / 4) + 16));
        p.tend = reinterpret_cast<uint32_t*>(take(4 * tl));
        p.supmin = reinterpret_cast<uint32_t*>(take(4 * ((tl + 31) / 32) * (size_t)(p.dp / 4)));
        p.stage = reinterpret_cast<int32_t*>(take(4 * n));
        p.tmask = p.dp >= 12 ? reinterpret_cast<uint32_t*>(take(16 * npad)) : nullptr;
    }
    __syncthreads();
    // 4. refinement items: class-major, larger queries first (buckets of
    // floor(log2 tiles), largest bucket first); order inside a bucket is free
    for (int q = tid; q < nq; q += kPT) {
        const int64_t t = qps[q].tiles;
        if (t > 0) {
            atomicAdd(&s_hist[item_key(qps[q].dpclass, t)], (unsigned long long)t);
        }
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long acc = 0;
        for (int k = 0; k < 128; ++k) {
            s_cur[k] = acc;
            acc += s_hist[k];
        }
        for (int c = 0; c < 4; ++c) {
            unsigned long long items = 0;
            for (int k = 0; k < 32; ++k) items += s_hist[c * 32 + k];
            cls[c] = (int)s_cur[c * 32];
            cls[4 + c] = (int)items;
        }
    }
    __syncthreads();
    for (int q = tid; q < nq; q += kPT) {
        const int64_t t = qps[q].tiles;
        if (t > 0) {
            itemoff[q] = (int64_t)atomicAdd(&s_cur[item_key(qps[q].dpclass, t)], (unsigned long long)t);
        } else {
            itemoff[q] = 0;
        }
    }
}

// Zeroes each query's leading arrays (result block to digit totals: every
// one of them 256-byte aligned and sized, so 16-byte stores cover them) and
// the work counters. Grid: (queries, kZeroSplit).
constexpr int kZeroSplit = 8;
__global__ void __launch_bounds__(256) kb_zero(const QueryPlan* __restrict__ qps, int nq, uint32_t* claims)
{
    const int q = blockIdx.x;
    if (q == 0 && blockIdx.y == 0 && threadIdx.x < 8) claims[threadIdx.x] = 0u;
    if (q >= nq) return;
    const QueryPlan& p = qps[q];
    uint4* z = reinterpret_cast<uint4*>(p.res);
    const int64_t n16 = (reinterpret_cast<const char*>(p.keys) - reinterpret_cast<const char*>(p.res)) / 16;
    for (int64_t i = blockIdx.y * 256 + threadIdx.x; i < n16; i += kZeroSplit * 256) z[i] = make_uint4(0, 0, 0, 0);
}

// The refinement items (query, p-tile) at each query's planned offset.
__global__ void __launch_bounds__(256) kb_items(const int64_t* __restrict__ ptile, int nq,
                                                const int64_t* __restrict__ itemoff, int2* items)
{
    const int64_t total = ptile[nq];
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < total; i += (int64_t)gridDim.x * 256) {
        int lo = 0, hi = nq - 1;   // the query whose tile range holds i (largest q with ptile[q] <= i)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ptile[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const int64_t t = i - ptile[lo];
        items[itemoff[lo] + t] = make_int2(lo, (int)t);
    }
}

int device_sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1) n = 1;
    }
    return n;
}

}  // namespace bplan

size_t batched_device_workspace_bytes(int n_cols, int nq, int64_t max_total_rows)
{
    return bplan::dev_layout(nq, n_cols, max_total_rows).total;
}

// Plans the batch on the device and enqueues every phase on `s`: no host
// synchronisation, no allocation, no copy. The batched kernels run with
// grids sized by the bounds (max_total_rows, n_queries) and read the
// planned counts; a query beyond the bounds reports SKY_ERR_TOO_LARGE.
cudaError_t launch_batched_device(const float* table, int64_t n_rows, int n_cols, int64_t rs, int64_t cs,
                                  const sky_query* d_queries, int nq, int64_t max_total_rows, void* ws, size_t ws_bytes,
                                  int32_t* out, int64_t capacity, int64_t* offsets, int32_t* status, cudaStream_t s)
{
    using namespace bplan;
    const DevLayout L = dev_layout(nq, n_cols, max_total_rows);
    char* w = static_cast<char*>(ws);
    auto* qps = reinterpret_cast<QueryPlan*>(w + L.qps);
    auto* pchunk = reinterpret_cast<int64_t*>(w + L.pchunk);
    auto* ptile = reinterpret_cast<int64_t*>(w + L.ptile);
    auto* items = reinterpret_cast<int2*>(w + L.items);
    auto* cls = reinterpret_cast<int*>(w + L.cls);
    auto* qoff = reinterpret_cast<int64_t*>(w + L.qoff);
    auto* itemoff = reinterpret_cast<int64_t*>(w + L.itemoff);
    auto* claims = reinterpret_cast<uint32_t*>(w + L.claims);
    kb_plan<<<1, kPT, 0, s>>>(d_queries, nq, table, n_rows, n_cols, rs, cs, w + L.data, ws_bytes - L.data,
                              max_total_rows, L.max_chunks, L.max_items, qps, pchunk, ptile, cls, qoff, itemoff);
    kb_zero<<<dim3((unsigned)(nq > 0 ? nq : 1), kZeroSplit), 256, 0, s>>>(qps, nq, claims);
    const int64_t ib = (L.max_items + 255) / 256;
    kb_items<<<(unsigned)(ib < device_sm_count() * 8 ? ib : device_sm_count() * 8), 256, 0, s>>>(ptile, nq, itemoff,
                                                                                                 items);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    BatchLaunch b;
    b.qps = qps;
    b.nq = nq;
    b.pchunk = pchunk;
    b.chunk_items = L.max_chunks;
    b.ptile = ptile;
    b.tile_items = L.max_items;
    b.items = items;
    const int imax = (int)(L.max_items < (int64_t)INT32_MAX ? L.max_items : INT32_MAX);
    for (int c = 0; c < 4; ++c) {
        b.class_begin[c] = 0;
        b.class_items[c] = imax;
    }
    b.claims = claims;
    b.max_passes = 4;
    b.max_words = kMaxWords;
    b.d_class = cls;
    b.out = out;
    b.capacity = capacity;
    b.offsets = offsets;
    b.status = status;
    return launch_batched(b, s);
}

}  // namespace sky
