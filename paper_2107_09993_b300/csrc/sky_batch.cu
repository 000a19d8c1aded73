// sky_batch.cu -- C ABI of the batched skyline (include/sky.h): planning of
// the per-query workspace on the host, one upload of the plan, and one CUDA
// graph that runs every phase for every query (k_batched.cu).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/sky.h"
#include "sky_common.cuh"
#include "sky_internal.h"

using namespace sky;

namespace {

thread_local std::string t_berr;

sky_status bfail(sky_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
sky_status bfail(sky_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_berr = buf;
    return s;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct QOff {   // byte offsets of one query's arrays inside the workspace
    size_t res, occ, lb_a, lb_b, keep, dt, cidx;                             // zero region
    size_t keys, pre, skey, sidx, key2, val2, hist, X, C, ids, sub, tend, supmin, stage, tmask;   // other
};

}  // namespace

struct sky_batch {
    const float* table = nullptr;
    int64_t n_rows = 0, rs = 0, cs = 0;
    int n_cols = 0;
    std::vector<QueryPlan> plans;       // host copy; pointers filled at bind time
    std::vector<QOff> off;
    std::vector<int64_t> pchunk, ptile;
    std::vector<int2> items;
    int class_begin[4] = {0, 0, 0, 0}, class_items[4] = {0, 0, 0, 0};
    size_t hdr_bytes = 0, off_qps = 0, off_pchunk = 0, off_ptile = 0, off_items = 0;
    size_t zero_begin = 0, zero_bytes = 0, off_claims = 0, total = 0;
    int max_passes = 0;
    int64_t max_words = 1;
    int refine_ctas_per_sm = 0;
    void* ws = nullptr;
    cudaGraphExec_t exec = nullptr;
    BatchLaunch launch;
};

extern "C" {

const char* sky_batch_last_error(void) { return t_berr.c_str(); }

sky_status sky_batch_create(const float* d_table, int64_t n_rows, int32_t n_cols, int64_t row_stride,
                            int64_t col_stride, const sky_query* h_queries, int32_t n_queries,
                            const sky_batch_tuning* tuning, sky_batch** out, size_t* ws_bytes)
{
    if (!out || !ws_bytes) return bfail(SKY_ERR_INVALID_ARGUMENT, "NULL output pointer");
    *out = nullptr;
    *ws_bytes = 0;
    if (n_rows < 0 || n_rows >= (int64_t(1) << 31)) return bfail(SKY_ERR_INVALID_ARGUMENT, "n_rows outside [0, 2^31)");
    if (n_cols < 1 || n_cols > 32) return bfail(SKY_ERR_INVALID_ARGUMENT, "n_cols outside [1, 32]");
    if (n_queries < 0 || (n_queries > 0 && !h_queries)) return bfail(SKY_ERR_INVALID_ARGUMENT, "bad query array");
    if (n_rows > 0 && !d_table) return bfail(SKY_ERR_INVALID_ARGUMENT, "NULL table");
    if (reinterpret_cast<uintptr_t>(d_table) & 3u) return bfail(SKY_ERR_INVALID_ARGUMENT, "table not 4-byte aligned");
    const bool row_major = col_stride == 1 && row_stride >= n_cols;
    const bool col_major = row_stride == 1 && col_stride >= n_rows;
    if (!row_major && !col_major)
        return bfail(SKY_ERR_INVALID_ARGUMENT, "strides must describe a row-major (col_stride 1) or "
                                               "column-major (row_stride 1) table");
    if (tuning && tuning->refine_ctas_per_sm < 0) return bfail(SKY_ERR_INVALID_ARGUMENT, "negative CTAs per SM");
    if (tuning) {
        for (int c = 0; c < 4; ++c) {
            if (tuning->class_ctas[c] < 0) return bfail(SKY_ERR_INVALID_ARGUMENT, "class %d: negative CTAs per SM", c);
            if (tuning->class_stages[c] != 0 && tuning->class_stages[c] != 4 && tuning->class_stages[c] != 8)
                return bfail(SKY_ERR_INVALID_ARGUMENT, "class %d: ring depth %d not in {0, 4, 8}", c,
                             tuning->class_stages[c]);
            if (tuning->class_code[c] < 0 || tuning->class_code[c] > 2)
                return bfail(SKY_ERR_INVALID_ARGUMENT, "class %d: pair-test code %d not in {0, 1, 2}", c,
                             tuning->class_code[c]);
        }
        if (tuning->concurrent_classes < 0 || tuning->concurrent_classes > 1)
            return bfail(SKY_ERR_INVALID_ARGUMENT, "concurrent_classes not in {0, 1}");
    }
    sky_batch* b = new (std::nothrow) sky_batch();
    if (!b) return bfail(SKY_ERR_OUT_OF_MEMORY, "host allocation failed");
    b->table = d_table;
    b->n_rows = n_rows;
    b->n_cols = n_cols;
    b->rs = row_stride;
    b->cs = col_stride;
    b->refine_ctas_per_sm = tuning ? tuning->refine_ctas_per_sm : 0;
    for (int c = 0; c < 4; ++c) {
        b->launch.class_ctas[c] = tuning ? tuning->class_ctas[c] : 0;
        b->launch.class_stages[c] = (tuning && tuning->class_stages[c]) ? tuning->class_stages[c] : 8;
        const int code = tuning ? tuning->class_code[c] : 0;
        b->launch.class_fast[c] = code == 0 ? (c == 3 ? 1 : 0) : (code == 2 ? 1 : 0);
    }
    b->launch.concurrent_classes = tuning && tuning->concurrent_classes == 1;
    const int nq = n_queries;
    b->plans.resize(nq);
    b->off.resize(nq);
    b->pchunk.assign(nq + 1, 0);
    b->ptile.assign(nq + 1, 0);

    // -------- per-query plan
    for (int q = 0; q < nq; ++q) {
        const sky_query& Q = h_queries[q];
        if ((Q.flags & ~SKY_QUERY_QUADRANT) != 0 || Q.row_begin < 0 || Q.row_count < 0 ||
            Q.row_begin + Q.row_count > n_rows) {
            delete b;
            return bfail(SKY_ERR_INVALID_ARGUMENT, "query %d: bad row range or unknown flag", q);
        }
        const uint32_t allowed = n_cols >= 32 ? 0xffffffffu : ((1u << n_cols) - 1u);
        const int d = __builtin_popcount(Q.dim_mask);
        if (Q.dim_mask == 0 || (Q.dim_mask & ~allowed) || d > kMaxDim) {
            delete b;
            return bfail(SKY_ERR_INVALID_ARGUMENT, "query %d: dim_mask selects no column, a missing column "
                                                   "or more than 16 columns", q);
        }
        QueryPlan& p = b->plans[q];
        memset(&p, 0, sizeof(p));
        p.n = Q.row_count;
        p.row_begin = Q.row_begin;
        p.rs = row_stride;
        p.cs = col_stride;
        p.d = d;
        p.dp = pad4(d);
        int c = 0;
        for (int k = 0; k < 32; ++k)
            if ((Q.dim_mask >> k) & 1u) p.col[c++] = k;
        p.quadrant = (Q.flags & SKY_QUERY_QUADRANT) ? 1 : 0;
        for (int k = 0; k < kMaxDim; ++k) p.origin[k] = (p.quadrant && k < d) ? Q.origin[k] : 0.0f;
        int lg = -1;
        if (tuning && tuning->h_log2g) lg = tuning->h_log2g[q];
        if (lg < 0) {
            lg = auto_log2g(p.n, d);
            while (lg > 1 && lg * d > 18) --lg;
        }
        if (lg * d > 18 || lg > 16) {
            delete b;
            return bfail(SKY_ERR_TOO_LARGE, "query %d: grid of 2^%d cells above the batched limit 2^18", q, lg * d);
        }
        p.log2g = lg;
        p.mbits = morton_bits_for(p.n, d);
        p.passes = (p.mbits * d + 7) / 8;
        p.dpclass = p.dp / 4 - 1;
        p.words = std::max<int64_t>(1, (1ll << (lg * d)) / 32);
        p.chunks = (p.n + kScanTile - 1) / kScanTile;
        p.tiles = (p.n + kRefineTile - 1) / kRefineTile;
        b->pchunk[q + 1] = b->pchunk[q] + p.chunks;
        b->ptile[q + 1] = b->ptile[q] + p.tiles;
        if (p.n > 0) {
            b->max_passes = std::max(b->max_passes, p.passes);
            b->max_words = std::max(b->max_words, p.words);
        }
    }
    // refinement items: grouped by padded-dimension class, larger queries first
    std::vector<int> order(nq);
    for (int q = 0; q < nq; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->plans[a].n > b->plans[c].n; });
    for (int cls = 0; cls < 4; ++cls) {
        b->class_begin[cls] = (int)b->items.size();
        for (int q : order) {
            const QueryPlan& p = b->plans[q];
            if (p.dpclass != cls) continue;
            for (int64_t t = 0; t < p.tiles; ++t) b->items.push_back(make_int2(q, (int)t));
        }
        b->class_items[cls] = (int)b->items.size() - b->class_begin[cls];
    }

    // -------- workspace layout
    size_t at = 0;
    b->off_qps = at;    at = a256(at + sizeof(QueryPlan) * (size_t)nq);
    b->off_pchunk = at; at = a256(at + sizeof(int64_t) * (size_t)(nq + 1));
    b->off_ptile = at;  at = a256(at + sizeof(int64_t) * (size_t)(nq + 1));
    b->off_items = at;  at = a256(at + sizeof(int2) * std::max<size_t>(1, b->items.size()));
    b->hdr_bytes = at;
    b->zero_begin = at;
    b->off_claims = at; at = a256(at + 8 * sizeof(uint32_t));
    for (int q = 0; q < nq; ++q) {
        const QueryPlan& p = b->plans[q];
        QOff& o = b->off[q];
        const size_t n = (size_t)std::max<int64_t>(p.n, 1);
        o.res = at;  at = a256(at + sizeof(DevResult));
        o.occ = at;  at = a256(at + 4 * (size_t)p.words);
        o.lb_a = at; at = a256(at + 8 * (size_t)std::max<int64_t>(p.chunks, 1));
        o.lb_b = at; at = a256(at + 8 * (size_t)std::max<int64_t>(p.chunks, 1));
        o.keep = at; at = a256(at + n + 16);
        o.dt = at;   at = a256(at + 4 * 256 * 4);
        o.cidx = at; at = a256(at + 8 * ((size_t)1 << p.d));
    }
    b->zero_bytes = at - b->zero_begin;
    for (int q = 0; q < nq; ++q) {
        const QueryPlan& p = b->plans[q];
        QOff& o = b->off[q];
        const size_t n = (size_t)std::max<int64_t>(p.n, 1);
        const size_t npad = (size_t)std::max<int64_t>(p.tiles, 1) * kRefineTile;
        o.keys = at;  at = a256(at + 8 * n);
        o.pre = at;   at = a256(at + 4 * (size_t)p.words);
        o.skey = at;  at = a256(at + 4 * n);
        o.sidx = at;  at = a256(at + 4 * n);
        o.key2 = at;  at = a256(at + 4 * n);
        o.val2 = at;  at = a256(at + 4 * n);
        o.hist = at;  at = a256(at + 4 * 256 * (size_t)std::max<int64_t>(p.chunks, 1));
        o.X = at;     at = a256(at + 4 * npad * (size_t)p.dp);
        o.C = at;     at = a256(at + npad * (size_t)p.dp);
        o.ids = at;   at = a256(at + 4 * npad);
        o.sub = at;   at = a256(at + 4 * (size_t)std::max<int64_t>(p.tiles, 1) * 5 * (size_t)(p.dp / 4) + 16);
        o.tend = at;  at = a256(at + 4 * (size_t)std::max<int64_t>(p.tiles, 1));
        o.supmin = at; at = a256(at + 4 * (size_t)((std::max<int64_t>(p.tiles, 1) + 31) / 32) * (size_t)(p.dp / 4));
        o.stage = at; at = a256(at + 4 * n);
        o.tmask = at; at = a256(at + (p.dp >= 12 ? 16 * npad : 0));   // threshold masks (mask probe)
    }
    b->total = at;
    *ws_bytes = at;
    *out = b;
    return SKY_OK;
}

size_t sky_batched_workspace_size(int64_t n_rows, int32_t n_cols, int64_t row_stride, int64_t col_stride,
                                  const sky_query* h_queries, int32_t n_queries, const sky_batch_tuning* tuning)
{
    sky_batch* b = nullptr;
    size_t bytes = 0;
    // a non-null, aligned placeholder: the size does not depend on the table address
    const float* fake = reinterpret_cast<const float*>(uintptr_t(256));
    if (sky_batch_create(fake, n_rows, n_cols, row_stride, col_stride, h_queries, n_queries, tuning, &b, &bytes) !=
        SKY_OK)
        return 0;
    delete b;
    return bytes;
}

sky_status sky_batch_bind(sky_batch* b, void* d_ws, size_t ws_bytes, int32_t* d_out_idx, int64_t out_capacity,
                          int64_t* d_out_offsets, int32_t* d_query_status, void* stream)
{
    if (!b) return bfail(SKY_ERR_INVALID_ARGUMENT, "NULL batch");
    if (!d_ws || ws_bytes < b->total) return bfail(SKY_ERR_CAPACITY, "workspace needs %zu bytes", b->total);
    if ((reinterpret_cast<uintptr_t>(d_ws) & 255u) != 0) return bfail(SKY_ERR_INVALID_ARGUMENT, "workspace not 256-byte aligned");
    if (!d_out_offsets || !d_query_status || out_capacity < 0 || (out_capacity > 0 && !d_out_idx))
        return bfail(SKY_ERR_INVALID_ARGUMENT, "bad output buffers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(d_ws);
    const int nq = (int)b->plans.size();
    for (int q = 0; q < nq; ++q) {
        QueryPlan& p = b->plans[q];
        const QOff& o = b->off[q];
        p.base = b->table + p.row_begin * b->rs;
        p.keys = reinterpret_cast<uint2*>(ws + o.keys);
        p.occ = reinterpret_cast<uint32_t*>(ws + o.occ);
        p.pre = reinterpret_cast<uint32_t*>(ws + o.pre);
        p.lb_a = reinterpret_cast<unsigned long long*>(ws + o.lb_a);
        p.lb_b = reinterpret_cast<unsigned long long*>(ws + o.lb_b);
        p.surv_key = reinterpret_cast<uint32_t*>(ws + o.skey);
        p.surv_idx = reinterpret_cast<uint32_t*>(ws + o.sidx);
        p.key2 = reinterpret_cast<uint32_t*>(ws + o.key2);
        p.val2 = reinterpret_cast<uint32_t*>(ws + o.val2);
        p.hist = reinterpret_cast<uint32_t*>(ws + o.hist);
        p.digit_total = reinterpret_cast<uint32_t*>(ws + o.dt);
        p.X = reinterpret_cast<float*>(ws + o.X);
        p.C = reinterpret_cast<uint32_t*>(ws + o.C);
        p.ids = reinterpret_cast<int32_t*>(ws + o.ids);
        p.sub = reinterpret_cast<uint32_t*>(ws + o.sub);
        p.tend = reinterpret_cast<uint32_t*>(ws + o.tend);
        p.supmin = reinterpret_cast<uint32_t*>(ws + o.supmin);
        p.cidx = reinterpret_cast<uint32_t*>(ws + o.cidx);
        p.keep = reinterpret_cast<uint8_t*>(ws + o.keep);
        p.stage = reinterpret_cast<int32_t*>(ws + o.stage);
        p.tmask = p.dp >= 12 ? reinterpret_cast<uint32_t*>(ws + o.tmask) : nullptr;
        p.res = reinterpret_cast<DevResult*>(ws + o.res);
    }
    std::vector<char> hdr(b->hdr_bytes, 0);
    if (nq) memcpy(hdr.data() + b->off_qps, b->plans.data(), sizeof(QueryPlan) * (size_t)nq);
    memcpy(hdr.data() + b->off_pchunk, b->pchunk.data(), sizeof(int64_t) * (size_t)(nq + 1));
    memcpy(hdr.data() + b->off_ptile, b->ptile.data(), sizeof(int64_t) * (size_t)(nq + 1));
    if (!b->items.empty()) memcpy(hdr.data() + b->off_items, b->items.data(), sizeof(int2) * b->items.size());
    cudaError_t e = cudaMemcpyAsync(ws, hdr.data(), b->hdr_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bfail(SKY_ERR_CUDA, "plan upload: %s", cudaGetErrorString(e));

    BatchLaunch& L = b->launch;
    L.qps = reinterpret_cast<const QueryPlan*>(ws + b->off_qps);
    L.nq = nq;
    L.pchunk = reinterpret_cast<const int64_t*>(ws + b->off_pchunk);
    L.chunk_items = b->pchunk[nq];
    L.ptile = reinterpret_cast<const int64_t*>(ws + b->off_ptile);
    L.tile_items = b->ptile[nq];
    L.items = reinterpret_cast<const int2*>(ws + b->off_items);
    for (int c = 0; c < 4; ++c) {
        L.class_begin[c] = b->class_begin[c];
        L.class_items[c] = b->class_items[c];
    }
    L.claims = reinterpret_cast<uint32_t*>(ws + b->off_claims);
    L.zero_base = ws + b->zero_begin;
    L.zero_bytes = b->zero_bytes;
    L.max_passes = b->max_passes;
    L.max_words = b->max_words;
    L.refine_ctas_per_sm = b->refine_ctas_per_sm;
    if (L.concurrent_classes && !L.fork) {
        e = cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming);
        for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
            e = cudaStreamCreateWithFlags(&L.class_streams[c], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.joins[c], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return bfail(SKY_ERR_CUDA, "class streams: %s", cudaGetErrorString(e));
    }
    L.out = d_out_idx;
    L.capacity = out_capacity;
    L.offsets = d_out_offsets;
    L.status = d_query_status;

    // one direct run first (sets kernel attributes outside capture), then capture
    e = launch_batched(L, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bfail(SKY_ERR_CUDA, "batched launch: %s", cudaGetErrorString(e));
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaStream_t cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bfail(SKY_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t e1 = launch_batched(L, cap);
        const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    b->ws = d_ws;
    if (e != cudaSuccess) {
        b->exec = nullptr;
        cudaGetLastError();
        return bfail(SKY_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    return SKY_OK;
}

sky_status sky_skyline_batched(sky_batch* b, void* stream)
{
    if (!b || !b->exec) return bfail(SKY_ERR_INVALID_ARGUMENT, "batch not bound");
    const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return bfail(SKY_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    return SKY_OK;
}

sky_status sky_batch_stats(const sky_batch* b, void* stream, sky_batch_stats_t* out)
{
    if (!b || !out || !b->ws) return bfail(SKY_ERR_INVALID_ARGUMENT, "batch not bound");
    memset(out, 0, sizeof(*out));
    const int nq = (int)b->plans.size();
    out->n_queries = nq;
    out->kernels = batched_kernel_count(b->launch);
    out->graph_launches_per_call = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bfail(SKY_ERR_CUDA, "%s", cudaGetErrorString(e));
    for (int q = 0; q < nq; ++q) {
        DevResult r{};
        e = cudaMemcpy(&r, b->plans[q].res, sizeof(r), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bfail(SKY_ERR_CUDA, "%s", cudaGetErrorString(e));
        out->points += b->plans[q].n;
        out->survivors += b->plans[q].n ? r.survivors : 0;
        out->skyline += b->plans[q].n ? r.count : 0;
        out->pairs += b->plans[q].n ? (int64_t)r.pairs : 0;
    }
    return SKY_OK;
}

void sky_batch_destroy(sky_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (int c = 0; c < 4; ++c) {
        if (b->launch.class_streams[c]) cudaStreamDestroy(b->launch.class_streams[c]);
        if (b->launch.joins[c]) cudaEventDestroy(b->launch.joins[c]);
    }
    if (b->launch.fork) cudaEventDestroy(b->launch.fork);
    delete b;
}

size_t sky_batched_device_workspace_size(int32_t n_cols, int32_t n_queries, int64_t max_total_rows)
{
    if (n_cols < 1 || n_cols > 32 || n_queries < 0 || max_total_rows < 0) return 0;
    return batched_device_workspace_bytes(n_cols, n_queries, max_total_rows);
}

sky_status sky_skyline_batched_device(const float* d_table, int64_t n_rows, int32_t n_cols, int64_t row_stride,
                                      int64_t col_stride, const sky_query* d_queries, int32_t n_queries,
                                      int64_t max_total_rows, void* d_ws, size_t ws_bytes, int32_t* d_out_idx,
                                      int64_t out_capacity, int64_t* d_out_offsets, int32_t* d_query_status,
                                      void* stream)
{
    if (n_rows < 0 || n_rows >= (int64_t(1) << 31)) return bfail(SKY_ERR_INVALID_ARGUMENT, "n_rows outside [0, 2^31)");
    if (n_cols < 1 || n_cols > 32) return bfail(SKY_ERR_INVALID_ARGUMENT, "n_cols outside [1, 32]");
    if (n_queries < 0 || (n_queries > 0 && !d_queries)) return bfail(SKY_ERR_INVALID_ARGUMENT, "bad query array");
    if (max_total_rows < 0 || max_total_rows >= (int64_t(1) << 31))
        return bfail(SKY_ERR_INVALID_ARGUMENT, "max_total_rows outside [0, 2^31)");
    if (n_rows > 0 && !d_table) return bfail(SKY_ERR_INVALID_ARGUMENT, "NULL table");
    if (reinterpret_cast<uintptr_t>(d_table) & 3u) return bfail(SKY_ERR_INVALID_ARGUMENT, "table not 4-byte aligned");
    const bool row_major = col_stride == 1 && row_stride >= n_cols;
    const bool col_major = row_stride == 1 && col_stride >= n_rows;
    if (!row_major && !col_major)
        return bfail(SKY_ERR_INVALID_ARGUMENT, "strides must describe a row-major (col_stride 1) or "
                                               "column-major (row_stride 1) table");
    if (!d_out_offsets || (n_queries > 0 && !d_query_status) || out_capacity < 0 || (out_capacity > 0 && !d_out_idx))
        return bfail(SKY_ERR_INVALID_ARGUMENT, "bad output buffers");
    const size_t need = batched_device_workspace_bytes(n_cols, n_queries, max_total_rows);
    if (!d_ws || ws_bytes < need) return bfail(SKY_ERR_CAPACITY, "workspace needs %zu bytes", need);
    if ((reinterpret_cast<uintptr_t>(d_ws) & 255u) != 0)
        return bfail(SKY_ERR_INVALID_ARGUMENT, "workspace not 256-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (n_queries == 0) e = cudaMemsetAsync(d_out_offsets, 0, sizeof(int64_t), s);
    else e = launch_batched_device(d_table, n_rows, n_cols, row_stride, col_stride, d_queries, n_queries, max_total_rows,
                                   d_ws, ws_bytes, d_out_idx, out_capacity, d_out_offsets, d_query_status, s);
    if (e != cudaSuccess) return bfail(SKY_ERR_CUDA, "batched launch: %s", cudaGetErrorString(e));
    return SKY_OK;
}

}  // extern "C"
