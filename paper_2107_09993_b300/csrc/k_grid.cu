// k_grid.cu -- steps (a), (b), (c) of the skyline path (sm_103a).
//
//   k_minmax        per-dimension min / max and the finiteness check
//                   (normalisation for data outside the unit cube)
//   k_params        value -> column scales (Eq. 1), code and sort-key scales
//   k_map_mark      step (a)+(b): cell key of every point (Eq. 1) and the
//                   occupancy bitmap of the finest layer; streams the points
//                   through shared memory with 1-D bulk (TMA) copies
//   k_prefix_or_dim step (c): inclusive prefix-OR of the bitmap along one
//                   dimension; after all d dimensions, bit c holds "some
//                   occupied cell c' <= c componentwise"
//   k_dominated     materialises Def. 3's dominated bitmap for inspection
//   k_snap          pre-filter proposals -> real data points
//   k_survivors     step (c) output: rows whose cell is not dominated (and
//                   that no snapped proposal dominates), compacted in row
//                   order by a decoupled look-back scan, with a Morton key
//                   for the refinement's spatial sort
#include <cfloat>
#include <cstdint>

#include "sky_common.cuh"
#include "sky_internal.h"

namespace sky {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float scale_for(float levels, float range)
{
    if (range == 0.0f) return 0.0f;
    if (isinf(range)) return __fdiv_rn(levels, FLT_MAX);
    return __fdiv_rn(levels, range);
}

// Row loader: d floats of row r into x[0..DP), zero padded. Vector loads only
// when every row starts 16-byte aligned and holds exactly DP floats.
template <int DP>
__device__ __forceinline__ void load_row(const float* __restrict__ row, int d, bool vec4, float (&x)[DP])
{
    if (vec4) {
#pragma unroll
        for (int k = 0; k < DP; k += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(row + k));
            x[k] = v.x; x[k + 1] = v.y; x[k + 2] = v.z; x[k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < DP; ++k) x[k] = (k < d) ? __ldg(row + k) : 0.0f;
    }
}

// ---------------------------------------------------------------------------
template <int DP>
__global__ void __launch_bounds__(kThreads) k_minmax(const float* __restrict__ pts, int64_t n, int d,
                                                     int64_t ld, bool vec4, uint32_t* mm_min,
                                                     uint32_t* mm_max, uint32_t* err)
{
    float mn[DP], mx[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) { mn[k] = INFINITY; mx[k] = -INFINITY; }
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    constexpr int U = 4;  // rows in flight per thread
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
        float x[U][DP];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) load_row<DP>(pts + i * ld, d, vec4, x[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i0 + u * stride >= n) break;
#pragma unroll
            for (int k = 0; k < DP; ++k) {
                if (k < d) {
                    bad |= !isfinite(x[u][k]);
                    mn[k] = fminf(mn[k], x[u][k]);
                    mx[k] = fmaxf(mx[k], x[u][k]);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < DP; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[k] = fminf(mn[k], __shfl_xor_sync(kFull, mn[k], o));
            mx[k] = fmaxf(mx[k], __shfl_xor_sync(kFull, mx[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < DP; ++k) {
            if (k < d && mn[k] <= mx[k]) {
                atomicMin(&mm_min[k], float_to_ordered(mn[k]));
                atomicMax(&mm_max[k], float_to_ordered(mx[k]));
            }
        }
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, SKY_DEV_ERR_NONFINITE);
}

// params layout: [0,16) offset, [16,32) cell scale, [32,48) 7-bit code scale,
// [48,64) Morton scale. normalise = 0: unit cube (Eq. 1 as printed), 1: per
// dimension min/max from mm_min / mm_max.
__device__ __forceinline__ void write_params(int k, int d, int log2g, int mbits, bool normalise,
                                             const uint32_t* mm_min, const uint32_t* mm_max, float* params)
{
    float off = 0.0f, cs = 0.0f, qs = 0.0f, ms = 0.0f;
    if (k < d) {
        const float G = (float)(1u << log2g);
        const float M = (float)(1u << mbits);
        if (!normalise) {
            off = 0.0f; cs = G; qs = 128.0f; ms = M;
        } else {
            const float lo = ordered_to_float(mm_min[k]);
            const float hi = ordered_to_float(mm_max[k]);
            const float range = __fsub_rn(hi, lo);
            off = lo;
            cs = scale_for(G, range);
            qs = scale_for(128.0f, range);
            ms = scale_for(M, range);
        }
    }
    params[k] = off;
    params[16 + k] = cs;
    params[32 + k] = qs;
    params[48 + k] = ms;
}

__global__ void k_params(const uint32_t* mm_min, const uint32_t* mm_max, int d, int log2g, int mbits,
                         int normalise, float* params)
{
    const int k = threadIdx.x;
    if (k < kMaxDim) write_params(k, d, log2g, mbits, normalise != 0, mm_min, mm_max, params);
}

// Automatic map: keep the unit-cube map when every dimension's values lie in
// [0, 1] and span at least half of it; otherwise switch to min/max scales and
// ask for a second map pass (the first pass tracked min / max).
__global__ void k_decide(const uint32_t* mm_min, const uint32_t* mm_max, int d, int log2g, int mbits,
                         float* params, DevResult* res)
{
    __shared__ int s_bad;
    const int k = threadIdx.x;
    if (k == 0) s_bad = 0;
    __syncthreads();
    if (k < d) {
        const float lo = ordered_to_float(mm_min[k]);
        const float hi = ordered_to_float(mm_max[k]);
        const bool unit_ok = (lo >= 0.0f) && (hi <= 1.0f) && (__fsub_rn(hi, lo) >= 0.5f);
        if (!unit_ok) atomicOr(&s_bad, 1);
    }
    __syncthreads();
    const bool redo = s_bad != 0;
    if (redo && k < kMaxDim) write_params(k, d, log2g, mbits, true, mm_min, mm_max, params);
    if (k == 0) res->redo = redo ? 1u : 0u;
}

__global__ void k_clear_if(uint32_t* words, int64_t n, const DevResult* res)
{
    if (!res->redo) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        words[i] = 0u;
}

// Per-thread min / max accumulation, reduced and published once per block.
template <int DP>
struct MinMaxAcc {
    float mn[DP], mx[DP];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int k = 0; k < DP; ++k) { mn[k] = INFINITY; mx[k] = -INFINITY; }
    }
    __device__ __forceinline__ void add(const float (&x)[DP])
    {
#pragma unroll
        for (int k = 0; k < DP; ++k) { mn[k] = fminf(mn[k], x[k]); mx[k] = fmaxf(mx[k], x[k]); }
    }
    __device__ __forceinline__ void publish(int d, uint32_t* mm_min, uint32_t* mm_max)
    {
#pragma unroll
        for (int k = 0; k < DP; ++k) {
            for (int o = 16; o > 0; o >>= 1) {
                mn[k] = fminf(mn[k], __shfl_xor_sync(kFull, mn[k], o));
                mx[k] = fmaxf(mx[k], __shfl_xor_sync(kFull, mx[k], o));
            }
        }
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int k = 0; k < DP; ++k) {
                if (k < d && mn[k] <= mx[k]) {
                    atomicMin(&mm_min[k], float_to_ordered(mn[k]));
                    atomicMax(&mm_max[k], float_to_ordered(mx[k]));
                }
            }
        }
    }
};

// ---------------------------------------------------------------------------
// Steps (a)+(b). One point -> (cell key, Morton key) -> bit. The bitmap OR
// is fire-and-forget; when a whole warp hits one word (hot cells of
// correlated data) the bits are merged first and one lane issues it.
template <int DP>
__device__ __forceinline__ void map_one(const float (&x)[DP], int d, int log2g, int mbits, const float* s_off,
                                        const float* s_sc, const float* s_ms, int64_t row,
                                        uint2* __restrict__ keys, uint32_t* occ, bool& bad)
{
    const uint32_t G = 1u << log2g;
    const uint32_t M = 1u << mbits;
    uint32_t key = 0;
    uint32_t mq[DP];
#pragma unroll
    for (int k = DP - 1; k >= 0; --k) {
        mq[k] = 0;
        if (k < d) {
            bad |= !isfinite(x[k]);
            const uint32_t c = column_of(x[k], s_off[k], s_sc[k], G);
            key = (key << log2g) | c;
            // the Morton map is only for locality: reuse the cell column when
            // it is at least as fine
            mq[k] = (mbits <= log2g) ? (c >> (log2g - mbits)) : column_of(x[k], s_off[k], s_ms[k], M);
        }
    }
    uint32_t code = 0;
    for (int l = mbits - 1; l >= 0; --l)
#pragma unroll
        for (int k = DP - 1; k >= 0; --k)
            if (k < d) code = (code << 1) | ((mq[k] >> l) & 1u);
    keys[row] = make_uint2(key, code);
    const uint32_t word = key >> 5;
    const uint32_t bit = 1u << (key & 31u);
    const uint32_t am = __activemask();
    const int leader = __ffs(am) - 1;
    const uint32_t w0 = __shfl_sync(am, word, leader);
    if (__all_sync(am, word == w0)) {
        const uint32_t bits = __reduce_or_sync(am, bit);
        if ((int)(threadIdx.x & 31) == leader) atomicOr(occ + word, bits);
    } else {
        atomicOr(occ + word, bit);
    }
}

template <int DP>
__global__ void __launch_bounds__(kThreads) k_map_mark_plain(const float* __restrict__ pts, int64_t n,
                                                             int d, int64_t ld, bool vec4, int log2g, int mbits,
                                                             const float* params, uint2* keys,
                                                             uint32_t* occ, uint32_t* err, const DevResult* gate,
                                                             uint32_t* mm_min, uint32_t* mm_max)
{
    if (gate && !gate->redo) return;
    __shared__ float s_off[kMaxDim], s_sc[kMaxDim], s_ms[kMaxDim];
    if (threadIdx.x < kMaxDim) {
        s_off[threadIdx.x] = params[threadIdx.x];
        s_sc[threadIdx.x] = params[16 + threadIdx.x];
        s_ms[threadIdx.x] = params[48 + threadIdx.x];
    }
    __syncthreads();
    MinMaxAcc<DP> acc;
    acc.init();
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_round = ((n + 31) / 32) * 32;   // whole warps stay in the loop together
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        if (i < n) {
            float x[DP];
            load_row<DP>(pts + i * ld, d, vec4, x);
            map_one<DP>(x, d, log2g, mbits, s_off, s_sc, s_ms, i, keys, occ, bad);
            if (mm_min) acc.add(x);
        }
    }
    if (mm_min) acc.publish(d, mm_min, mm_max);
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, SKY_DEV_ERR_NONFINITE);
}

// Bulk-copy streaming version: rows are contiguous (ld == d) and the base is
// 16-byte aligned. Chunks of kThreads rows (kThreads*d*4 bytes, a multiple of
// 16) go through kStages shared-memory buffers; one thread issues the copies.
constexpr int kMapStages = 4;

template <int DP>
__global__ void __launch_bounds__(kThreads) k_map_mark_tma(const float* __restrict__ pts, int64_t n,
                                                           int d, int log2g, int mbits, const float* params,
                                                           uint2* keys, uint32_t* occ, uint32_t* err,
                                                           const DevResult* gate, uint32_t* mm_min, uint32_t* mm_max)
{
    if (gate && !gate->redo) return;
    extern __shared__ __align__(128) float s_buf[];  // [kMapStages][kThreads * d]
    __shared__ float s_off[kMaxDim], s_sc[kMaxDim], s_ms[kMaxDim];
    __shared__ __align__(8) uint64_t s_bar[kMapStages];
    const int tid = threadIdx.x;
    if (tid < kMaxDim) {
        s_off[tid] = params[tid];
        s_sc[tid] = params[16 + tid];
        s_ms[tid] = params[48 + tid];
    }
    if (tid == 0) {
        for (int s = 0; s < kMapStages; ++s) mbar_init(&s_bar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    const int64_t nfull = n / kThreads;
    const uint32_t chunk_bytes = (uint32_t)(kThreads * d * sizeof(float));
    const int64_t my_chunks = (nfull > blockIdx.x) ? (nfull - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    if (tid == 0) {
        for (int64_t i = 0; i < my_chunks && i < kMapStages; ++i) {
            const int64_t c = blockIdx.x + i * gridDim.x;
            mbar_arrive_expect_tx(&s_bar[i], chunk_bytes);
            bulk_g2s(s_buf + i * kThreads * d, pts + c * kThreads * d, chunk_bytes, &s_bar[i]);
        }
    }
    bool bad = false;
    bool timed_out = false;
    MinMaxAcc<DP> acc;
    acc.init();
    for (int64_t i = 0; i < my_chunks; ++i) {
        const int s = (int)(i % kMapStages);
        const uint32_t parity = (uint32_t)((i / kMapStages) & 1);
        if (!mbar_wait(&s_bar[s], parity, err)) { timed_out = true; }
        if (__syncthreads_or(timed_out)) {
            // Let every copy already issued land before the block exits.
            if (tid == 0) {
                for (int64_t j = i; j < my_chunks && j < i + kMapStages; ++j)
                    mbar_wait(&s_bar[j % kMapStages], (uint32_t)((j / kMapStages) & 1), nullptr);
            }
            __syncthreads();
            return;
        }
        const int64_t c = blockIdx.x + i * gridDim.x;
        const float* r = s_buf + s * kThreads * d + tid * d;
        float x[DP];
#pragma unroll
        for (int k = 0; k < DP; ++k) x[k] = (k < d) ? r[k] : 0.0f;
        map_one<DP>(x, d, log2g, mbits, s_off, s_sc, s_ms, c * kThreads + tid, keys, occ, bad);
        if (mm_min) acc.add(x);
        __syncthreads();  // every thread is done with stage s
        if (tid == 0 && i + kMapStages < my_chunks) {
            const int64_t c2 = blockIdx.x + (i + kMapStages) * gridDim.x;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar[s], chunk_bytes);
            bulk_g2s(s_buf + s * kThreads * d, pts + c2 * kThreads * d, chunk_bytes, &s_bar[s]);
        }
    }
    // Tail rows (fewer than one chunk): the last block loads them directly.
    if (blockIdx.x == gridDim.x - 1) {
        const int64_t i = nfull * kThreads + tid;
        if (i < n) {
            float x[DP];
            load_row<DP>(pts + i * d, d, false, x);
            map_one<DP>(x, d, log2g, mbits, s_off, s_sc, s_ms, i, keys, occ, bad);
            if (mm_min) acc.add(x);
        }
    }
    if (mm_min) acc.publish(d, mm_min, mm_max);
    if (__any_sync(kFull, bad) && (tid & 31) == 0) atomicOr(err, SKY_DEV_ERR_NONFINITE);
}

// ---------------------------------------------------------------------------
// One dimension of the prefix-OR over the whole grid (global memory).
__global__ void __launch_bounds__(kThreads) k_prefix_or_dim(uint32_t* R, int64_t words, int log2g, int k)
{
    prefix_or_dim(R, words, log2g, k, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                  (int64_t)gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(kThreads) k_dominated(const uint32_t* R, uint32_t* dom, int64_t words,
                                                        int log2g, int d)
{
    const uint32_t ones = ones_key(log2g, d);
    const int64_t total = 1ll << (log2g * d);
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t out = 0;
        for (int b = 0; b < 32; ++b) {
            const int64_t c = w * 32 + b;
            if (c >= total) break;
            if (!all_columns_positive((uint32_t)c, log2g, d)) continue;
            const uint32_t src = (uint32_t)c - ones;
            if ((R[src >> 5] >> (src & 31u)) & 1u) out |= 1u << b;
        }
        dom[w] = out;
    }
}

__global__ void __launch_bounds__(kThreads) k_cell_stats(const uint32_t* occ, const uint32_t* dom,
                                                         int64_t words, DevResult* res)
{
    uint32_t occ_c = 0, surv_c = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        occ_c += __popc(occ[w]);
        surv_c += __popc(occ[w] & ~dom[w]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        occ_c += __shfl_xor_sync(kFull, occ_c, o);
        surv_c += __shfl_xor_sync(kFull, surv_c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&res->occupied_cells, occ_c);
        atomicAdd(&res->surviving_cells, surv_c);
    }
}

// ---------------------------------------------------------------------------
// Pre-filter proposals. For proposal f_j, the data point q <= f_j (all
// dimensions) with the smallest binary32 coordinate sum, ties to the lower
// row, found by a packed 64-bit atomic min.
template <int DP>
__global__ void __launch_bounds__(kThreads) k_snap(const float* __restrict__ pts, int64_t n, int d,
                                                   int64_t ld, bool vec4, const float* __restrict__ prop,
                                                   int n_prop, unsigned long long* snap)
{
    __shared__ float s_f[16 * kMaxDim];
    for (int t = threadIdx.x; t < n_prop * d; t += blockDim.x) s_f[t] = prop[t];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_round = ((n + 31) / 32) * 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        const bool valid = i < n;
        float x[DP];
        float sum = 0.0f;
        if (valid) {
            load_row<DP>(pts + i * ld, d, vec4, x);
#pragma unroll
            for (int k = 0; k < DP; ++k)
                if (k < d) sum = __fadd_rn(sum, x[k]);
        }
        const unsigned long long packed =
            ((unsigned long long)float_to_ordered(sum) << 32) | (unsigned long long)(uint32_t)i;
        for (int j = 0; j < n_prop; ++j) {
            bool le = valid;
            if (valid) {
#pragma unroll
                for (int k = 0; k < DP; ++k)
                    if (k < d) le &= x[k] <= s_f[j * d + k];
            }
            if (__any_sync(kFull, le)) {
                unsigned long long v = le ? packed : ~0ull;
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long w = __shfl_xor_sync(kFull, v, o);
                    v = w < v ? w : v;
                }
                if ((threadIdx.x & 31) == 0) atomicMin(&snap[j], v);
            }
        }
    }
}

__global__ void k_snap_finalize(const float* __restrict__ pts, int d, int64_t ld,
                                const unsigned long long* snap, int n_prop, float* filt, DevResult* res)
{
    if (threadIdx.x != 0) return;
    int used = 0;
    for (int j = 0; j < n_prop; ++j) {
        if (snap[j] == ~0ull) continue;
        const int64_t row = (int64_t)(snap[j] & 0xffffffffull);
        for (int k = 0; k < kMaxDim; ++k) filt[used * kMaxDim + k] = (k < d) ? pts[row * ld + k] : 0.0f;
        ++used;
    }
    res->n_filter_used = (uint32_t)used;
}

// ---------------------------------------------------------------------------
// Survivors of step (c), compacted in row order, with their Morton keys
// (computed by the map pass). Reads only the 8-byte (cell key, Morton key)
// pairs; a row itself is read only when proposals are in use.
template <int DP>
__global__ void __launch_bounds__(kThreads) k_survivors(
    const float* __restrict__ pts, int64_t n, int d, int64_t ld, bool vec4, int log2g,
    const uint2* __restrict__ keys, const uint32_t* __restrict__ pre,
    const float* __restrict__ filt, int n_filter_max, DevResult* res, unsigned long long* states,
    uint32_t* tile_counter, uint32_t* surv_key, uint32_t* surv_idx)
{
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ float s_f[16 * kMaxDim];
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    const int nf = n_filter_max ? (int)res->n_filter_used : 0;
    for (int t = tid; t < nf * kMaxDim; t += kThreads) s_f[t] = filt[t];
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t ones = ones_key(log2g, d);
    const int64_t base = (int64_t)tile * kScanTile + (int64_t)tid * kScanItems;
    uint2 kk[kScanItems];
    if (base + kScanItems <= n) {
        const uint4* src = reinterpret_cast<const uint4*>(keys + base);
#pragma unroll
        for (int h = 0; h < kScanItems / 2; ++h) {
            const uint4 v = src[h];
            kk[2 * h] = make_uint2(v.x, v.y);
            kk[2 * h + 1] = make_uint2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) kk[j] = (base + j < n) ? keys[base + j] : make_uint2(0u, 0u);
    }
    // all bitmap words first (independent loads), then the tests
    uint32_t word[kScanItems];
    bool probe[kScanItems];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        probe[j] = (base + j < n) && all_columns_positive(kk[j].x, log2g, d);
        const uint32_t src = kk[j].x - ones;
        word[j] = probe[j] ? __ldg(pre + (src >> 5)) : 0u;
    }
    uint32_t flags = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + j;
        if (i >= n) continue;
        const uint32_t src = kk[j].x - ones;
        const bool dominated = probe[j] && ((word[j] >> (src & 31u)) & 1u);
        if (dominated) continue;
        if (nf) {
            float x[DP];
            load_row<DP>(pts + i * ld, d, vec4, x);
            bool filtered = false;
            for (int f = 0; f < nf && !filtered; ++f) {
                bool le = true, lt = false;
#pragma unroll
                for (int k = 0; k < DP; ++k) {
                    if (k < d) {
                        const float q = s_f[f * kMaxDim + k];
                        le &= q <= x[k];
                        lt |= q < x[k];
                    }
                }
                filtered = le && lt;  // Definition 1: the snapped point dominates x
            }
            if (filtered) continue;
        }
        flags |= 1u << j;
    }
    uint32_t total;
    const uint32_t excl = block_excl_scan((uint32_t)__popc(flags), s_warp, total);
    if (tid < 32) {
        const uint32_t prefix = lookback_prefix(states, tile, total, &res->err);
        if (tid == 0) s_prefix = prefix;
    }
    __syncthreads();
    uint32_t pos = s_prefix + excl;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (flags & (1u << j)) {
            surv_key[pos] = kk[j].y;
            surv_idx[pos] = (uint32_t)(base + j);
            ++pos;
        }
    }
    const uint32_t ntiles = (uint32_t)((n + kScanTile - 1) / kScanTile);
    if (tile == ntiles - 1 && tid == 0) res->survivors = s_prefix + total;
}

int grid_for(int64_t work, int per_block, int max_blocks)
{
    int64_t b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

int g_num_sms = 0;
int num_sms()
{
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return g_num_sms;
}

}  // namespace

#define SKY_DISPATCH_DP(d, ...)                                 \
    switch (pad4(d)) {                                          \
        case 4: { constexpr int DP = 4; __VA_ARGS__; } break;   \
        case 8: { constexpr int DP = 8; __VA_ARGS__; } break;   \
        case 12: { constexpr int DP = 12; __VA_ARGS__; } break; \
        default: { constexpr int DP = 16; __VA_ARGS__; } break; \
    }

static bool vec4_ok(const Plan& p)
{
    return (p.d % 4 == 0) && (p.ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(p.pts) & 15u) == 0);
}

static cudaError_t launch_map(const Plan& p, const DevResult* gate, bool track, cudaStream_t s)
{
    uint32_t* mn = track ? p.mm_min : nullptr;
    uint32_t* mx = track ? p.mm_max : nullptr;
    if (p.tma_ok && p.n >= kThreads) {
        const size_t smem = (size_t)kMapStages * kThreads * p.d * sizeof(float);
        const int64_t nchunks = p.n / kThreads;
        const int blocks = grid_for(nchunks, 1, num_sms() * 4);
        SKY_DISPATCH_DP(p.d, {
            static bool attr_set = false;
            if (!attr_set) {
                cudaFuncSetAttribute(k_map_mark_tma<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kMapStages * kThreads * 16 * (int)sizeof(float));
                attr_set = true;
            }
            k_map_mark_tma<DP><<<blocks, kThreads, smem, s>>>(p.pts, p.n, p.d, p.log2g, p.morton_bits, p.params,
                                                              p.keys, p.occ, &p.res->err, gate, mn, mx);
        });
    } else {
        const int blocks = grid_for(p.n, kThreads * 4, num_sms() * 8);
        const bool v = vec4_ok(p);
        SKY_DISPATCH_DP(p.d, k_map_mark_plain<DP><<<blocks, kThreads, 0, s>>>(
                                 p.pts, p.n, p.d, p.ld, v, p.log2g, p.morton_bits, p.params, p.keys, p.occ,
                                 &p.res->err, gate, mn, mx));
    }
    return cudaGetLastError();
}

cudaError_t launch_build(const Plan& p, cudaStream_t s)
{
    cudaMemsetAsync(p.occ, 0, sizeof(uint32_t) * p.words, s);
    if (p.map_mode != kMapUnit) {
        cudaMemsetAsync(p.mm_min, 0xff, sizeof(uint32_t) * kMaxDim, s);
        cudaMemsetAsync(p.mm_max, 0x00, sizeof(uint32_t) * kMaxDim, s);
    }
    if (p.n == 0) return cudaGetLastError();
    if (p.map_mode == kMapMinMax) {
        const int blocks = grid_for(p.n, kThreads * 8, num_sms() * 8);
        const bool v = vec4_ok(p);
        SKY_DISPATCH_DP(p.d, k_minmax<DP><<<blocks, kThreads, 0, s>>>(p.pts, p.n, p.d, p.ld, v, p.mm_min,
                                                                       p.mm_max, &p.res->err));
        k_params<<<1, 32, 0, s>>>(p.mm_min, p.mm_max, p.d, p.log2g, p.morton_bits, 1, p.params);
        return launch_map(p, nullptr, false, s);
    }
    k_params<<<1, 32, 0, s>>>(p.mm_min, p.mm_max, p.d, p.log2g, p.morton_bits, 0, p.params);
    if (p.map_mode == kMapUnit) return launch_map(p, nullptr, false, s);
    // automatic: unit map with min/max tracking, then a gated second pass
    launch_map(p, nullptr, true, s);
    k_decide<<<1, 32, 0, s>>>(p.mm_min, p.mm_max, p.d, p.log2g, p.morton_bits, p.params, p.res);
    k_clear_if<<<grid_for(p.words, kThreads, num_sms() * 4), kThreads, 0, s>>>(p.occ, p.words, p.res);
    return launch_map(p, p.res, false, s);
}

int build_kernel_count(const Plan& p)
{
    if (p.n == 0) return 0;
    if (p.map_mode == kMapMinMax) return 3;
    if (p.map_mode == kMapUnit) return 2;
    return 5;
}

cudaError_t launch_prefix_or(const Plan& p, cudaStream_t s)
{
    cudaMemcpyAsync(p.pre, p.occ, sizeof(uint32_t) * p.words, cudaMemcpyDeviceToDevice, s);
    for (int k = 0; k < p.d; ++k) {
        const int blocks = grid_for(p.words, kThreads, num_sms() * 8);
        k_prefix_or_dim<<<blocks, kThreads, 0, s>>>(p.pre, p.words, p.log2g, k);
    }
    return cudaGetLastError();
}

cudaError_t launch_dominated(const Plan& p, cudaStream_t s)
{
    const int blocks = grid_for(p.words, kThreads, num_sms() * 8);
    k_dominated<<<blocks, kThreads, 0, s>>>(p.pre, p.dom, p.words, p.log2g, p.d);
    k_cell_stats<<<blocks, kThreads, 0, s>>>(p.occ, p.dom, p.words, p.res);
    return cudaGetLastError();
}

cudaError_t launch_snap(const Plan& p, const float* d_prop, int n_prop, cudaStream_t s)
{
    cudaMemsetAsync(p.snap, 0xff, sizeof(unsigned long long) * 16, s);
    if (n_prop > 0 && p.n > 0) {
        const int blocks = grid_for(p.n, kThreads * 4, num_sms() * 8);
        const bool v = vec4_ok(p);
        SKY_DISPATCH_DP(p.d, k_snap<DP><<<blocks, kThreads, 0, s>>>(p.pts, p.n, p.d, p.ld, v, d_prop, n_prop,
                                                                     p.snap));
    }
    k_snap_finalize<<<1, 32, 0, s>>>(p.pts, p.d, p.ld, p.snap, n_prop, p.filt, p.res);
    return cudaGetLastError();
}

cudaError_t launch_survivors(const Plan& p, int n_filter, cudaStream_t s)
{
    if (p.n == 0) return cudaGetLastError();
    const int64_t ntiles = (p.n + kScanTile - 1) / kScanTile;
    cudaMemsetAsync(p.lb_states, 0, sizeof(unsigned long long) * ntiles, s);
    cudaMemsetAsync(p.lb_counter, 0, sizeof(uint32_t), s);
    const bool v = vec4_ok(p);
    SKY_DISPATCH_DP(p.d, k_survivors<DP><<<(unsigned)ntiles, kThreads, 0, s>>>(
                             p.pts, p.n, p.d, p.ld, v, p.log2g, p.keys, p.pre, p.filt, n_filter, p.res,
                             p.lb_states, p.lb_counter, p.surv_key, p.surv_idx));
    return cudaGetLastError();
}

cudaError_t launch_cell_stats(const Plan& p, cudaStream_t s)
{
    return launch_dominated(p, s);
}

int auto_log2g(int64_t n, int d)
{
    int r = 24 / d;
    if (r < 1) r = 1;
    if (r > 16) r = 16;
    while (r > 1 && (double)(1ull << (r * d)) > 32.0 * (double)(n > 1 ? n : 1)) --r;
    return r;
}

// Bits per dimension of the Morton sort key: about log2(n) + 6 bits in all
// (never above 32), so that the sort resolves point neighbourhoods without
// spending radix passes on empty precision.
int morton_bits_for(int64_t n, int d)
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

}  // namespace sky
