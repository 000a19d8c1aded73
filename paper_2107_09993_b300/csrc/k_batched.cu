// k_batched.cu -- many skylines (row ranges x attribute subsets of one table)
// in one CUDA-graph launch (sm_103a).
//
// Every phase of the single-set path runs once for the whole batch: each
// kernel walks a flat list of (query, block) work items, found from per-query
// prefix counts by binary search, so small and large queries share the same
// launches. The refinement is a persistent kernel per padded dimension class
// that pulls (query, p-tile) items from a global counter, largest queries
// first, and runs the same per-tile refinement as the single-set kernel.
// Look-back scans stay inside one query (its tiles are claimed in order).
//
// The value -> column map is Eq. 1 on the unit cube with clamping (exact for
// any finite data; pruning is best for data in [0,1]).
#include <algorithm>
#include <cstdint>

#include "sky_common.cuh"
#include "sky_internal.h"
#include "sky_refine.cuh"
#include "sky_sort.cuh"

namespace sky {
namespace batched {

constexpr int kT = 256;
constexpr int kChunk = kScanTile;           // 2048 rows: map, survivors, sort and emit blocks
static_assert(kChunk == kSortTile, "survivor and sort blocks share one granularity");
using refine::kTQ;
using refine::kSubSlots;

// Query of flat item `item` given the exclusive prefix of per-query counts.
__device__ __forceinline__ int find_query(const int64_t* prefix, int nq, int64_t item)
{
    int lo = 0, hi = nq;  // prefix[lo] <= item < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ float elem(const QueryPlan& q, int64_t r, int k)
{
    return __ldg(q.base + r * q.rs + (int64_t)q.col[k] * q.cs);
}

// Key of a row outside a quadrant query's quadrant (batched grids have at
// most 2^18 cells, so no cell key reaches it).
constexpr uint32_t kOutsideKey = 0xffffffffu;

// ---------------------------------------------------------------- (a)+(b)
// A count of work items passed as -1 is read from the prefix array (a batch
// planned on the device, whose counts the host does not know); the grids of
// such launches are sized by bounds and blocks past the count exit at once.
__device__ __forceinline__ int64_t items_of(const int64_t* prefix, int nq, int64_t nitems)
{
    return nitems >= 0 ? nitems : prefix[nq];
}

__global__ void __launch_bounds__(kT) kb_map(const QueryPlan* __restrict__ qps, int nq,
                                             const int64_t* __restrict__ pchunk, int64_t nitems)
{
    nitems = items_of(pchunk, nq, nitems);
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int qi = find_query(pchunk, nq, item);
        const QueryPlan& q = qps[qi];
        const int64_t r0 = (item - pchunk[qi]) * kChunk;
        const uint32_t G = 1u << q.log2g, M = 1u << q.mbits;
        const float sc = (float)G, sm = (float)M;
        bool bad = false;
        for (int64_t r = r0 + threadIdx.x; r < r0 + kChunk && r < q.n; r += kT) {
            uint32_t key = 0, mq[kMaxDim];
            bool outside = false;   // quadrant query: below the origin in some column
#pragma unroll
            for (int k = kMaxDim - 1; k >= 0; --k) {
                mq[k] = 0;
                if (k < q.d) {
                    const float x = elem(q, r, k);
                    bad |= !isfinite(x);
                    outside |= q.quadrant && !(x >= q.origin[k]);
                    const uint32_t c = column_of(x, 0.0f, sc, G);
                    key = (key << q.log2g) | c;
                    mq[k] = (q.mbits <= q.log2g) ? (c >> (q.log2g - q.mbits)) : column_of(x, 0.0f, sm, M);
                }
            }
            uint32_t code = 0;
            for (int l = q.mbits - 1; l >= 0; --l)
#pragma unroll
                for (int k = kMaxDim - 1; k >= 0; --k)
                    if (k < q.d) code = (code << 1) | ((mq[k] >> l) & 1u);
            if (outside) {
                // takes no part: marks no cell and never survives step (c)
                q.keys[r] = make_uint2(kOutsideKey, code);
                continue;
            }
            q.keys[r] = make_uint2(key, code);
            atomicOr(q.occ + (key >> 5), 1u << (key & 31u));
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&q.res->err, SKY_DEV_ERR_NONFINITE);
    }
}

// One CTA per query: the d prefix-OR passes in shared memory.
__global__ void __launch_bounds__(512) kb_prefix(const QueryPlan* __restrict__ qps)
{
    extern __shared__ uint32_t s_words[];
    const QueryPlan& q = qps[blockIdx.x];
    if (q.n == 0) return;
    for (int64_t w = threadIdx.x; w < q.words; w += blockDim.x) s_words[w] = q.occ[w];
    __syncthreads();
    for (int k = 0; k < q.d; ++k) {
        prefix_or_dim(s_words, q.words, q.log2g, k, threadIdx.x, blockDim.x);
        __syncthreads();
    }
    for (int64_t w = threadIdx.x; w < q.words; w += blockDim.x) q.pre[w] = s_words[w];
}

// -------------------------------------------------------------------- (c)
__global__ void __launch_bounds__(kT) kb_survivors(const QueryPlan* __restrict__ qps, int nq,
                                                   const int64_t* __restrict__ pchunk, uint32_t* claim)
{
    __shared__ uint32_t s_warp[kT / 32];
    __shared__ uint32_t s_prefix;
    __shared__ int64_t s_item;
    if (threadIdx.x == 0) s_item = atomicAdd(claim, 1u);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= pchunk[nq]) return;
    const int qi = find_query(pchunk, nq, item);
    const QueryPlan& q = qps[qi];
    const uint32_t tile = (uint32_t)(item - pchunk[qi]);
    const uint32_t ones = ones_key(q.log2g, q.d);
    const int64_t base = (int64_t)tile * kChunk + (int64_t)threadIdx.x * kScanItems;
    uint32_t flags = 0, mk[kScanItems];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + j;
        mk[j] = 0;
        if (i >= q.n) continue;
        const uint2 kk = q.keys[i];
        mk[j] = kk.y;
        if (kk.x == kOutsideKey) continue;   // outside the query's quadrant
        bool dominated = false;
        if (all_columns_positive(kk.x, q.log2g, q.d)) {
            const uint32_t src = kk.x - ones;
            dominated = (q.pre[src >> 5] >> (src & 31u)) & 1u;
        }
        if (!dominated) flags |= 1u << j;
    }
    uint32_t total;
    const uint32_t excl = block_excl_scan<kT>((uint32_t)__popc(flags), s_warp, total);
    if (threadIdx.x < 32) {
        const uint32_t prefix = lookback_prefix(q.lb_a, tile, total, &q.res->err);
        if (threadIdx.x == 0) s_prefix = prefix;
    }
    __syncthreads();
    uint32_t pos = s_prefix + excl;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (flags & (1u << j)) {
            q.surv_key[pos] = mk[j];
            q.surv_idx[pos] = (uint32_t)(base + j);
            ++pos;
        }
    }
    if (tile == q.chunks - 1 && threadIdx.x == 0) q.res->survivors = s_prefix + total;
}

// ------------------------------------------------------------------- sort
__device__ __forceinline__ void pass_buffers(const QueryPlan& q, int ps, const uint32_t*& kin,
                                             const uint32_t*& vin, uint32_t*& kout, uint32_t*& vout)
{
    const bool even = (ps & 1) == 0;
    kin = even ? q.surv_key : q.key2;
    vin = even ? q.surv_idx : q.val2;
    kout = even ? q.key2 : q.surv_key;
    vout = even ? q.val2 : q.surv_idx;
}

__global__ void __launch_bounds__(kT) kb_radix_hist(const QueryPlan* __restrict__ qps, int nq,
                                                    const int64_t* __restrict__ pchunk, int ps)
{
    const int64_t item = blockIdx.x;
    if (item >= pchunk[nq]) return;
    const int qi = find_query(pchunk, nq, item);
    const QueryPlan& q = qps[qi];
    if (ps >= q.passes) return;
    const uint32_t* kin; const uint32_t* vin; uint32_t* kout; uint32_t* vout;
    pass_buffers(q, ps, kin, vin, kout, vout);
    radix::radix_hist_block(kin, q.res->survivors, 8 * ps, q.hist, q.chunks, q.digit_total + 256 * ps,
                            (uint32_t)(item - pchunk[qi]));
}

// One CTA per query; thread t owns digit t and walks its row of blocks.
__global__ void __launch_bounds__(256) kb_radix_scan(const QueryPlan* __restrict__ qps, int ps)
{
    __shared__ uint32_t s_warp[8];
    const QueryPlan& q = qps[blockIdx.x];
    if (ps >= q.passes || q.n == 0) return;
    const uint32_t m = q.res->survivors;
    const int64_t nblk = ((int64_t)m + kChunk - 1) / kChunk;
    uint32_t total;
    uint32_t off = block_excl_scan<256>(q.digit_total[256 * ps + threadIdx.x], s_warp, total);
    uint32_t* row = q.hist + (int64_t)threadIdx.x * q.chunks;
    for (int64_t b = 0; b < nblk; ++b) {
        const uint32_t v = row[b];
        row[b] = off;
        off += v;
    }
}

__global__ void __launch_bounds__(kT) kb_radix_scatter(const QueryPlan* __restrict__ qps, int nq,
                                                       const int64_t* __restrict__ pchunk, int ps)
{
    const int64_t item = blockIdx.x;
    if (item >= pchunk[nq]) return;
    const int qi = find_query(pchunk, nq, item);
    const QueryPlan& q = qps[qi];
    if (ps >= q.passes) return;
    const uint32_t* kin; const uint32_t* vin; uint32_t* kout; uint32_t* vout;
    pass_buffers(q, ps, kin, vin, kout, vout);
    radix::radix_scatter_block(kin, vin, kout, vout, q.res->survivors, 8 * ps, q.hist, q.chunks,
                               (uint32_t)(item - pchunk[qi]));
}

// ----------------------------------------------------------------- layout
// Survivors of one query in Morton order: coordinates padded to dp, 7-bit
// codes, local row ids, sub-tile and tile minimum codes.
__global__ void __launch_bounds__(kTQ) kb_gather(const QueryPlan* __restrict__ qps, int nq,
                                                 const int64_t* __restrict__ ptile)
{
    __shared__ uint32_t s_sub[kTQ / 32][4];
    const int64_t item = blockIdx.x;
    if (item >= ptile[nq]) return;
    const int qi = find_query(ptile, nq, item);
    const QueryPlan& q = qps[qi];
    const uint32_t t = (uint32_t)(item - ptile[qi]);
    const uint32_t m = q.res->survivors;
    if (t >= (m + kTQ - 1) / kTQ) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int dp = q.dp, dw = dp / 4;
    const int64_t j = (int64_t)t * kTQ + tid;
    const bool valid = j < m;
    const uint32_t* sorted = (q.passes & 1) ? q.val2 : q.surv_idx;
    const uint32_t row = valid ? sorted[j] : 0u;
    float x[kMaxDim];
    uint32_t code[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < kMaxDim; ++k) {
        x[k] = 0.0f;
        if (k < dp) {
            uint32_t c = 127u;
            if (valid) {
                c = 0u;
                if (k < q.d) {
                    x[k] = elem(q, row, k);
                    c = column_of(x[k], 0.0f, 128.0f, 128u);
                }
            } else {
                x[k] = INFINITY;
            }
            code[k / 4] |= c << (8 * (k % 4));
        }
    }
#pragma unroll
    for (int k = 0; k < kMaxDim; k += 4)
        if (k < dp)
            *reinterpret_cast<float4*>(q.X + j * dp + k) = make_float4(x[k], x[k + 1], x[k + 2], x[k + 3]);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        if (w < dw) {
            q.C[j * dw + w] = code[w];
            uint32_t c = code[w];
            for (int o = 16; o > 0; o >>= 1) c = __vminu4(c, __shfl_xor_sync(kFull, c, o));
            if (lane == 0) {
                q.sub[((int64_t)t * kSubSlots + warp) * dw + w] = c;
                s_sub[warp][w] = c;
            }
        }
    }
    q.ids[j] = valid ? (int32_t)row : -1;
    // threshold masks of this warp's 32-point sub-tile for the mask probe
    // (dp >= 12): word k * 8 + l = the lanes whose 3-bit code in dimension k
    // is <= l (dimensions past dp: code 0; padding points: code 127)
    if (q.tmask != nullptr) {
        uint32_t v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t c3 = (code[k >> 2] >> (8 * (k & 3) + 4)) & 7u;
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                const uint32_t b = l == 7 ? kFull : __ballot_sync(kFull, c3 <= (uint32_t)l);
                const int e = k * 8 + l;
                if (lane == (e & 31)) v[e >> 5] = b;
            }
        }
        uint32_t* o = q.tmask + ((int64_t)t * (kTQ / 32) + warp) * 128;
#pragma unroll
        for (int r = 0; r < 4; ++r) o[r * 32 + lane] = v[r];
    }
    // layer-1 cell index of the query (zeroed with the query's counters): per
    // cell (bit k: code k >= 64), ~first and last + 1 of the tiles holding
    // one of its points; one update per distinct cell of a warp
    {
        uint32_t cell = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (w < dw) cell |= refine::cell_bits4(code[w]) << (4 * w);
        const uint32_t peers = __match_any_sync(kFull, valid ? cell : 0xffffffffu);
        if (valid && lane == __ffs(peers) - 1) {
            atomicMax(q.cidx + cell, ~t);
            atomicMax(q.cidx + (1u << q.d) + cell, t + 1u);
        }
    }
    __syncthreads();
    if (tid < dw) {
        uint32_t c = s_sub[0][tid];
        for (int w = 1; w < kTQ / 32; ++w) c = __vminu4(c, s_sub[w][tid]);
        q.sub[((int64_t)t * kSubSlots + kTQ / 32) * dw + tid] = c;
    }
    // the last q-tile whose first Morton key is <= this tile's last key (a
    // dominator never sorts after its victim); warp 0, ties in rounds of 32
    if (warp == 0) {
        const uint32_t* skeys = (q.passes & 1) ? q.key2 : q.surv_key;
        const uint32_t T = (m + kTQ - 1) / kTQ;
        const uint32_t last = skeys[min((int64_t)m, ((int64_t)t + 1) * kTQ) - 1];
        uint32_t e = t;
        while (true) {
            const uint32_t tn = e + 1 + lane;
            const bool tie = tn < T && skeys[(int64_t)tn * kTQ] <= last;
            const uint32_t run = __ballot_sync(kFull, !tie);
            const uint32_t k = run ? (uint32_t)(__ffs(run) - 1) : 32u;
            e += k;
            if (k < 32u) break;
        }
        if (lane == 0) q.tend[t] = e;
    }
}

// Super-tile minima: the byte-wise minimum code of each run of 32 q-tiles of
// a query (the refinement skips a super-tile whose minimum is out of every
// live group's reach). One warp per tile item; the warps of the first tile of
// each run do the work.
__global__ void __launch_bounds__(256) kb_supmin(const QueryPlan* __restrict__ qps, int nq,
                                                 const int64_t* __restrict__ ptile, int64_t items)
{
    const int lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (item >= items_of(ptile, nq, items)) return;
    const int qi = find_query(ptile, nq, item);
    const QueryPlan& q = qps[qi];
    const uint32_t t0 = (uint32_t)(item - ptile[qi]);
    if (t0 & 31u) return;
    const uint32_t m = q.res->survivors;
    const uint32_t T = (m + kTQ - 1) / kTQ;
    if (t0 >= T) return;
    const int dw = q.dp / 4;
    for (int w = 0; w < dw; ++w) {
        const uint32_t t = t0 + (uint32_t)lane;
        uint32_t c = t < T ? q.sub[((int64_t)t * kSubSlots + kTQ / 32) * dw + w] : 0x7f7f7f7fu;
        for (int o = 16; o > 0; o >>= 1) c = __vminu4(c, __shfl_xor_sync(kFull, c, o));
        if (lane == 0) q.supmin[(int64_t)(t0 / 32u) * dw + w] = c;
    }
}

// -------------------------------------------------------------------- (d)
// Persistent CTAs per SM by padded dimension (the launch bound caps the
// registers: 8 -> 48, 7 -> 56, 6 -> 64, 5 -> 72 per thread; 1 leaves the
// choice to the compiler). Measured on the 4,096-query launch: 539 ms with
// 8 / 8 / 8 / compiler's choice (91 registers at d = 16), 526 ms with
// 8 / 8 / 7 / 6.
#ifndef SKY_BATCH_MINB_4
#define SKY_BATCH_MINB_4 8
#endif
#ifndef SKY_BATCH_MINB_8
#define SKY_BATCH_MINB_8 8
#endif
#ifndef SKY_BATCH_MINB_12
#define SKY_BATCH_MINB_12 7
#endif
#ifndef SKY_BATCH_MINB_16
#define SKY_BATCH_MINB_16 6
#endif
template <int DP>
struct BatchMinBlocks {
    static constexpr int value = DP == 4 ? SKY_BATCH_MINB_4
                               : DP == 8 ? SKY_BATCH_MINB_8
                               : DP == 12 ? SKY_BATCH_MINB_12 : SKY_BATCH_MINB_16;
};

// 1: the batched refinement also finishes p-tiles with few live points in
// sparse mode and keeps the producer's group maxima in registers, like the
// single-set kernel; 0: ring to the end, maxima in shared memory
#ifndef SKY_BATCH_SPARSE
#define SKY_BATCH_SPARSE 0
#endif
constexpr bool kBatchSparse = SKY_BATCH_SPARSE != 0;

// S: ring stages; FAST: fast-code list probe (both chosen per padded-
// dimension class at launch time, e.g. by the autotuner).
// d_class (a batch planned on the device): the class's first item and item
// count are d_class[cls] and d_class[4 + cls] instead of `items` / `nitems`.
// The mask probe of the single-set refinement in the batched kernel: from
// padded dimension 12 (masks and codes staged at 12, masks only at 16; the
// queries' threshold masks are written by kb_gather)
#ifndef SKY_BATCH_MASK_MIN_DP
#define SKY_BATCH_MASK_MIN_DP 12
#endif
template <int DP>
struct BatchMask {
    static constexpr int value = (DP < 12 || DP < SKY_BATCH_MASK_MIN_DP) ? 0 : DP == 16 ? 2 : 1;
};

template <int DP, int S, bool FAST>
__global__ void __launch_bounds__(kTQ + 32, BatchMinBlocks<DP>::value) kb_refine(const QueryPlan* __restrict__ qps,
                                                      const int2* __restrict__ items, int nitems, uint32_t* claim,
                                                      const int* __restrict__ d_class, int cls)
{
    extern __shared__ __align__(256) unsigned char smem_raw[];   // the mask probe's tables are 256-byte aligned
    using SM = refine::RefineSmem<DP, S, FAST, kTQ / 32, BatchMask<DP>::value>;
    SM& sm = *reinterpret_cast<SM*>(smem_raw);
    __shared__ int s_item;
    if (d_class) {
        items += d_class[cls];
        nitems = d_class[4 + cls];
    }
    while (true) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(claim, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const int2 w = items[it];
        const QueryPlan& q = qps[w.x];
        const uint32_t m = q.res->survivors;
        if ((uint32_t)w.y < (m + kTQ - 1) / kTQ)
            refine::refine_ptile<DP, kBatchSparse, false, SM>(sm, q.X, q.C, q.ids, q.sub, q.tend, q.supmin, m,
                                                              (uint32_t)w.y, q.res, q.keep, nullptr, q.cidx,
                                                              q.cidx + (1u << q.d), q.tmask);
    }
}

__global__ void __launch_bounds__(kT) kb_emit(const QueryPlan* __restrict__ qps, int nq,
                                              const int64_t* __restrict__ pchunk, uint32_t* claim)
{
    __shared__ uint32_t s_warp[kT / 32];
    __shared__ uint32_t s_prefix;
    __shared__ int64_t s_item;
    if (threadIdx.x == 0) s_item = atomicAdd(claim, 1u);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= pchunk[nq]) return;
    const int qi = find_query(pchunk, nq, item);
    const QueryPlan& q = qps[qi];
    const uint32_t tile = (uint32_t)(item - pchunk[qi]);
    const int64_t base = (int64_t)tile * kChunk + (int64_t)threadIdx.x * kScanItems;
    uint32_t flags = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < q.n && q.keep[base + j]) flags |= 1u << j;
    uint32_t total;
    const uint32_t excl = block_excl_scan<kT>((uint32_t)__popc(flags), s_warp, total);
    if (threadIdx.x < 32) {
        const uint32_t prefix = lookback_prefix(q.lb_b, tile, total, &q.res->err);
        if (threadIdx.x == 0) s_prefix = prefix;
    }
    __syncthreads();
    uint32_t pos = s_prefix + excl;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (flags & (1u << j)) q.stage[pos++] = (int32_t)(q.row_begin + base + j);
    if (tile == q.chunks - 1 && threadIdx.x == 0) q.res->count = s_prefix + total;
}

// Output offsets (exclusive scan of the counts in query order) and status.
__global__ void __launch_bounds__(1024) kb_finish(const QueryPlan* __restrict__ qps, int nq, int64_t capacity,
                                                  int64_t* offsets, int32_t* status)
{
    __shared__ int64_t s_part[1024];
    const int per = (nq + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(nq, lo + per);
    int64_t sum = 0;
    for (int q = lo; q < hi; ++q) sum += qps[q].n ? qps[q].res->count : 0;
    s_part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int64_t v = threadIdx.x >= (unsigned)o ? s_part[threadIdx.x - o] : 0;
        __syncthreads();
        s_part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = s_part[threadIdx.x] - sum;
    for (int q = lo; q < hi; ++q) {
        const QueryPlan& p = qps[q];
        const int64_t c = p.n ? p.res->count : 0;
        offsets[q] = run;
        const uint32_t err = p.n ? p.res->err : 0u;
        int32_t st = 0;                                   // SKY_OK
        if (p.invalid) {   // planned on the device: a bad query, or beyond the workspace bound
            status[q] = p.invalid == 1 ? 1 : 6;          // SKY_ERR_INVALID_ARGUMENT / SKY_ERR_TOO_LARGE
            continue;
        }
        if (err & SKY_DEV_ERR_NONFINITE) st = 2;          // SKY_ERR_NONFINITE
        else if (err & SKY_DEV_ERR_TIMEOUT) st = 7;       // SKY_ERR_TIMEOUT
        else if (run + c > capacity) st = 3;              // SKY_ERR_CAPACITY
        status[q] = st;
        run += c;
    }
    if (threadIdx.x == 1023) offsets[nq] = s_part[1023];
}

__global__ void __launch_bounds__(kT) kb_copy(const QueryPlan* __restrict__ qps, int nq,
                                              const int64_t* __restrict__ pchunk, int64_t nitems,
                                              const int64_t* __restrict__ offsets, int32_t* out, int64_t capacity)
{
    nitems = items_of(pchunk, nq, nitems);
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int qi = find_query(pchunk, nq, item);
        const QueryPlan& q = qps[qi];
        const int64_t c = q.res->count;
        const int64_t off = offsets[qi];
        const int64_t i0 = (item - pchunk[qi]) * kChunk;
        for (int64_t i = i0 + threadIdx.x; i < i0 + kChunk && i < c; i += kT)
            if (off + i < capacity) out[off + i] = q.stage[i];
    }
}

}  // namespace batched

// ============================================================ host side ===
namespace {

int sm_count()
{
    int dev = 0, n = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
}

template <int DP, int S, bool FAST>
cudaError_t launch_kb_refine_v(const QueryPlan* qps, const int2* items, int nitems, uint32_t* claim, int ctas_per_sm,
                               const int* d_class, int cls, cudaStream_t s)
{
    auto* kern = batched::kb_refine<DP, S, FAST>;
    const int smem = (int)sizeof(refine::RefineSmem<DP, S, FAST, refine::kTQ / 32, batched::BatchMask<DP>::value>);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    int resident = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kern, refine::kTQ + 32, smem);
    if (resident < 1) resident = 1;
    const int per_sm = (ctas_per_sm <= 0 || ctas_per_sm > resident) ? resident : ctas_per_sm;
    int grid = sm_count() * per_sm;
    if (grid > nitems) grid = nitems;   // device-planned: nitems is the bound
    if (grid < 1) return cudaSuccess;
    kern<<<grid, refine::kTQ + 32, smem, s>>>(qps, items, nitems, claim, d_class, cls);
    return cudaGetLastError();
}

// The refinement variant of one padded-dimension class: ring depth 4 or 8
// (other values: 8), fast codes on or off.
// Ring depth of the classes with the mask probe (0: the tuned or default
// depth, 4 or 8); their stages hold masks as well, so a shallow ring keeps
// the persistent CTAs resident. Measured on B300 (4,096-query launch, ms):
// list probe 519.6; mask probe with the tuned depths (8 for d = 9-12)
// 477.0, depth 6 447.4, depth 4 430.4. With a fixed depth the autotuner's
// depth knob applies to the classes below padded dimension 12 only.
#ifndef SKY_BATCH_MASK_STAGES
#define SKY_BATCH_MASK_STAGES 4
#endif
template <int DP>
cudaError_t launch_kb_refine(const QueryPlan* qps, const int2* items, int nitems, uint32_t* claim, int ctas_per_sm,
                             int stages, bool fast, const int* d_class, int cls, cudaStream_t s)
{
    if constexpr (batched::BatchMask<DP>::value != 0 && SKY_BATCH_MASK_STAGES != 0) {
        static_assert(SKY_BATCH_MASK_STAGES >= 2 && SKY_BATCH_MASK_STAGES <= 12, "a ring of 2 to 12 stages");
        return launch_kb_refine_v<DP, SKY_BATCH_MASK_STAGES, (DP >= SKY_REFINE_FAST_MIN_DP)>(
            qps, items, nitems, claim, ctas_per_sm, d_class, cls, s);
    }
    if (stages == 4)
        return fast ? launch_kb_refine_v<DP, 4, true>(qps, items, nitems, claim, ctas_per_sm, d_class, cls, s)
                    : launch_kb_refine_v<DP, 4, false>(qps, items, nitems, claim, ctas_per_sm, d_class, cls, s);
    return fast ? launch_kb_refine_v<DP, 8, true>(qps, items, nitems, claim, ctas_per_sm, d_class, cls, s)
                : launch_kb_refine_v<DP, 8, false>(qps, items, nitems, claim, ctas_per_sm, d_class, cls, s);
}

}  // namespace

cudaError_t launch_batched(const BatchLaunch& b, cudaStream_t s)
{
    using namespace batched;
    // a batch planned on the device passes bounds as counts; the kernels read
    // the actual counts (-1 below) and its planner has zeroed its arrays
    const bool dev = b.d_class != nullptr;
    if (!dev) cudaMemsetAsync(b.zero_base, 0, b.zero_bytes, s);
    if (b.chunk_items > 0) {
        const int grid = (int)std::min<int64_t>(b.chunk_items, (int64_t)sm_count() * 8);
        kb_map<<<grid, kT, 0, s>>>(b.qps, b.nq, b.pchunk, dev ? -1 : b.chunk_items);
        kb_prefix<<<b.nq, 512, (size_t)b.max_words * 4, s>>>(b.qps);
        kb_survivors<<<(unsigned)b.chunk_items, kT, 0, s>>>(b.qps, b.nq, b.pchunk, b.claims + 0);
        for (int ps = 0; ps < b.max_passes; ++ps) {
            kb_radix_hist<<<(unsigned)b.chunk_items, kT, 0, s>>>(b.qps, b.nq, b.pchunk, ps);
            kb_radix_scan<<<b.nq, 256, 0, s>>>(b.qps, ps);
            kb_radix_scatter<<<(unsigned)b.chunk_items, kT, 0, s>>>(b.qps, b.nq, b.pchunk, ps);
        }
    }
    if (b.tile_items > 0) {
        kb_gather<<<(unsigned)b.tile_items, kTQ, 0, s>>>(b.qps, b.nq, b.ptile);
        kb_supmin<<<(unsigned)((b.tile_items + 7) / 8), 256, 0, s>>>(b.qps, b.nq, b.ptile, dev ? -1 : b.tile_items);
    }
    // step (d): one persistent kernel per padded-dimension class, in turn on
    // `s`, or (concurrent_classes) as parallel branches on the class streams
    const bool par = b.concurrent_classes && b.class_streams[0] && b.fork && b.joins[0];
    if (par) {
        cudaError_t e = cudaEventRecord(b.fork, s);
        if (e != cudaSuccess) return e;
    }
    for (int c = 0; c < 4; ++c) {
        const int n = b.class_items[c];
        if (!n) continue;
        const int2* it = b.items + b.class_begin[c];
        uint32_t* claim = b.claims + 2 + c;
        cudaStream_t cs = s;
        if (par) {
            cs = b.class_streams[c];
            cudaError_t e = cudaStreamWaitEvent(cs, b.fork, 0);
            if (e != cudaSuccess) return e;
        }
        const int ctas = b.class_ctas[c] > 0 ? b.class_ctas[c] : b.refine_ctas_per_sm;
        const int st = b.class_stages[c];
        const bool fast = b.class_fast[c] != 0;
        cudaError_t e = cudaSuccess;
        switch (c) {
            case 0: e = launch_kb_refine<4>(b.qps, it, n, claim, ctas, st, fast, b.d_class, c, cs); break;
            case 1: e = launch_kb_refine<8>(b.qps, it, n, claim, ctas, st, fast, b.d_class, c, cs); break;
            case 2: e = launch_kb_refine<12>(b.qps, it, n, claim, ctas, st, fast, b.d_class, c, cs); break;
            default: e = launch_kb_refine<16>(b.qps, it, n, claim, ctas, st, fast, b.d_class, c, cs); break;
        }
        if (e != cudaSuccess) return e;
        if (par) {
            e = cudaEventRecord(b.joins[c], cs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b.joins[c], 0);
            if (e != cudaSuccess) return e;
        }
    }
    if (b.chunk_items > 0) kb_emit<<<(unsigned)b.chunk_items, kT, 0, s>>>(b.qps, b.nq, b.pchunk, b.claims + 1);
    kb_finish<<<1, 1024, 0, s>>>(b.qps, b.nq, b.capacity, b.offsets, b.status);
    if (b.chunk_items > 0) {
        const int grid = (int)std::min<int64_t>(b.chunk_items, (int64_t)sm_count() * 8);
        kb_copy<<<grid, kT, 0, s>>>(b.qps, b.nq, b.pchunk, dev ? -1 : b.chunk_items, b.offsets, b.out, b.capacity);
    }
    return cudaGetLastError();
}

int batched_kernel_count(const BatchLaunch& b)
{
    int k = 0;
    if (b.chunk_items > 0) k += 3 + 3 * b.max_passes + 2;  // map, prefix, survivors, sort, emit, copy
    if (b.tile_items > 0) k += 2;   // gather, super-tile minima
    for (int c = 0; c < 4; ++c) k += b.class_items[c] ? 1 : 0;
    return k + 1;                                           // finish
}

}  // namespace sky
