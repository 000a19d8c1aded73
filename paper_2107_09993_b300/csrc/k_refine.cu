// k_refine.cu -- step (d): exact dominance refinement and compaction (sm_103a).
//
//   k_gather  lays the survivors out in Morton order: coordinates (padded to
//             a multiple of 4 floats), 7-bit per-dimension codes packed four
//             to a word, row ids, and per-tile bounding boxes.
//   k_refine  one CTA per tile of 128 survivors ("p" points). It lists the
//             tiles whose lower box corner is <= the CTA's upper box corner
//             (no other tile can hold a dominator), streams them into shared
//             memory with 1-D bulk (TMA) copies, and for each streamed tile
//             gives every lane one "q" point and loops the warp over the p's
//             that are still undominated and inside the tile's box. A pair is
//             tested first by a SIMD-within-a-word compare of 7-bit codes
//             (code(q) <= code(p) in every dimension is necessary because the
//             code map is monotone), then by the exact Definition 1 test on
//             the float values. The CTA stops when all its p's are dominated.
//   k_emit    ascending row ids of the kept points, by a decoupled look-back
//             scan over the per-row keep flags.
//
// Completeness: every survivor is tested against every survivor that could
// dominate it. If any point dominates p, some skyline point does
// (transitivity, Lemma 1 for cells / Definition 1 for points), and skyline
// points are never removed by step (c). Unlike the paper's RefineSkyline,
// which refines each candidate cell alone, tests cross cell boundaries: a
// point of one candidate cell can dominate a point of another.
#include <cstdint>

#include "sky_common.cuh"
#include "sky_internal.h"

namespace sky {

namespace {

constexpr int kTQ = kRefineTile;
constexpr int kSubSlots = kTQ / 32 + 1;   // sub-tile minima + the whole-tile minimum
constexpr uint32_t kHigh = 0x80808080u;

template <int DP>
__global__ void __launch_bounds__(kTQ) k_gather(const float* __restrict__ pts, int d, int64_t ld, bool vec4,
                                                const uint32_t* __restrict__ sorted_idx, const DevResult* res,
                                                const float* __restrict__ params, float* X, uint32_t* C,
                                                int32_t* ids, float* bbox, uint32_t* subcode)
{
    constexpr int DW = DP / 4;
    __shared__ float s_min[kTQ / 32][DP], s_max[kTQ / 32][DP];
    const uint32_t m = res->survivors;
    const uint32_t T = (m + kTQ - 1) / kTQ;
    if (blockIdx.x >= T) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t j = (int64_t)blockIdx.x * kTQ + tid;
    const bool valid = j < m;
    float x[DP];
    uint32_t row = 0;
    if (valid) {
        row = sorted_idx[j];
        const float* r = pts + (int64_t)row * ld;
        if (vec4) {
#pragma unroll
            for (int k = 0; k < DP; k += 4) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(r + k));
                x[k] = v.x; x[k + 1] = v.y; x[k + 2] = v.z; x[k + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < DP; ++k) x[k] = (k < d) ? __ldg(r + k) : 0.0f;
        }
    } else {
#pragma unroll
        for (int k = 0; k < DP; ++k) x[k] = INFINITY;
    }
    uint32_t code[DW];
#pragma unroll
    for (int w = 0; w < DW; ++w) code[w] = 0;
#pragma unroll
    for (int k = 0; k < DP; ++k) {
        uint32_t c;
        if (!valid) c = 127u;
        else if (k < d) c = column_of(x[k], __ldg(params + k), __ldg(params + 32 + k), 128u);
        else c = 0u;
        code[k / 4] |= c << (8 * (k % 4));
    }
    float4* xo = reinterpret_cast<float4*>(X + j * DP);
#pragma unroll
    for (int k = 0; k < DP; k += 4) xo[k / 4] = make_float4(x[k], x[k + 1], x[k + 2], x[k + 3]);
#pragma unroll
    for (int w = 0; w < DW; ++w) C[j * DW + w] = code[w];
    ids[j] = valid ? (int32_t)row : -1;

    // byte-wise minimum code of each 32-point sub-tile (slots 0..3) and of
    // the whole tile (slot 4)
    __shared__ uint32_t s_sub[kTQ / 32][DW];
#pragma unroll
    for (int w = 0; w < DW; ++w) {
        uint32_t c = code[w];
        for (int o = 16; o > 0; o >>= 1) c = __vminu4(c, __shfl_xor_sync(kFull, c, o));
        if (lane == 0) {
            subcode[((int64_t)blockIdx.x * kSubSlots + warp) * DW + w] = c;
            s_sub[warp][w] = c;
        }
    }

    // tile bounding box over the valid points
#pragma unroll
    for (int k = 0; k < DP; ++k) {
        float lo = valid ? x[k] : INFINITY;
        float hi = valid ? x[k] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(kFull, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, o));
        }
        if (lane == 0) { s_min[warp][k] = lo; s_max[warp][k] = hi; }
    }
    __syncthreads();
    if (tid < DW) {
        uint32_t c = s_sub[0][tid];
        for (int w = 1; w < kTQ / 32; ++w) c = __vminu4(c, s_sub[w][tid]);
        subcode[((int64_t)blockIdx.x * kSubSlots + kTQ / 32) * DW + tid] = c;
    }
    if (tid < DP) {
        float lo = s_min[0][tid], hi = s_max[0][tid];
        for (int w = 1; w < kTQ / 32; ++w) {
            lo = fminf(lo, s_min[w][tid]);
            hi = fmaxf(hi, s_max[w][tid]);
        }
        bbox[(int64_t)blockIdx.x * 2 * DP + tid] = lo;
        bbox[(int64_t)blockIdx.x * 2 * DP + DP + tid] = hi;
    }
}

// One CTA per p-tile of 128 survivors (Morton neighbours), split in 4 groups
// of 32, plus a producer warp. The producer scans the q-tiles in Morton
// order, keeps those whose byte-wise minimum code is <= the byte-wise maximum
// code of the live p's of some group (no other tile can hold a dominator of
// a live p), and streams them into a ring of shared-memory stages by bulk
// (TMA) copies, gated by full/empty mbarriers. Consumer warp w owns the 32
// q's of sub-tile w of each streamed tile (one per lane); it marks, by ballot,
// the live p's whose codes are >= the sub-tile's minimum code and loops over
// them, so every lane does a useful pair test on every step. When
// code(q) < code(p) in every dimension, q dominates p without looking at the
// floats; only pairs with some equal code need the exact Definition 1 test.
// A dominated p is flagged; when none is left the producer stops issuing and
// the consumers drain the ring. No block-wide barrier in the steady state.
constexpr int kRingStages = 4;
constexpr uint32_t kEndTile = 0xffffffffu;

template <int DP>
struct RefineSmem {
    static constexpr int DW = DP / 4;
    float qX[kRingStages][kTQ * DP];     // streamed q-tiles
    uint32_t qC[kRingStages][kTQ * DW];
    float pX[kTQ * DP];                  // own p coordinates (exact tests)
    uint32_t pP[kTQ * DW];               // own p codes | 0x80 per byte
    uint32_t livemask[kTQ / 32];         // bit l of word g: p g*32+l is still undominated
    uint32_t gmax[kTQ / 32][DW];         // byte-wise max code of each group's live p's (producer)
    uint32_t glive[kTQ / 32];            // live p's per group (producer)
    uint32_t stage_tile[kRingStages];
    uint32_t stage_mask[kRingStages];    // bit 4w+g: sub-tile w may dominate a live p of group g
    uint32_t stage_sub[kRingStages][kTQ / 32][DW];   // sub-tile minimum codes of the staged tile
    uint64_t full[kRingStages];
    uint64_t empty[kRingStages];
    uint32_t live;                       // live p's of the CTA
    uint32_t failed;
};

__device__ __forceinline__ uint32_t has_zero_byte(uint32_t x)
{
    return (x - 0x01010101u) & ~x & 0x80808080u;
}

// every byte of lo <= the matching byte of hi (both 7-bit codes)
template <int DW>
__device__ __forceinline__ bool bytes_le(const uint32_t* lo, const uint32_t* hi)
{
    uint32_t r = kHigh;
#pragma unroll
    for (int w = 0; w < DW; ++w) r &= (hi[w] | kHigh) - lo[w];
    return r == kHigh;
}

template <int DP>
__global__ void __launch_bounds__(kTQ + 32) k_refine(const float* __restrict__ X, const uint32_t* __restrict__ C,
                                                     const int32_t* __restrict__ ids,
                                                     const uint32_t* __restrict__ SUB, DevResult* res,
                                                     uint8_t* keep)
{
    constexpr int DW = DP / 4;
    constexpr int NG = kTQ / 32;
    constexpr int S = kRingStages;
    constexpr uint32_t kBytesX = kTQ * DP * sizeof(float);
    constexpr uint32_t kBytesC = kTQ * DW * sizeof(uint32_t);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    RefineSmem<DP>& sm = *reinterpret_cast<RefineSmem<DP>*>(smem_raw);

    const uint32_t m = res->survivors;
    const uint32_t T = (m + kTQ - 1) / kTQ;
    if (blockIdx.x >= T) return;
    uint32_t* err = &res->err;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t pbase = (int64_t)blockIdx.x * kTQ;
    if (tid < kTQ) {
        const bool valid = pbase + tid < m;
#pragma unroll
        for (int w = 0; w < DW; ++w) sm.pP[tid * DW + w] = C[(pbase + tid) * DW + w] | kHigh;
#pragma unroll
        for (int k = 0; k < DP; k += 4)
            *reinterpret_cast<float4*>(&sm.pX[tid * DP + k]) =
                *reinterpret_cast<const float4*>(X + (pbase + tid) * DP + k);
        const uint32_t vm = __ballot_sync(kFull, valid);
        if ((tid & 31) == 0) sm.livemask[tid >> 5] = vm;
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], NG);
        }
        mbar_fence_init();
        sm.live = (m - pbase) < (uint32_t)kTQ ? (m - (uint32_t)pbase) : (uint32_t)kTQ;
        sm.failed = 0;
    }
    __syncthreads();

    if (warp == NG) {
        // ------------------------------------------------------------ producer
        uint32_t issued = 0;
        auto summarise = [&]() {
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const int pi = g * 32 + lane;
                const uint32_t lm = sm.livemask[g];
                const bool live = (lm >> lane) & 1u;
                const uint32_t nl = __popc(lm);
#pragma unroll
                for (int w = 0; w < DW; ++w) {
                    uint32_t c = live ? (sm.pP[pi * DW + w] & 0x7f7f7f7fu) : 0u;
                    for (int o = 16; o > 0; o >>= 1) c = __vmaxu4(c, __shfl_xor_sync(kFull, c, o));
                    if (lane == 0) sm.gmax[g][w] = c;
                }
                if (lane == 0) sm.glive[g] = nl;
            }
            __syncwarp();
        };
        // claims the next ring slot (waits until the consumers released it)
        auto claim = [&](int& s) -> bool {
            s = (int)(issued % S);
            bool ok = true;
            if (issued >= (uint32_t)S) ok = mbar_wait(&sm.empty[s], ((issued / S) & 1u) ^ 1u, err);
            return __all_sync(kFull, ok);
        };
        summarise();
        bool stop = false;
        uint32_t since = 0;
        // shared flags are read by lane 0 and broadcast, so that every branch
        // around the warp-wide votes below stays uniform
        auto all_dead = [&]() -> bool {
            return __shfl_sync(kFull, (sm.live == 0u || sm.failed != 0u) ? 1 : 0, 0) != 0;
        };
        // codes of the next 32 tiles are fetched one batch ahead
        uint32_t tm[DW], sc[NG][DW];
        auto fetch = [&](uint32_t t) {
#pragma unroll
            for (int w = 0; w < DW; ++w) tm[w] = t < T ? __ldg(SUB + ((int64_t)t * kSubSlots + NG) * DW + w) : 0u;
#pragma unroll
            for (int q = 0; q < NG; ++q)
#pragma unroll
                for (int w = 0; w < DW; ++w) sc[q][w] = t < T ? __ldg(SUB + ((int64_t)t * kSubSlots + q) * DW + w) : 0u;
        };
        fetch(lane);
        for (uint32_t t0 = 0; t0 < T && !stop; t0 += 32) {
            if (all_dead()) break;
            if (since >= 32) { summarise(); since = 0; }
            const uint32_t t = t0 + lane;
            uint32_t ctm[DW], csc[NG][DW];
#pragma unroll
            for (int w = 0; w < DW; ++w) ctm[w] = tm[w];
#pragma unroll
            for (int q = 0; q < NG; ++q)
#pragma unroll
                for (int w = 0; w < DW; ++w) csc[q][w] = sc[q][w];
            fetch(t + 32);
            // relevance of each (sub-tile, group) pair of this q-tile
            uint32_t rmask = 0;
            if (t < T) {
                bool any = false;
#pragma unroll
                for (int g = 0; g < NG; ++g) any |= (sm.glive[g] != 0u) && bytes_le<DW>(ctm, sm.gmax[g]);
                if (any) {
#pragma unroll
                    for (int q = 0; q < NG; ++q)
#pragma unroll
                        for (int g = 0; g < NG; ++g)
                            if (sm.glive[g] != 0u && bytes_le<DW>(csc[q], sm.gmax[g])) rmask |= 1u << (q * NG + g);
                }
            }
            uint32_t mask = __ballot_sync(kFull, rmask != 0u);
            while (mask) {
                const int b = __ffs(mask) - 1;
                mask &= mask - 1;
                const uint32_t bmask = __shfl_sync(kFull, rmask, b);
                int s;
                if (!claim(s)) { if (lane == 0) sm.failed = 1u; stop = true; break; }
                {
                    // every lane holds its own tile's codes; move tile b's to the slot
#pragma unroll
                    for (int q = 0; q < NG; ++q)
#pragma unroll
                        for (int w = 0; w < DW; ++w) {
                            const uint32_t v = __shfl_sync(kFull, csc[q][w], b);
                            if (lane == 0) sm.stage_sub[s][q][w] = v;
                        }
                }
                if (lane == 0) {
                    const uint32_t tt = t0 + b;
                    sm.stage_tile[s] = tt;
                    sm.stage_mask[s] = bmask;
                    mbar_arrive_expect_tx(&sm.full[s], kBytesX + kBytesC);
                    bulk_g2s(sm.qX[s], X + (int64_t)tt * kTQ * DP, kBytesX, &sm.full[s]);
                    bulk_g2s(sm.qC[s], C + (int64_t)tt * kTQ * DW, kBytesC, &sm.full[s]);
                }
                __syncwarp();
                ++issued;
                ++since;
                if (all_dead()) { stop = true; break; }
            }
        }
        if (lane == 0 && issued) atomicAdd(&res->tiles, (unsigned long long)issued);
        // end-of-stream marker
        int s;
        const bool marked = claim(s);
        if (marked) {
            if (lane == 0) {
                sm.stage_tile[s] = kEndTile;
                mbar_arrive(&sm.full[s]);
            }
        } else if (lane == 0) {
            sm.failed = 1u;
        }
        // Every bulk copy issued by this warp has landed before the CTA can
        // exit. (On the normal path the consumers have waited for all of them;
        // this matters after a timeout.) The slot reused by the marker was
        // released by the consumers, so its copy has landed already.
        if (lane == 0) {
            uint32_t first = issued > (uint32_t)S ? issued - S : 0u;
            if (marked && issued >= (uint32_t)S) first += 1;
            for (uint32_t k = first; k < issued; ++k) mbar_wait(&sm.full[k % S], (k / S) & 1u, nullptr);
        }
    } else {
        // ------------------------------------------------------------ consumers
        const int qi = warp * 32 + lane;
        unsigned long long pairs = 0, gscans = 0;
        for (uint32_t k = 0;; ++k) {
            const int s = (int)(k % S);
            const bool ok = mbar_wait(&sm.full[s], (k / S) & 1u, err);
            if (!__all_sync(kFull, ok)) {
                if (lane == 0) sm.failed = 1u;
                break;
            }
            const uint32_t tt = sm.stage_tile[s];
            if (tt == kEndTile) break;
            const uint32_t gm = (sm.stage_mask[s] >> (warp * NG)) & ((1u << NG) - 1u);
            const bool any_live = __shfl_sync(kFull, sm.live != 0u ? 1 : 0, 0) != 0;
            if (any_live && gm) {
                uint32_t Mw[DW];
#pragma unroll
                for (int w = 0; w < DW; ++w) Mw[w] = sm.stage_sub[s][warp][w];
                uint32_t Q[DW];
#pragma unroll
                for (int w = 0; w < DW; ++w) Q[w] = sm.qC[s][qi * DW + w];
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    if (!((gm >> g) & 1u)) continue;   // no live p of group g within reach
                    ++gscans;
                    const int pg = g * 32 + lane;
                    uint32_t r = kHigh;
#pragma unroll
                    for (int w = 0; w < DW; ++w) r &= sm.pP[pg * DW + w] - Mw[w];
                    uint32_t mask = __ballot_sync(kFull, r == kHigh) & sm.livemask[g];
                    pairs += 32ull * __popc(mask);
                    while (mask) {
                        const int pi = g * 32 + __ffs(mask) - 1;
                        mask &= mask - 1;
                        uint32_t D[DW];
                        uint32_t a = kHigh;
#pragma unroll
                        for (int w = 0; w < DW; ++w) {
                            D[w] = sm.pP[pi * DW + w] - Q[w];
                            a &= D[w];
                        }
                        if (a == kHigh) {  // code(q) <= code(p) in every dimension
                            uint32_t eq = 0;
#pragma unroll
                            for (int w = 0; w < DW; ++w) eq |= has_zero_byte(D[w] ^ kHigh);
                            bool dom = true;   // strictly lower code everywhere: q < p everywhere
                            if (eq) {
                                const float* qx = &sm.qX[s][qi * DP];
                                const float* px = &sm.pX[pi * DP];
                                bool le = true, lt = false;
#pragma unroll
                                for (int kk = 0; kk < DP; kk += 4) {
                                    const float4 u = *reinterpret_cast<const float4*>(qx + kk);
                                    const float4 v = *reinterpret_cast<const float4*>(px + kk);
                                    le &= (u.x <= v.x) & (u.y <= v.y) & (u.z <= v.z) & (u.w <= v.w);
                                    lt |= (u.x < v.x) | (u.y < v.y) | (u.z < v.z) | (u.w < v.w);
                                }
                                dom = le && lt;
                            }
                            if (dom) {
                                const uint32_t bit = 1u << (pi & 31);
                                if (atomicAnd(&sm.livemask[pi >> 5], ~bit) & bit) atomicSub(&sm.live, 1u);
                            }
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[s]);
        }
        if (lane == 0 && pairs) atomicAdd(&res->pairs, pairs);  // 32 q-lanes per listed p, per warp
        if (lane == 0 && gscans) atomicAdd(&res->groups, gscans);
    }
    __syncthreads();
    if (tid < kTQ && pbase + tid < m && !sm.failed && ((sm.livemask[tid >> 5] >> (tid & 31)) & 1u))
        keep[ids[pbase + tid]] = 1;
}

// Ascending row ids of the kept rows (decoupled look-back over 8 rows per
// thread). Writes beyond `capacity` are dropped; the count is always exact.
__global__ void __launch_bounds__(kScanThreads) k_emit(const uint8_t* __restrict__ keep, int64_t n,
                                                       int32_t* out, int64_t capacity, DevResult* res,
                                                       unsigned long long* states, uint32_t* tile_counter)
{
    __shared__ uint32_t s_warp[kScanThreads / 32];
    __shared__ uint32_t s_tile, s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * kScanTile + (int64_t)tid * kScanItems;
    uint32_t flags = 0;
    if (base + kScanItems <= n) {
        const uint2 v = *reinterpret_cast<const uint2*>(keep + base);
        const uint64_t b = ((uint64_t)v.y << 32) | v.x;
#pragma unroll
        for (int jj = 0; jj < kScanItems; ++jj)
            if ((b >> (8 * jj)) & 0xffull) flags |= 1u << jj;
    } else {
        for (int jj = 0; jj < kScanItems; ++jj)
            if (base + jj < n && keep[base + jj]) flags |= 1u << jj;
    }
    // block exclusive scan of per-thread counts
    const uint32_t v = __popc(flags);
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < warp) before += s_warp[w];
        total += s_warp[w];
    }
    const uint32_t excl = before + x - v;
    if (tid < 32) {
        const uint32_t prefix = lookback_prefix(states, tile, total, &res->err);
        if (tid == 0) s_prefix = prefix;
    }
    __syncthreads();
    int64_t pos = (int64_t)s_prefix + excl;
    for (int jj = 0; jj < kScanItems; ++jj) {
        if (flags & (1u << jj)) {
            if (pos < capacity) out[pos] = (int32_t)(base + jj);
            ++pos;
        }
    }
    const uint32_t ntiles = (uint32_t)((n + kScanTile - 1) / kScanTile);
    if (tile == ntiles - 1 && tid == 0) res->count = s_prefix + total;
}

}  // namespace

#define SKY_DISPATCH_DP(d, ...)                                 \
    switch (pad4(d)) {                                          \
        case 4: { constexpr int DP = 4; __VA_ARGS__; } break;   \
        case 8: { constexpr int DP = 8; __VA_ARGS__; } break;   \
        case 12: { constexpr int DP = 12; __VA_ARGS__; } break; \
        default: { constexpr int DP = 16; __VA_ARGS__; } break; \
    }

cudaError_t launch_gather(const Plan& p, cudaStream_t s)
{
    const int64_t tiles = (p.n + kTQ - 1) / kTQ;
    if (tiles == 0) return cudaGetLastError();
    const bool v = (p.d % 4 == 0) && (p.ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(p.pts) & 15u) == 0);
    SKY_DISPATCH_DP(p.d, k_gather<DP><<<(unsigned)tiles, kTQ, 0, s>>>(p.pts, p.d, p.ld, v, p.sorted_val, p.res,
                                                                       p.params, p.X, p.C, p.ids, p.bbox,
                                                                       p.subcode));
    return cudaGetLastError();
}

cudaError_t launch_refine(const Plan& p, cudaStream_t s)
{
    cudaMemsetAsync(p.keep, 0, (size_t)p.n, s);
    const int64_t tiles = (p.n + kTQ - 1) / kTQ;
    if (tiles == 0) return cudaGetLastError();
    SKY_DISPATCH_DP(p.d, {
        const int smem = (int)sizeof(RefineSmem<DP>);
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_refine<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            attr_set = true;
        }
        k_refine<DP><<<(unsigned)tiles, kTQ + 32, smem, s>>>(p.X, p.C, p.ids, p.subcode, p.res, p.keep);
    });
    return cudaGetLastError();
}

cudaError_t launch_emit(const Plan& p, int32_t* out, int64_t capacity, cudaStream_t s)
{
    if (p.n == 0) return cudaGetLastError();
    const int64_t ntiles = (p.n + kScanTile - 1) / kScanTile;
    cudaMemsetAsync(p.lb_states, 0, sizeof(unsigned long long) * ntiles, s);
    cudaMemsetAsync(p.lb_counter + 1, 0, sizeof(uint32_t), s);
    k_emit<<<(unsigned)ntiles, kScanThreads, 0, s>>>(p.keep, p.n, out, capacity, p.res, p.lb_states,
                                                     p.lb_counter + 1);
    return cudaGetLastError();
}

}  // namespace sky
