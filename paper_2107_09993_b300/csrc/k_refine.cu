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
#include <algorithm>
#include <cstdint>

#include "sky_common.cuh"
#include "sky_internal.h"
#include "sky_refine.cuh"

namespace sky {

namespace {

using namespace refine;

// Pre-pass of the refinement (at least kPreMinRows rows and survivors): every
// p-tile is first refined against itself and the first kPreTiles q-tiles of
// the Morton order only (the points nearest the origin, which dominate the
// most); the survivors of that pass are compacted in order and the full
// refinement runs on them. Exact: the pre-pass removes only points it has
// found dominated, and every dominated point has a skyline dominator, which
// no pass removes, so skyline(survivors) = skyline(pre-pass survivors).
// What it saves: the full refinement no longer streams and tests the
// dominated points as q's. Measured on B300 (ms, one sky_skyline call, no
// pre-pass / 4 / 8 / 16 tiles): 10^7 x 12 independent 40.5 / 24.2 / 22.1 /
// 20.8, 10^7 x 16 anti-correlated 107.5 / 109.5 / 109.2 / 109.1 (nothing to
// remove there: 82 % of its points are skyline points); on 10^6 x 8 sets its
// fixed cost (three launches, a second gather) outweighs it (independent
// 0.72 -> 0.82-0.86 ms), hence the row threshold.
#ifndef SKY_REFINE_PRE_TILES
#define SKY_REFINE_PRE_TILES 16
#endif
constexpr uint32_t kPreTiles = SKY_REFINE_PRE_TILES;   // 0: no pre-pass
#ifndef SKY_REFINE_PRE_MIN_ROWS
#define SKY_REFINE_PRE_MIN_ROWS (int64_t(1) << 21)
#endif
constexpr int64_t kPreMinRows = SKY_REFINE_PRE_MIN_ROWS;

template <int DP>
__global__ void __launch_bounds__(kTQ) k_gather(const float* __restrict__ pts, int d, int64_t ld, bool vec4,
                                                const uint32_t* __restrict__ sorted_idx,
                                                const uint32_t* __restrict__ sorted_key, const uint32_t* mcount,
                                                const float* __restrict__ params, float* X, uint32_t* C,
                                                int32_t* ids, uint32_t* tmax, uint32_t* subcode,
                                                uint32_t* tile_end, uint32_t* cidx, uint32_t* tend_pre,
                                                uint32_t* tmask)
{
    constexpr int DW = DP / 4;
    const uint32_t m = *mcount;
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

    // layer-1 cell index: per cell (bit k: code k >= 64), the first and last
    // tile holding one of its points, as ~first (cidx[cell]) and last + 1
    // (cidx[2^d + cell]) by atomicMax into arrays the call's first kernel
    // zeroed; one update per distinct cell of a warp
    if (cidx != nullptr) {
        const uint32_t cell = cell_of_codes<DW>(code);
        const uint32_t peers = __match_any_sync(kFull, valid ? cell : 0xffffffffu);
        if (valid && lane == __ffs(peers) - 1) {
            atomicMax(cidx + cell, ~(uint32_t)blockIdx.x);
            atomicMax(cidx + (1u << d) + cell, (uint32_t)blockIdx.x + 1u);
        }
    }

    // threshold masks of this warp's 32-point sub-tile (the refinement's
    // mask probe): word k * 8 + l = the lanes whose 3-bit code (the top three
    // bits of the 7-bit code) in dimension k is <= l; padding points (code
    // 127) pass only level 7, which every point passes
    if constexpr (DP >= 8) {
        if (tmask != nullptr) {
            uint32_t v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                // dimensions past the padded ones: every point at level 0
                const uint32_t c3 = k < DP ? (code[k < DP ? k >> 2 : 0] >> (8 * (k & 3) + 4)) & 7u : 0u;
#pragma unroll
                for (int l = 0; l < 8; ++l) {
                    const uint32_t b = l == 7 ? kFull : __ballot_sync(kFull, c3 <= (uint32_t)l);
                    const int e = k * 8 + l;
                    if (lane == (e & 31)) v[e >> 5] = b;
                }
            }
            uint32_t* o = tmask + ((int64_t)blockIdx.x * (kTQ / 32) + warp) * 128;
#pragma unroll
            for (int r = 0; r < 4; ++r) o[r * 32 + lane] = v[r];
        }
    }

    // byte-wise minimum code of each 32-point sub-tile (slots 0..3) and of
    // the whole tile (slot 4); byte-wise maximum code of the tile's valid
    // points (the order of the p-tiles uses it)
    __shared__ uint32_t s_sub[kTQ / 32][DW], s_top[kTQ / 32][DW];
#pragma unroll
    for (int w = 0; w < DW; ++w) {
        uint32_t c = code[w];
        uint32_t t = valid ? code[w] : 0u;
        for (int o = 16; o > 0; o >>= 1) {
            c = __vminu4(c, __shfl_xor_sync(kFull, c, o));
            t = __vmaxu4(t, __shfl_xor_sync(kFull, t, o));
        }
        if (lane == 0) {
            subcode[((int64_t)blockIdx.x * kSubSlots + warp) * DW + w] = c;
            s_sub[warp][w] = c;
            s_top[warp][w] = t;
        }
    }
    __syncthreads();
    if (tid < DW) {
        uint32_t c = s_sub[0][tid], t = s_top[0][tid];
        for (int w = 1; w < kTQ / 32; ++w) {
            c = __vminu4(c, s_sub[w][tid]);
            t = __vmaxu4(t, s_top[w][tid]);
        }
        subcode[((int64_t)blockIdx.x * kSubSlots + kTQ / 32) * DW + tid] = c;
        tmax[(int64_t)blockIdx.x * DW + tid] = t;
    }
    // The last q-tile that can hold a dominator of a point of this tile: a
    // dominator's Morton key is <= its victim's (monotone columns), so only
    // tiles whose first key is <= this tile's last key qualify. Ties across
    // tile boundaries are the only reason to look past this tile.
    // Warp 0 checks the first keys of the next 32 tiles at once (one round of
    // loads; ties spanning more tiles take further rounds).
    if (warp == 0) {
        const uint32_t last = sorted_key[min((int64_t)m, ((int64_t)blockIdx.x + 1) * kTQ) - 1];
        uint32_t e = blockIdx.x;
        while (true) {
            const uint32_t t = e + 1 + lane;
            const bool tie = t < T && sorted_key[(int64_t)t * kTQ] <= last;
            const uint32_t run = __ballot_sync(kFull, !tie);   // first lane that is not a tie ends the run
            const uint32_t k = run ? (uint32_t)(__ffs(run) - 1) : 32u;
            e += k;
            if (k < 32u) break;
        }
        if (lane == 0) {
            tile_end[blockIdx.x] = e;
            if (tend_pre) tend_pre[blockIdx.x] = min(e, kPreTiles - 1u);
        }
    }
}

// Cost estimate of each p-tile for the launch order of the refinement: how
// many q-tiles of an evenly strided sample (at most kCostSamples) up to the
// p-tile's Morton cutoff (TEND: no later tile is scanned) have a
// tile-minimum code <= the p-tile's maximum code in every byte, i.e. could
// hold a dominator of one of its points and would be streamed while any of
// them is alive. (Measured on the three families at n = 10^6, d = 8, this
// plain count orders the grid better than refinements that try to predict
// early termination.) One warp per p-tile.
constexpr int kCostSamples = 1024;

template <int DW>
__global__ void __launch_bounds__(256) k_tile_cost(const uint32_t* __restrict__ SUB, const uint32_t* __restrict__ tmax,
                                                   const uint32_t* __restrict__ tend, const uint32_t* mcount,
                                                   uint32_t* cost, uint32_t* supmin)
{
    // the sampled q-tiles' minimum codes, shared by the block's eight warps
    // (one p-tile each)
    __shared__ uint32_t s_qmin[kCostSamples][DW];
    const uint32_t T = (*mcount + kTQ - 1) / kTQ;
    if (blockIdx.x * 8 >= T) return;
    {
        // warp w of block b: byte-wise minimum code of super-tile 8b + w (32
        // tiles, one per lane; tiles past the end count as the largest code)
        const uint32_t sx = blockIdx.x * 8 + (threadIdx.x >> 5);
        const uint32_t tq = sx * 32 + (threadIdx.x & 31);
        if (sx * 32 < T) {
#pragma unroll
            for (int w = 0; w < DW; ++w) {
                uint32_t c = tq < T ? __ldg(SUB + ((int64_t)tq * kSubSlots + kTQ / 32) * DW + w) : 0x7f7f7f7fu;
                for (int o = 16; o > 0; o >>= 1) c = __vminu4(c, __shfl_xor_sync(kFull, c, o));
                if ((threadIdx.x & 31) == 0) supmin[(int64_t)sx * DW + w] = c;
            }
        }
    }
    const uint32_t step = (T + kCostSamples - 1) / kCostSamples;   // ns <= kCostSamples
    const uint32_t ns = (T + step - 1) / step;
    for (uint32_t i = threadIdx.x; i < ns; i += blockDim.x) {
        const int64_t q = (int64_t)i * step;
#pragma unroll
        for (int w = 0; w < DW; ++w) {
            s_qmin[i][w] = __ldg(SUB + (q * kSubSlots + kTQ / 32) * DW + w);
        }
    }
    __syncthreads();
    const uint32_t pt = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (pt >= T) return;
    uint32_t top[DW];
#pragma unroll
    for (int w = 0; w < DW; ++w) top[w] = tmax[(int64_t)pt * DW + w] | kHigh;
    uint32_t cnt = 0;
    const uint32_t nse = min(ns, tend[pt] / step + 1u);   // samples at tiles <= the cutoff
    for (uint32_t i = lane; i < nse; i += 32u) {
        uint32_t r = kHigh;
#pragma unroll
        for (int w = 0; w < DW; ++w) r &= top[w] - s_qmin[i][w];
        cnt += (r == kHigh) ? 1u : 0u;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    if (lane == 0) cost[pt] = cnt;
}

// Launch order of the p-tiles, largest estimated cost first (longest job
// first evens out the end of the grid): a counting sort over the exact cost
// values (at most kCostOrderBuckets - 1) in one CTA. Order among equal costs
// is arbitrary; the result does not depend on it. A p-tile of nt
// consecutive 128-point tiles costs the sum of theirs.
// (Power-of-two buckets, the earlier form, put every p-tile of half the
// maximum cost or more into one bucket in arbitrary order; at 2*10^6 x 16
// anti-correlated the busiest SM then stayed active 20 % past the average.)
constexpr int kCostOrderBuckets = 2 * kCostSamples;
// Split scans from this padded dimension up (0: never). Split parts run
// neither the sparse tail nor the super-tile test (their windows must be the
// same sequence in every part), which cost more than the split saved on
// 10^6 x 8 sets (anti-correlated 1.20 -> 1.30 ms, independent 0.69 ->
// 0.84 ms with splits from half the span). Only launches of at most
// SKY_REFINE_SPLIT_MAX_WAVES waves of p-tiles split: with more, the
// longest-first order already evens out the end (10^7 x 16 anti-correlated:
// slots 98.7 % busy) and splitting measured 0.5 % slower there.
#ifndef SKY_REFINE_SPLIT_MIN_DP
#define SKY_REFINE_SPLIT_MIN_DP 12
#endif
#ifndef SKY_REFINE_SPLIT_MAX_WAVES
#define SKY_REFINE_SPLIT_MAX_WAVES 32
#endif

// Split scans: a p-tile's scan is one CTA's serial work, and on sets of a
// few million points the costliest one can span the whole launch. With
// `slots` resident CTAs, span = (sum of the costs) / slots; a p-tile costing
// more than span gets K = min(8, ceil(2 cost / span)) order entries (parts),
// part k taking every K-th window of the scan (the own tiles go to part 0),
// and the parts merge their kills (refine_ptile). Since K - 1 < 2 cost /
// span, the extra entries stay below 2 * slots, and the split p-tiles below
// slots (kSplitExtra, kSplitSlots). nt = 1 only (128-point p-tiles); slots =
// 0: no split.
__global__ void __launch_bounds__(1024) k_cost_order(const uint32_t* __restrict__ cost, const uint32_t* mcount,
                                                     uint32_t* order, uint32_t nt, uint32_t* part,
                                                     uint32_t* split, uint32_t slots)
{
    static_assert(kCostOrderBuckets == 2 * 1024, "two buckets per thread of the scan");
    __shared__ uint32_t s_cnt[kCostOrderBuckets];
    __shared__ uint32_t s_warp[32];
    __shared__ unsigned long long s_total;
    __shared__ uint32_t s_slot;
    const uint32_t T0 = (*mcount + kTQ - 1) / kTQ;
    const uint32_t T = (T0 + nt - 1) / nt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto item_cost = [&](uint32_t t) -> uint32_t {
        uint32_t c = 0;
        for (uint32_t h = 0; h < nt && t * nt + h < T0; ++h) c += cost[t * nt + h];
        return c;
    };
    // bucket of item t: kCostOrderBuckets - 1 - cost, so that ascending
    // buckets are descending costs
    auto bucket = [&](uint32_t c) -> uint32_t {
        return (uint32_t)kCostOrderBuckets - 1u - min(c, (uint32_t)kCostOrderBuckets - 1u);
    };
    for (int i = tid; i < kSplitSlots * 5; i += blockDim.x) split[i] = 0u;
    s_cnt[2 * tid] = 0u;
    s_cnt[2 * tid + 1] = 0u;
    if (tid == 0) { s_total = 0ull; s_slot = 0u; }
    __syncthreads();
    unsigned long long mine = 0;
    if (slots != 0u)
        for (uint32_t t = tid; t < T; t += blockDim.x) mine += item_cost(t);
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(kFull, mine, o);
    if (lane == 0) atomicAdd(&s_total, mine);
    __syncthreads();
    const unsigned long long total = s_total;
    // parts of an item: 2 cost * slots vs total (no split for two-tile p-tiles)
    auto parts = [&](uint32_t c) -> uint32_t {
        if (nt != 1u || total == 0ull || (unsigned long long)c * slots <= total) return 1u;
        const unsigned long long k = (2ull * c * slots + total - 1ull) / total;
        return (uint32_t)min(k, 8ull);
    };
    for (uint32_t t = tid; t < T; t += blockDim.x) {
        const uint32_t c = item_cost(t);
        atomicAdd(&s_cnt[bucket(c)], parts(c));
    }
    __syncthreads();
    // exclusive scan of the bucket counts (thread i: buckets 2i and 2i + 1)
    const uint32_t c0 = s_cnt[2 * tid], c1 = s_cnt[2 * tid + 1];
    uint32_t x = c0 + c1;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const uint32_t before = (warp ? s_warp[warp - 1] : 0u) + x - (c0 + c1);
    if (tid == 0) split[kSplitSlots * 5] = s_warp[31];   // order entries
    __syncthreads();   // every thread has read its counts
    s_cnt[2 * tid] = before;
    s_cnt[2 * tid + 1] = before + c0;
    __syncthreads();
    for (uint32_t t = tid; t < T; t += blockDim.x) {
        const uint32_t c = item_cost(t);
        const uint32_t k = parts(c);
        const uint32_t pos = atomicAdd(&s_cnt[bucket(c)], k);
        const uint32_t slot = k > 1u ? atomicAdd(&s_slot, 1u) : 0u;
        for (uint32_t j = 0; j < k; ++j) {
            order[pos + j] = t;
            part[pos + j] = j | (k << 8) | (slot << 16);
        }
    }
}

// Resident CTAs per SM by padded dimension (the launch bound caps the
// registers: 9 -> 40, 8 -> 48, 7 -> 56, 6 -> 64, 5 -> 72 per thread). A
// common cap of nine spilled 432 bytes a thread at d = 16 and 128 at d = 12
// to local memory, and long-scoreboard stalls on the spill loads dominated;
// measured on B300 (10^7 x 16 anti-correlated 233.9 -> 132.8 ms, 10^7 x 12
// independent 61.0 -> 45.3 ms, 10^6 x 8 anti-correlated 1.26 -> 1.20 ms),
// the best of 5-9 per class.
#ifndef SKY_REFINE_MINB_4
#define SKY_REFINE_MINB_4 9
#endif
#ifndef SKY_REFINE_MINB_8
#define SKY_REFINE_MINB_8 8
#endif
#ifndef SKY_REFINE_MINB_12
#define SKY_REFINE_MINB_12 7
#endif
#ifndef SKY_REFINE_MINB_16
#define SKY_REFINE_MINB_16 6
#endif
// The mask probe (see sky_refine.cuh) from this padded dimension up (built
// for 8, 12 and 16; larger: off) and its CTAs per SM (72 / 64 / 48
// registers; five CTAs at d = 12 measured 10^7 x 12 independent 17.3 ->
// 18.8 ms). At padded dimension 8 it did not pay (ms, list -> mask probe
// with 8 / 7 CTAs per SM): 10^6 x 8 anti-correlated 1.20 -> 1.21 / 1.17,
// independent 0.70 -> 0.72 / 0.74, correlated 0.29 -> 0.36, 2*10^6 x 8
// anti-correlated 2.29 -> 2.00 / 2.07; hence from 12.
#ifndef SKY_REFINE_MASK_MIN_DP
#define SKY_REFINE_MASK_MIN_DP 12
#endif
#ifndef SKY_REFINE_MINB_16_MASK
#define SKY_REFINE_MINB_16_MASK 6
#endif
// masks only in the stages (see RefineSmem) from this padded dimension up,
// with this ring depth. Measured on B300 (ms, one call; masks and codes in
// 6 stages, 5 CTAs per SM -> masks only in 8 stages, 6 CTAs per SM): 10^7 x
// 16 anti-correlated 83.7 -> 75.9, 2*10^6 x 16 independent 12.7 -> 11.5,
// anti-correlated 11.8 -> 12.0, correlated 10.7 -> 13.0 (many 3-bit passes,
// each now reading its q's codes from global memory); at d = 12 (masks
// only, 8 stages, 7 CTAs) 10^7 x 12 independent 17.2 -> 17.8, hence 16;
// bench step 101.2 -> 93.2 ms.
#ifndef SKY_REFINE_MASK_ONLY_MIN_DP
#define SKY_REFINE_MASK_ONLY_MIN_DP 16
#endif
#ifndef SKY_REFINE_MASK_ONLY_STAGES
#define SKY_REFINE_MASK_ONLY_STAGES 10
#endif
#ifndef SKY_REFINE_MINB_12_MASK
#define SKY_REFINE_MINB_12_MASK 6
#endif
#ifndef SKY_REFINE_MINB_8_MASK
#define SKY_REFINE_MINB_8_MASK 8
#endif
template <int DP>
struct RefineMask {
    static constexpr bool value = DP >= 8 && DP >= SKY_REFINE_MASK_MIN_DP;
    // RefineSmem's MASK: 0 off, 1 masks and codes staged, 2 masks only
    static constexpr int mode = !value ? 0 : (DP >= SKY_REFINE_MASK_ONLY_MIN_DP && SKY_REFINE_MASK_MIN_LIST <= 1) ? 2 : 1;
    static constexpr int stages = mode == 2 ? SKY_REFINE_MASK_ONLY_STAGES : mode == 1 ? SKY_REFINE_MASK_STAGES
                                                                                     : kRingStages;
};
template <int DP>
struct RefineMinBlocks {
    static constexpr int value = DP == 4 ? SKY_REFINE_MINB_4
                               : DP == 8 ? (RefineMask<DP>::value ? SKY_REFINE_MINB_8_MASK : SKY_REFINE_MINB_8)
                               : DP == 12 ? (RefineMask<DP>::value ? SKY_REFINE_MINB_12_MASK : SKY_REFINE_MINB_12)
                               : RefineMask<DP>::value ? SKY_REFINE_MINB_16_MASK : SKY_REFINE_MINB_16;
};

// p's per CTA of the full refinement by padded dimension: from
// SKY_REFINE_WIDE_MIN_DP up, 256 (two consecutive 128-point tiles, eight
// groups of 32: each streamed q-tile, its relevance test and its stage
// hand-offs serve twice the p's); below it, 128. The p coordinates of a
// 256-point CTA stay in global memory (SKY_REFINE_PX_SMEM_WIDE), so its
// shared memory and launch bound are those of the 128-point form. The
// pre-pass keeps 128. Measured on B300 (ms, one sky_skyline call, seed 1,
// 128 -> 256 p's): 10^7 x 16 anti-correlated 109.1 -> 115.4, 2*10^6 x 16
// anti-correlated 14.8 -> 19.2, independent 14.2 -> 15.9, correlated 10.7
// -> 14.9; at d = 12 (from 12 up) 2*10^6 anti-correlated 8.3 -> 10.1,
// 10^7 independent 20.9 -> 21.1. Streamed q-tiles fell by a third and the
// instructions by 3 %, but a p-tile's scan is one CTA's serial work: at
// 2*10^6 x 16 the longest CTA spans the whole launch (ncu: busiest SM active
// 40.3 M cycles against a 25.7 M average, 29.2 M against 24.4 M with 128
// p's), and doubling the p's doubles that critical path. So off (32: never).
#ifndef SKY_REFINE_WIDE_MIN_DP
#define SKY_REFINE_WIDE_MIN_DP 32
#endif
template <int DP>
struct RefineGroups {
    static constexpr int value = DP >= SKY_REFINE_WIDE_MIN_DP ? 2 * (kTQ / 32) : kTQ / 32;
};
template <int DP, int PG>
using SetSmem = RefineSmem<DP, RefineMask<DP>::stages, (DP >= SKY_REFINE_FAST_MIN_DP), PG, RefineMask<DP>::mode>;

// WIT: witness mode (see refine_ptile); `wit` is unused otherwise. PG:
// groups of 32 p's per CTA (4 or 8). ORDER / PART / SPLIT (the full pass):
// the p-tile, part and split record of block b's entry (k_cost_order), and
// the number of entries; NULL: p-tile b, one part.
template <int DP, bool WIT, int PG>
__global__ void __launch_bounds__(kTQ + 32, RefineMinBlocks<DP>::value) k_refine(const float* __restrict__ X, const uint32_t* __restrict__ C,
                                                     const int32_t* __restrict__ ids,
                                                     const uint32_t* __restrict__ SUB,
                                                     const uint32_t* __restrict__ tend,
                                                     const uint32_t* __restrict__ supmin,
                                                     const uint32_t* __restrict__ order, const uint32_t* mcount,
                                                     DevResult* res,
                                                     uint8_t* keep, int32_t* wit, const uint32_t* __restrict__ cidx,
                                                     int d, uint32_t min_m, const uint32_t* __restrict__ tmask,
                                                     const uint32_t* __restrict__ part, uint32_t* split)
{
    extern __shared__ __align__(256) unsigned char smem_raw[];
    using SM = SetSmem<DP, PG>;
    SM& sm = *reinterpret_cast<SM*>(smem_raw);
    const uint32_t m = *mcount;
    constexpr uint32_t kTP = SM::kTP;
    const uint32_t entries = part ? split[kSplitSlots * 5] : (m + kTP - 1) / kTP;
    if (m < min_m || blockIdx.x >= entries) return;   // min_m: the pre-pass's survivor threshold
    const uint32_t ptile = order ? order[blockIdx.x] : blockIdx.x;
    const uint32_t pinfo = part ? part[blockIdx.x] : (1u << 8);   // part | parts << 8 | slot << 16
    refine_ptile<DP, true, WIT, SM>(sm, X, C, ids, SUB, tend, supmin, m, ptile, res, keep, wit, cidx,
                                    cidx ? cidx + (1u << d) : nullptr, tmask, pinfo & 0xffu, (pinfo >> 8) & 0xffu,
                                    split ? split + (size_t)(pinfo >> 16) * 5 : nullptr);
}

// Ascending row ids of the kept rows (decoupled look-back over 8 rows per
// thread). Writes beyond `capacity` are dropped; the count is always exact.
// Compaction after the pre-pass: the sorted survivors (Morton key, row)
// whose row the pre-pass kept, in the same order, by a decoupled look-back
// over tiles of kScanTile entries claimed in order. It also clears those
// rows' keep bytes (the full refinement sets them again) and the layer-1
// cell index (rebuilt by the next gather), and writes the new count to
// res->refine_m. With fewer than kPreMinRows survivors the pre-pass kernel
// returned at once, and every entry is kept.
__global__ void __launch_bounds__(kScanThreads) k_pre_compact(const uint32_t* __restrict__ skey,
                                                              const uint32_t* __restrict__ sval, uint8_t* keep,
                                                              DevResult* res, unsigned long long* states,
                                                              uint32_t* tile_counter, uint32_t* okey, uint32_t* oval,
                                                              uint32_t* cidx, int64_t cidx_words)
{
    __shared__ uint32_t s_warp[kScanThreads / 32];
    __shared__ uint32_t s_tile, s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < cidx_words; i += (int64_t)gridDim.x * blockDim.x)
        cidx[i] = 0u;
    const uint32_t m = res->survivors;
    const bool all = (int64_t)m < kPreMinRows;   // the pre-pass did not run: every entry stays
    const uint32_t ntiles = (m + kScanTile - 1) / kScanTile;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= ntiles) return;
    const int64_t base = (int64_t)tile * kScanTile + (int64_t)tid * kScanItems;
    uint32_t flags = 0, rows[kScanItems];
#pragma unroll
    for (int jj = 0; jj < kScanItems; ++jj) {
        rows[jj] = 0u;
        if (base + jj < m) {
            rows[jj] = sval[base + jj];
            if (all || keep[rows[jj]]) flags |= 1u << jj;
        }
    }
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
    if (tid < 32) {
        const uint32_t prefix = lookback_prefix(states, tile, total, &res->err);
        if (tid == 0) s_prefix = prefix;
    }
    __syncthreads();
    uint32_t pos = s_prefix + before + x - v;
#pragma unroll
    for (int jj = 0; jj < kScanItems; ++jj) {
        if (flags & (1u << jj)) {
            okey[pos] = skey[base + jj];
            oval[pos] = rows[jj];
            keep[rows[jj]] = 0;
            ++pos;
        }
    }
    if (tile == ntiles - 1 && tid == 0) res->refine_m = s_prefix + total;
}

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

cudaError_t launch_gather(const Plan& p, cudaStream_t s, const uint32_t* mcount)
{
    const int64_t tiles = (p.n + kTQ - 1) / kTQ;
    if (tiles == 0) return cudaGetLastError();
    const bool v = (p.d % 4 == 0) && (p.ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(p.pts) & 15u) == 0);
    if (!mcount) mcount = &p.res->survivors;
    SKY_DISPATCH_DP(p.d, k_gather<DP><<<(unsigned)tiles, kTQ, 0, s>>>(p.pts, p.d, p.ld, v, p.sorted_val,
                                                                       p.sorted_key, mcount, p.params, p.X, p.C,
                                                                       p.ids, p.tmax, p.subcode, p.tile_end,
                                                                       p.cidx, p.tend_pre, p.tmask));
    return cudaGetLastError();
}

bool refine_mask_probe(int d)
{
    bool on = false;
    SKY_DISPATCH_DP(d, on = RefineMask<DP>::value);
    return on;
}

bool refine_prepass(const Plan& p)
{
    return kPreTiles > 0 && p.n >= kPreMinRows && p.tend_pre != nullptr && p.pre_states != nullptr;
}

namespace {

// One refinement launch over the tiles of the first *mcount sorted survivors,
// PG groups of 32 p's per CTA: TEND is each 128-point tile's last q-tile,
// SUPMIN the super-tile minima (NULL: none), ORDER the p-tile order (NULL:
// p-tile b in block b).
// Resident refinement CTAs of the GPU (the split rule's slots), at most
// 148 x 9 (the bound kSplitExtra and kSplitSlots are sized for).
template <int DP>
uint32_t refine_slots()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, n = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        sms = n > 0 ? n : 148;
    }
    return (uint32_t)std::min(sms * RefineMinBlocks<DP>::value, 148 * 9);
}

template <int DP, int PG>
void refine_launch(const Plan& p, cudaStream_t s, int64_t tiles, const uint32_t* tend, const uint32_t* supmin,
                   const uint32_t* order, const uint32_t* mcount, uint32_t min_m = 0, bool split = false)
{
    const int smem = (int)sizeof(SetSmem<DP, PG>);
    // split scans add up to 2 * slots entries (k_cost_order)
    const unsigned grid = (unsigned)((tiles + SetSmem<DP, PG>::kTiles - 1) / SetSmem<DP, PG>::kTiles) +
                          (split ? 2u * refine_slots<DP>() : 0u);
    const uint32_t* part = split ? p.tile_part : nullptr;
    uint32_t* sst = split ? p.split_state : nullptr;
    if (p.witness) {
        cudaFuncSetAttribute(k_refine<DP, true, PG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_refine<DP, true, PG><<<grid, kTQ + 32, smem, s>>>(p.X, p.C, p.ids, p.subcode, tend, supmin, order,
                                                             mcount, p.res, p.keep, p.witness, p.cidx, p.d, min_m,
                                                             p.tmask, part, sst);
    } else {
        cudaFuncSetAttribute(k_refine<DP, false, PG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_refine<DP, false, PG><<<grid, kTQ + 32, smem, s>>>(p.X, p.C, p.ids, p.subcode, tend, supmin, order,
                                                              mcount, p.res, p.keep, nullptr, p.cidx, p.d, min_m,
                                                              p.tmask, part, sst);
    }
}

}  // namespace

cudaError_t launch_refine(const Plan& p, cudaStream_t s)
{
    // p.keep was zeroed by the survivor pass (k_surv_flags)
    const int64_t tiles = (p.n + kTQ - 1) / kTQ;
    if (tiles == 0) return cudaGetLastError();
    const uint32_t* mcount = &p.res->survivors;
    if (refine_prepass(p)) {
        // the pre-pass: each p-tile against itself and the first kPreTiles
        // q-tiles (TEND clipped by the gather), no super-tile minima yet
        SKY_DISPATCH_DP(p.d, refine_launch<DP, kTQ / 32>(p, s, tiles, p.tend_pre, nullptr, nullptr, mcount,
                                                         (uint32_t)kPreMinRows));
        // its survivors, compacted in order into the sort's other buffers
        Plan q = p;
        const bool first = p.sorted_key == p.surv_key;
        q.sorted_key = first ? p.sort_key2 : p.surv_key;
        q.sorted_val = first ? p.sort_val2 : p.surv_idx;
        const int64_t ntiles = (p.n + kScanTile - 1) / kScanTile;
        // p.pre_states and p.lb_counter were zeroed by the call's first kernel
        k_pre_compact<<<(unsigned)ntiles, kScanThreads, 0, s>>>(p.sorted_key, p.sorted_val, p.keep, p.res,
                                                                p.pre_states, p.lb_counter + 2,
                                                                const_cast<uint32_t*>(q.sorted_key),
                                                                const_cast<uint32_t*>(q.sorted_val), p.cidx,
                                                                int64_t(2) << p.d);
        mcount = &p.res->refine_m;
        const cudaError_t e = launch_gather(q, s, mcount);
        if (e != cudaSuccess) return e;
    }
    SKY_DISPATCH_DP(p.d, {
        constexpr int DW = DP / 4;
        k_tile_cost<DW><<<(unsigned)((tiles + 7) / 8), 256, 0, s>>>(p.subcode, p.tmax, p.tile_end, mcount,
                                                                   p.tile_cost, p.supmin);
        constexpr int PG = RefineGroups<DP>::value;
        constexpr uint32_t NT = (uint32_t)SetSmem<DP, PG>::kTiles;
        const uint32_t slots = (SKY_REFINE_SPLIT_MIN_DP > 0 && DP >= SKY_REFINE_SPLIT_MIN_DP && NT == 1u &&
                                tiles <= (int64_t)SKY_REFINE_SPLIT_MAX_WAVES * refine_slots<DP>())
                                   ? refine_slots<DP>() : 0u;   // 0: no split
        k_cost_order<<<1, 1024, 0, s>>>(p.tile_cost, mcount, p.tile_order, NT, p.tile_part, p.split_state,
                                        slots);
        refine_launch<DP, PG>(p, s, tiles, p.tile_end, p.supmin, p.tile_order, mcount, 0, slots > 0u);
    });
    return cudaGetLastError();
}

cudaError_t launch_emit(const Plan& p, int32_t* out, int64_t capacity, cudaStream_t s)
{
    if (p.n == 0) return cudaGetLastError();
    const int64_t ntiles = (p.n + kScanTile - 1) / kScanTile;
    // p.lb_states and p.lb_counter were zeroed by the call's first kernel (k_clear)
    k_emit<<<(unsigned)ntiles, kScanThreads, 0, s>>>(p.keep, p.n, out, capacity, p.res, p.lb_states,
                                                     p.lb_counter + 1);
    return cudaGetLastError();
}

}  // namespace sky
