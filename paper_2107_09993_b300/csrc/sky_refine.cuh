// sky_refine.cuh -- the refinement of step (d) for one p-tile, shared by the
// single-set kernel (k_refine.cu) and the batched persistent kernel
// (k_batched.cu). Device code only.
#pragma once

#include <cstdint>

#include "sky_common.cuh"
#include "sky_internal.h"

namespace sky {
namespace refine {

constexpr int kTQ = kRefineTile;
constexpr int kSubSlots = kTQ / 32 + 1;   // sub-tile minima + the whole-tile minimum
constexpr uint32_t kHigh = 0x80808080u;

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

// Refines p-tile `ptile` (< ceil(m / 128)) of one point set. Called by all
// kTQ + 32 threads of the CTA with the CTA's shared memory; leaves the
// shared memory free for the next call (barriers invalidated).
template <int DP>
__device__ __forceinline__ void refine_ptile(RefineSmem<DP>& sm, const float* __restrict__ X,
                                             const uint32_t* __restrict__ C, const int32_t* __restrict__ ids,
                                             const uint32_t* __restrict__ SUB, uint32_t m, uint32_t ptile,
                                             DevResult* res, uint8_t* keep)
{
    constexpr int DW = DP / 4;
    constexpr int NG = kTQ / 32;
    constexpr int S = kRingStages;
    constexpr uint32_t kBytesX = kTQ * DP * sizeof(float);
    constexpr uint32_t kBytesC = kTQ * DW * sizeof(uint32_t);
    const uint32_t T = (m + kTQ - 1) / kTQ;
    uint32_t* err = &res->err;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t pbase = (int64_t)ptile * kTQ;
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
        uint32_t hits = 0, exact = 0;   // per lane
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
                            ++hits;
                            uint32_t eq = 0;
#pragma unroll
                            for (int w = 0; w < DW; ++w) eq |= has_zero_byte(D[w] ^ kHigh);
                            bool dom = true;   // strictly lower code everywhere: q < p everywhere
                            if (eq) {
                                ++exact;
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
        const uint32_t wh = __reduce_add_sync(kFull, hits), we = __reduce_add_sync(kFull, exact);
        if (lane == 0 && wh) atomicAdd(&res->hits, (unsigned long long)wh);
        if (lane == 0 && we) atomicAdd(&res->exact, (unsigned long long)we);
    }
    __syncthreads();
    if (tid < kTQ && pbase + tid < m && !sm.failed && ((sm.livemask[tid >> 5] >> (tid & 31)) & 1u))
        keep[ids[pbase + tid]] = 1;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_inval(&sm.full[s]);
            mbar_inval(&sm.empty[s]);
        }
    }
    __syncthreads();
}

}  // namespace refine
}  // namespace sky
