// k_refine.cu -- step (d): exact dominance refinement and compaction (sm_103a).
//
//   k_gather  lays the survivors out in Morton order: coordinates (padded to
//             a multiple of 4 floats), 7-bit per-dimension codes packed four
//             to a word, row ids, and per-tile bounding boxes.
//   k_refine  one CTA per tile of 128 survivors ("p" points, one per thread).
//             It lists the tiles whose lower box corner is <= the CTA's upper
//             box corner (no other tile can hold a dominator), streams them
//             into shared memory with 1-D bulk (TMA) copies, and tests every
//             pair: first a SIMD-within-a-word compare of the 7-bit codes
//             (code(q) <= code(p) in every dimension is necessary for q to
//             dominate p because the code map is monotone), then the exact
//             Definition 1 test on the float values. A point is dropped at
//             its first dominator; a warp leaves a tile as soon as all of its
//             points are dropped, a CTA as soon as all 128 are.
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
constexpr int kStages = 2;
constexpr int kList = 1024;
constexpr uint32_t kHigh = 0x80808080u;

template <int DP>
__global__ void __launch_bounds__(kTQ) k_gather(const float* __restrict__ pts, int d, int64_t ld, bool vec4,
                                                const uint32_t* __restrict__ sorted_idx, const DevResult* res,
                                                const float* __restrict__ params, float* X, uint32_t* C,
                                                int32_t* ids, float* bbox)
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

template <int DW>
__device__ __forceinline__ bool codes_le(const uint32_t (&P)[DW], const uint32_t* cq)
{
    // byte b of (P_w - q_w) keeps its high bit iff code_q[b] <= code_p[b]
    // (P_w = code_p | 0x80 per byte, codes < 128: no borrow crosses a byte)
    uint32_t r = kHigh;
    if constexpr (DW == 1) {
        r &= P[0] - cq[0];
    } else if constexpr (DW == 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(cq);
        r &= (P[0] - v.x) & (P[1] - v.y);
    } else if constexpr (DW == 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(cq);
        r &= (P[0] - v.x) & (P[1] - v.y) & (P[2] - v.z) & (P[3] - v.w);
    } else {
#pragma unroll
        for (int w = 0; w < DW; ++w) r &= P[w] - cq[w];
    }
    return r == kHigh;
}

template <int DP>
__device__ __forceinline__ bool dominates_exact(const float* xq, const float (&p)[DP])
{
    bool le = true, lt = false;
#pragma unroll
    for (int k = 0; k < DP; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(xq + k);
        le &= (v.x <= p[k]) & (v.y <= p[k + 1]) & (v.z <= p[k + 2]) & (v.w <= p[k + 3]);
        lt |= (v.x < p[k]) | (v.y < p[k + 1]) | (v.z < p[k + 2]) | (v.w < p[k + 3]);
    }
    return le && lt;
}

template <int DP>
__global__ void __launch_bounds__(kTQ) k_refine(const float* __restrict__ X, const uint32_t* __restrict__ C,
                                                const int32_t* __restrict__ ids, const float* __restrict__ BB,
                                                DevResult* res, uint8_t* keep)
{
    constexpr int DW = DP / 4;
    constexpr uint32_t kBytesX = kTQ * DP * sizeof(float);
    constexpr uint32_t kBytesC = kTQ * DW * sizeof(uint32_t);
    __shared__ __align__(128) float sX[kStages][kTQ * DP];
    __shared__ __align__(128) uint32_t sC[kStages][kTQ * DW];
    __shared__ __align__(8) uint64_t s_bar[kStages];
    __shared__ uint32_t s_list[kList];
    __shared__ uint32_t s_cnt;
    __shared__ uint32_t s_wc[kTQ / 32];

    const uint32_t m = res->survivors;
    const uint32_t T = (m + kTQ - 1) / kTQ;
    if (blockIdx.x >= T) return;
    uint32_t* err = &res->err;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&s_bar[s], 1);
        mbar_fence_init();
    }
    const int64_t j = (int64_t)blockIdx.x * kTQ + tid;
    const bool valid = j < m;
    float p[DP], pmax[DP];
    uint32_t P[DW];
#pragma unroll
    for (int k = 0; k < DP; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(X + j * DP + k);
        p[k] = v.x; p[k + 1] = v.y; p[k + 2] = v.z; p[k + 3] = v.w;
        const float4 u = *reinterpret_cast<const float4*>(BB + (int64_t)blockIdx.x * 2 * DP + DP + k);
        pmax[k] = u.x; pmax[k + 1] = u.y; pmax[k + 2] = u.z; pmax[k + 3] = u.w;
    }
#pragma unroll
    for (int w = 0; w < DW; ++w) P[w] = C[j * DW + w] | kHigh;
    bool active = valid;
    unsigned long long pairs = 0;
    uint32_t uses[kStages];
#pragma unroll
    for (int s = 0; s < kStages; ++s) uses[s] = 0;
    __syncthreads();

    bool stop = false, failed = false;
    uint32_t t0 = 0;
    while (t0 < T && !stop) {
        // ---- list the tiles that may hold a dominator of some point here
        if (tid == 0) s_cnt = 0;
        __syncthreads();
        while (t0 < T) {
            const uint32_t t = t0 + tid;
            bool ok = false;
            if (t < T) {
                ok = true;
                const float* lo = BB + (int64_t)t * 2 * DP;
#pragma unroll
                for (int k = 0; k < DP; ++k) ok &= __ldg(lo + k) <= pmax[k];
            }
            const uint32_t bal = __ballot_sync(kFull, ok);
            if (lane == 0) s_wc[warp] = __popc(bal);
            __syncthreads();
            uint32_t pos = s_cnt;
            for (int w = 0; w < warp; ++w) pos += s_wc[w];
            if (ok) s_list[pos + __popc(bal & lanemask_lt())] = t;
            __syncthreads();
            if (tid == 0) {
                uint32_t add = 0;
                for (int w = 0; w < kTQ / 32; ++w) add += s_wc[w];
                s_cnt += add;
            }
            __syncthreads();
            t0 += kTQ;
            if (s_cnt > kList - kTQ) break;
        }
        const uint32_t L = s_cnt;

        // ---- stream the listed tiles through two shared-memory stages
        if (tid == 0) {
            for (uint32_t i = 0; i < L && i < (uint32_t)kStages; ++i) {
                const uint32_t t = s_list[i];
                mbar_arrive_expect_tx(&s_bar[i], kBytesX + kBytesC);
                bulk_g2s(sX[i], X + (int64_t)t * kTQ * DP, kBytesX, &s_bar[i]);
                bulk_g2s(sC[i], C + (int64_t)t * kTQ * DW, kBytesC, &s_bar[i]);
            }
        }
        for (uint32_t i = 0; i < L; ++i) {
            const int s = (int)(i % kStages);
            const bool ok = mbar_wait(&s_bar[s], uses[s] & 1u, err);
            ++uses[s];
            if (__syncthreads_or(!ok)) { failed = true; stop = true; }
            if (!failed) {
                const uint32_t t = s_list[i];
                bool rel = active;
                if (rel) {
                    const float* lo = BB + (int64_t)t * 2 * DP;
#pragma unroll
                    for (int k = 0; k < DP; ++k) rel &= __ldg(lo + k) <= p[k];
                }
                if (__any_sync(kFull, rel)) {
                    const uint32_t* cq = sC[s];
                    const float* xq = sX[s];
                    for (int q0 = 0; q0 < kTQ; q0 += 32) {
                        if (rel) pairs += 32;
#pragma unroll 8
                        for (int q = q0; q < q0 + 32; ++q) {
                            if (codes_le<DW>(P, cq + q * DW) && rel) {
                                if (dominates_exact<DP>(xq + q * DP, p)) { active = false; rel = false; }
                            }
                        }
                        if (!__any_sync(kFull, rel)) break;
                    }
                }
                if (!__syncthreads_or(active)) stop = true;
            }
            if (stop) {
                // let the copy already in flight land before leaving
                if (tid == 0 && i + 1 < L) {
                    const int s2 = (int)((i + 1) % kStages);
                    mbar_wait(&s_bar[s2], uses[s2] & 1u, nullptr);
                }
                break;
            }
            if (tid == 0 && i + kStages < L) {
                const uint32_t t = s_list[i + kStages];
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&s_bar[s], kBytesX + kBytesC);
                bulk_g2s(sX[s], X + (int64_t)t * kTQ * DP, kBytesX, &s_bar[s]);
                bulk_g2s(sC[s], C + (int64_t)t * kTQ * DW, kBytesC, &s_bar[s]);
            }
        }
        __syncthreads();
    }
    if (valid && active && !failed) keep[ids[j]] = 1;
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kFull, pairs, o);
    if (lane == 0 && pairs) atomicAdd(&res->pairs, pairs);
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
                                                                       p.params, p.X, p.C, p.ids, p.bbox));
    return cudaGetLastError();
}

cudaError_t launch_refine(const Plan& p, cudaStream_t s)
{
    cudaMemsetAsync(p.keep, 0, (size_t)p.n, s);
    const int64_t tiles = (p.n + kTQ - 1) / kTQ;
    if (tiles == 0) return cudaGetLastError();
    SKY_DISPATCH_DP(p.d, k_refine<DP><<<(unsigned)tiles, kTQ, 0, s>>>(p.X, p.C, p.ids, p.bbox, p.res, p.keep));
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
