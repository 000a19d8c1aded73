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
#include "sky_refine.cuh"

namespace sky {

namespace {

using namespace refine;

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

template <int DP>
__global__ void __launch_bounds__(kTQ + 32) k_refine(const float* __restrict__ X, const uint32_t* __restrict__ C,
                                                     const int32_t* __restrict__ ids,
                                                     const uint32_t* __restrict__ SUB, DevResult* res,
                                                     uint8_t* keep)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    RefineSmem<DP>& sm = *reinterpret_cast<RefineSmem<DP>*>(smem_raw);
    const uint32_t m = res->survivors;
    if (blockIdx.x >= (m + kTQ - 1) / kTQ) return;
    refine_ptile<DP>(sm, X, C, ids, SUB, m, blockIdx.x, res, keep);
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
