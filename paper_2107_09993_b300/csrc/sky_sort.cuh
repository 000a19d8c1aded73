// sky_sort.cuh -- per-block pieces of the stable LSD radix sort (8-bit
// digits), shared by the single-set sort (k_sort.cu) and the batched one
// (k_batched.cu). Device code only.
#pragma once

#include <cstdint>

#include "sky_common.cuh"
#include "sky_internal.h"

namespace sky {
namespace radix {

constexpr int kT = kSortThreads;
constexpr int kI = kSortItems;
constexpr int kTile = kSortTile;
constexpr int kWarps = kT / 32;

// Digit histogram of sort block `blk` (kTile keys) of an m-key sequence.
__device__ __forceinline__ void radix_hist_block(const uint32_t* __restrict__ keys, uint32_t m, int shift,
                                                 uint32_t* hist, int64_t nblk_max, uint32_t* digit_total,
                                                 uint32_t blk)
{
    __shared__ uint32_t s_h[256];
    const int64_t base = (int64_t)blk * kTile;
    if (base >= m) return;
    s_h[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kI; ++r) {
        const int64_t i = base + r * kT + threadIdx.x;
        if (i < m) atomicAdd(&s_h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    const uint32_t c = s_h[threadIdx.x];
    hist[(int64_t)threadIdx.x * nblk_max + blk] = c;
    if (c) atomicAdd(&digit_total[threadIdx.x], c);
}

// Stable scatter of sort block `blk` to the offsets in `hist` (already scanned).
__device__ __forceinline__ void radix_scatter_block(const uint32_t* __restrict__ kin,
                                                    const uint32_t* __restrict__ vin, uint32_t* kout,
                                                    uint32_t* vout, uint32_t m, int shift,
                                                    const uint32_t* __restrict__ hist, int64_t nblk_max,
                                                    uint32_t blk)
{
    __shared__ uint32_t s_wcnt[kWarps][256];
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_start[256];
    __shared__ uint32_t s_key[kTile];
    __shared__ uint32_t s_val[kTile];
    __shared__ uint32_t s_warp[kWarps];
    const int64_t base = (int64_t)blk * kTile;
    if (base >= m) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int w = 0; w < kWarps; ++w) s_wcnt[w][tid] = 0;
    s_run[tid] = 0;
    __syncthreads();

    uint32_t key[kI], val[kI], rank[kI];
#pragma unroll
    for (int r = 0; r < kI; ++r) {
        const int64_t i = base + r * kT + tid;
        const bool valid = i < m;
        key[r] = valid ? kin[i] : 0u;
        val[r] = valid ? vin[i] : 0u;
        const uint32_t digit = valid ? ((key[r] >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(kFull, digit);
        const uint32_t below = __popc(peers & lanemask_lt());
        const bool leader = (__ffs(peers) - 1) == lane;
        if (valid && leader) s_wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = s_run[digit];
            for (int w = 0; w < warp; ++w) pre += s_wcnt[w][digit];
            rank[r] = pre + below;
        }
        __syncthreads();
        {
            uint32_t tot = 0;
            for (int w = 0; w < kWarps; ++w) {
                tot += s_wcnt[w][tid];
                s_wcnt[w][tid] = 0;
            }
            s_run[tid] += tot;
        }
        __syncthreads();
    }
    // local digit starts (exclusive scan of the block's digit counts)
    {
        const uint32_t c = s_run[tid];
        uint32_t x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += s_warp[w];
        s_start[tid] = before + x - c;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kI; ++r) {
        const int64_t i = base + r * kT + tid;
        if (i < m) {
            const uint32_t digit = (key[r] >> shift) & 255u;
            const uint32_t pos = s_start[digit] + rank[r];
            s_key[pos] = key[r];
            s_val[pos] = val[r];
        }
    }
    __syncthreads();
    const int64_t cnt = (m - base) < kTile ? (m - base) : kTile;
    for (int j = tid; j < cnt; j += kT) {
        const uint32_t k = s_key[j];
        const uint32_t digit = (k >> shift) & 255u;
        const uint32_t g = hist[(int64_t)digit * nblk_max + blk] + (j - s_start[digit]);
        kout[g] = k;
        vout[g] = s_val[j];
    }
}

}  // namespace radix
}  // namespace sky
