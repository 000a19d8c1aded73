// k_sort.cu -- stable LSD radix sort of the survivors by Morton key (sm_103a).
//
// The refinement compares tiles of points whose bounding boxes overlap; a
// Morton (Z-order) arrangement of the survivors makes consecutive points
// spatially close, so most tile pairs can be skipped by one box test. The
// sort is deterministic (stable, no atomics on the output positions): per
// 8-bit digit, (1) per-block digit histograms and digit totals, (2) one CTA
// per digit scanning its row of the [digit][block] matrix, (3) a stable scatter that ranks keys inside the
// block with warp match masks and writes digit runs contiguously. The number
// of survivors is read on the device, so no host synchronisation is needed.
#include <cstdint>

#include "sky_common.cuh"
#include "sky_internal.h"
#include "sky_sort.cuh"

namespace sky {

namespace {

using namespace radix;

__global__ void __launch_bounds__(kT) k_radix_hist(const uint32_t* __restrict__ keys, const DevResult* res,
                                                   int shift, uint32_t* hist, int64_t nblk_max,
                                                   uint32_t* digit_total)
{
    radix_hist_block(keys, res->survivors, shift, hist, nblk_max, digit_total, blockIdx.x);
}

// One CTA per digit: exclusive scan of that digit's row of block counts,
// offset by the total of all smaller digits.
__global__ void __launch_bounds__(kT) k_radix_scan(uint32_t* hist, const DevResult* res, int64_t nblk_max,
                                                   const uint32_t* digit_total)
{
    __shared__ uint32_t s_warp[kWarps];
    const uint32_t m = res->survivors;
    const int64_t nblk = ((int64_t)m + kTile - 1) / kTile;
    const int dg = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // offset = sum of the totals of digits below dg
    uint32_t v = tid < dg ? digit_total[tid] : 0u;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    uint32_t off = 0;
    for (int w = 0; w < kWarps; ++w) off += s_warp[w];
    __syncthreads();
    uint32_t* row = hist + (int64_t)dg * nblk_max;
    for (int64_t b0 = 0; b0 < nblk; b0 += kT) {
        const int64_t b = b0 + tid;
        const uint32_t c = b < nblk ? row[b] : 0u;
        uint32_t x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t before = 0, tot = 0;
        for (int w = 0; w < kWarps; ++w) {
            if (w < warp) before += s_warp[w];
            tot += s_warp[w];
        }
        if (b < nblk) row[b] = off + before + x - c;
        off += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kT) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                      const uint32_t* __restrict__ vin, uint32_t* kout,
                                                      uint32_t* vout, const DevResult* res, int shift,
                                                      const uint32_t* __restrict__ hist, int64_t nblk_max)
{
    radix_scatter_block(kin, vin, kout, vout, res->survivors, shift, hist, nblk_max, blockIdx.x);
}

}  // namespace

cudaError_t launch_sort(Plan& p, cudaStream_t s)
{
    const int bits = p.morton_bits * p.d;
    const int passes = (bits + 7) / 8;
    const uint32_t* kin = p.surv_key;
    const uint32_t* vin = p.surv_idx;
    uint32_t* kout = p.sort_key2;
    uint32_t* vout = p.sort_val2;
    const unsigned nblk = (unsigned)p.sort_blocks;
    // p.digit_total was zeroed by the call's first kernel (k_clear)
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = ps * 8;
        uint32_t* tot = p.digit_total + 256 * ps;
        k_radix_hist<<<nblk, kT, 0, s>>>(kin, p.res, shift, p.hist, p.sort_blocks, tot);
        k_radix_scan<<<256, kT, 0, s>>>(p.hist, p.res, p.sort_blocks, tot);
        k_radix_scatter<<<nblk, kT, 0, s>>>(kin, vin, kout, vout, p.res, shift, p.hist, p.sort_blocks);
        // ping-pong
        const uint32_t* tk = kout;
        const uint32_t* tv = vout;
        kout = const_cast<uint32_t*>(kin);
        vout = const_cast<uint32_t*>(vin);
        kin = tk;
        vin = tv;
    }
    p.sorted_val = vin;
    p.sorted_key = kin;
    return cudaGetLastError();
}

}  // namespace sky
