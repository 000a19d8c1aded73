// k_witness.cu -- witness mode of the single-set path (a checking aid, not part
// of the hot path): for every point the path drops, the row of a point that
// dominates it (Definition 1), so that a caller can verify every dropped point
// in O(n d) on the host.
//
// Where a point is dropped, and where its witness comes from:
//   step (c), dominated cell  cell c is dominated when some occupied cell c'
//                             has c'[k] < c[k] in every dimension (Def. 3);
//                             then any point of c' is strictly smaller than
//                             every point of c in every dimension (the value ->
//                             column map is monotone). Found here from a
//                             per-cell representative row and its prefix over
//                             the d dimensions (the same box identity as the
//                             prefix-OR, carrying a row instead of a bit),
//                             read at c - (1, ..., 1).
//   step (c'), proposals      the snapped proposal (a real row) that dominates
//                             the point, re-tested here by Definition 1.
//   step (d), refinement      the surviving point q whose test removed p,
//                             written by the refinement kernel itself.
// A point that step (c) dropped but for which neither source gives a witness
// gets -2, which the caller's check reports as an error of step (c).
#include <cstdint>

#include "sky_common.cuh"
#include "sky_internal.h"

namespace sky {

namespace {

constexpr int kWitThreads = 256;

// rep[ckey[i]] = i: every occupied cell receives the row of one of its points
// (concurrent plain stores of rows of the same cell leave one of them). The
// keys are below the cell count; the mask (a no-op for them) keeps the store
// inside rep if the map pass gave up before writing some keys.
__global__ void __launch_bounds__(kWitThreads) k_wit_rep(const uint32_t* __restrict__ ckey, int64_t n, uint32_t cmask,
                                                         int32_t* rep)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        rep[ckey[i] & cmask] = (int32_t)i;
}

// Inclusive prefix along dimension k: walking each line of 2^log2g cells
// (stride 2^(log2g k)) upwards, an empty cell (-1) takes the value of the
// nearest non-empty cell below it on the line. After the passes over all d
// dimensions, rep[c] is the row of a point of some occupied cell c' <= c
// (componentwise), or -1 when there is none.
__global__ void __launch_bounds__(kWitThreads) k_wit_prefix(int32_t* rep, int64_t cells, int log2g, int k)
{
    const int64_t G = int64_t(1) << log2g;
    const int64_t stride = int64_t(1) << (log2g * k);
    const int64_t lines = cells / G;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < lines; l += step) {
        const int64_t lo = l % stride, hi = l / stride;
        int32_t* line = rep + hi * stride * G + lo;
        int32_t cur = -1;
        for (int64_t j = 0; j < G; ++j) {
            const int32_t v = line[j * stride];
            if (v >= 0) cur = v;
            else if (cur >= 0) line[j * stride] = cur;
        }
    }
}

// Definition 1 on two rows of the input.
__device__ __forceinline__ bool row_dominates(const float* q, const float* p, int d)
{
    bool le = true, lt = false;
    for (int k = 0; k < d; ++k) {
        le &= q[k] <= p[k];
        lt |= q[k] < p[k];
    }
    return le && lt;
}

// Witness of every point whose survivor flag (step c) is clear.
__global__ void __launch_bounds__(kWitThreads) k_wit_dropped(const float* __restrict__ pts, int64_t n, int d,
                                                             int64_t ld, int log2g,
                                                             const uint32_t* __restrict__ ckey,
                                                             const uint32_t* __restrict__ sflags,
                                                             const int32_t* __restrict__ prerep,
                                                             const unsigned long long* __restrict__ snap, int n_prop,
                                                             int32_t* wit)
{
    const uint32_t ones = ones_key(log2g, d);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if ((sflags[i >> 5] >> (i & 31)) & 1u) continue;   // a survivor of step (c)
        const uint32_t key = ckey[i];
        int32_t w = -2;
        if (log2g > 0 && all_columns_positive(key, log2g, d)) {
            const int32_t r = prerep[(key - ones) & (uint32_t)((uint64_t(1) << (log2g * d)) - 1u)];
            if (r >= 0) w = r;
        }
        for (int j = 0; j < n_prop && w < 0; ++j) {
            if (snap[j] == ~0ull) continue;
            const int64_t row = (int64_t)(snap[j] & 0xffffffffull);
            if (row_dominates(pts + row * ld, pts + i * ld, d)) w = (int32_t)row;
        }
        wit[i] = w;
    }
}

unsigned grid_of(int64_t work)
{
    const int64_t b = (work + kWitThreads - 1) / kWitThreads;
    return (unsigned)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

}  // namespace

cudaError_t launch_witness_cells(const Plan& p, int32_t* rep, int n_prop, cudaStream_t s)
{
    if (p.n == 0) return cudaGetLastError();
    const int64_t cells = int64_t(1) << (p.log2g * p.d);
    cudaError_t e = cudaMemsetAsync(rep, 0xff, sizeof(int32_t) * (size_t)cells, s);
    if (e != cudaSuccess) return e;
    k_wit_rep<<<grid_of(p.n), kWitThreads, 0, s>>>(p.ckey, p.n, (uint32_t)(cells - 1), rep);
    if (p.log2g > 0)
        for (int k = 0; k < p.d; ++k)
            k_wit_prefix<<<grid_of(cells >> p.log2g), kWitThreads, 0, s>>>(rep, cells, p.log2g, k);
    k_wit_dropped<<<grid_of(p.n), kWitThreads, 0, s>>>(p.pts, p.n, p.d, p.ld, p.log2g, p.ckey, p.sflags, rep,
                                                      p.snap, n_prop, p.witness);
    return cudaGetLastError();
}

}  // namespace sky
