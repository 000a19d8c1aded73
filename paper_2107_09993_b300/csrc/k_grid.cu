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
#include <algorithm>
#include <cfloat>
#include <cstdint>

#include <cooperative_groups.h>

#include "sky_common.cuh"
#include "sky_internal.h"

namespace sky {

namespace cg = cooperative_groups;

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

// Clears the call's result block and the occupancy bitmap in one launch (two
// memset nodes in a CUDA graph cost several microseconds of scheduling each).
// Both start 256-byte aligned; the bitmap is cleared in 16-byte stores.
// What a call zeroes before its first step: the result block, the bitmap
// and, when the plan has them, the sort's digit totals and the compaction's
// look-back state (these would otherwise be memset nodes of their own, a few
// microseconds each in a graph). Thread tid of nthr.
struct ClearSet {
    DevResult* res = nullptr;
    uint32_t* occ = nullptr;
    int64_t words = 0;
    uint32_t* digit_total = nullptr;           // [4][256]
    uint32_t* lb_counter = nullptr;            // [4]
    unsigned long long* lb_states = nullptr;   // [lb_tiles]
    int64_t lb_tiles = 0;
    uint32_t* cidx = nullptr;                  // layer-1 cell index of the refinement
    int64_t cidx_words = 0;                    // (a multiple of 4)
    unsigned long long* pre_states = nullptr;  // [lb_tiles] the refinement pre-pass's look-back states
};

__device__ __forceinline__ void clear_set(const ClearSet& c, int64_t tid, int64_t nthr)
{
    constexpr int kResWords = (int)(sizeof(DevResult) / sizeof(uint32_t));
    if (tid < kResWords) reinterpret_cast<uint32_t*>(c.res)[tid] = 0u;
    if (c.digit_total)
        for (int64_t i = tid; i < 4 * 256; i += nthr) c.digit_total[i] = 0u;
    if (c.lb_counter && tid < 4) c.lb_counter[tid] = 0u;
    if (c.lb_states)
        for (int64_t i = tid; i < c.lb_tiles; i += nthr) c.lb_states[i] = 0ull;
    const int64_t q = c.words / 4;
    uint4* o4 = reinterpret_cast<uint4*>(c.occ);
    for (int64_t i = tid; i < q; i += nthr) o4[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t i = q * 4 + tid; i < c.words; i += nthr) c.occ[i] = 0u;
    uint4* x4 = reinterpret_cast<uint4*>(c.cidx);
    for (int64_t i = tid; i < c.cidx_words / 4; i += nthr) x4[i] = make_uint4(0u, 0u, 0u, 0u);
    if (c.pre_states)
        for (int64_t i = tid; i < c.lb_tiles; i += nthr) c.pre_states[i] = 0ull;
}

__global__ void __launch_bounds__(kThreads) k_clear(ClearSet c)
{
    clear_set(c, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Automatic map, decided on the strided sample of rows 0, t, 2t, ... < n
// with t = ceil(n / kDecideSample): the unit-cube map (Eq. 1 as printed) when
// every sampled dimension lies in [0, 1] and spans at least half of it,
// otherwise min / max scales from the sample's range. Rows outside that range
// clamp into the edge columns, so the map stays monotone -- all that pruning
// and the refinement's codes need. The sample's min / max are exact, so the
// decision does not depend on the reduction order.
//
// One cluster of kDecideCluster CTAs, one sampled row per thread: CTA r reads
// the r-th contiguous slice of the sample (its rows span 1/kDecideCluster of
// the input, so each SM walks fewer pages), reduces it in shared memory, and
// CTA 0 combines the slices through distributed shared memory. (A single CTA
// walking all 4,096 rows was latency-bound: 40 us on a 640 MB input.)
constexpr int kDecideSample = 4096;
constexpr int kDecideCluster = 8;
constexpr int kDecideThreads = kDecideSample / kDecideCluster;   // 512

template <int DP>
__global__ void __cluster_dims__(kDecideCluster, 1, 1) __launch_bounds__(kDecideThreads)
    k_sample_params(const float* __restrict__ pts, int64_t n, int d, int64_t ld, bool vec4, int log2g, int mbits,
                    uint32_t* mm_min, uint32_t* mm_max, float* params, ClearSet clear)
{
    __shared__ float s_mn[kDecideThreads / 32][DP], s_mx[kDecideThreads / 32][DP];
    __shared__ float c_mn[DP], c_mx[DP];   // this CTA's slice; read by CTA 0 of the cluster
    __shared__ int s_bad;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t t = (n + kDecideSample - 1) / kDecideSample;
    if (t < 1) t = 1;
    const int64_t rows = (n + t - 1) / t;
    const int64_t r = (int64_t)rank * kDecideThreads + tid;
    float x[DP];
    if (r < rows) {
        load_row<DP>(pts + r * t * ld, d, vec4, x);
#pragma unroll
        for (int k = 0; k < DP; ++k)
            if (k >= d) x[k] = NAN;
    } else {
#pragma unroll
        for (int k = 0; k < DP; ++k) x[k] = NAN;   // fminf / fmaxf ignore NaN
    }
    float mn[DP], mx[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) {
        mn[k] = x[k];
        mx[k] = x[k];
        for (int o = 16; o > 0; o >>= 1) {
            mn[k] = fminf(mn[k], __shfl_xor_sync(kFull, mn[k], o));
            mx[k] = fmaxf(mx[k], __shfl_xor_sync(kFull, mx[k], o));
        }
        if (lane == 0) { s_mn[warp][k] = mn[k]; s_mx[warp][k] = mx[k]; }
    }
    if (tid == 0) s_bad = 0;
    // what k_clear would zero, when this launch replaces it (res != NULL)
    if (clear.res) clear_set(clear, r, (int64_t)kDecideSample);
    __syncthreads();
    if (tid < DP) {
        float lo = NAN, hi = NAN;
        for (int w = 0; w < kDecideThreads / 32; ++w) { lo = fminf(lo, s_mn[w][tid]); hi = fmaxf(hi, s_mx[w][tid]); }
        c_mn[tid] = lo;
        c_mx[tid] = hi;
    }
    cluster.sync();   // every slice is in its CTA's shared memory
    if (rank == 0) {
        if (tid < d) {
            float lo = INFINITY, hi = -INFINITY;
            for (int q = 0; q < kDecideCluster; ++q) {
                lo = fminf(lo, *cluster.map_shared_rank(&c_mn[tid], q));
                hi = fmaxf(hi, *cluster.map_shared_rank(&c_mx[tid], q));
            }
            mm_min[tid] = float_to_ordered(lo);
            mm_max[tid] = float_to_ordered(hi);
            const bool unit_ok = (lo >= 0.0f) && (hi <= 1.0f) && (__fsub_rn(hi, lo) >= 0.5f);
            if (!unit_ok) atomicOr(&s_bad, 1);
        }
    }
    cluster.sync();   // CTA 0 has read every slice; the other CTAs may exit
    if (rank == 0) {
        __syncthreads();
        if (tid < kMaxDim) write_params(tid, d, log2g, mbits, s_bad != 0, mm_min, mm_max, params);
    }
}

// ---------------------------------------------------------------------------
// Steps (a)+(b). One point -> (cell key, Morton key) -> bit. The bitmap OR
// is fire-and-forget; when a whole warp hits one word (hot cells of
// correlated data) the bits are merged first and one lane issues it.
//
// Morton key: bit l of dimension k's column goes to bit l * d + k. When
// d - 1 >= mbits, one multiply spreads all mbits bits of a column at once:
// q * sum_j 2^(j (d-1)) places bit l at l + j (d-1) for every j < mbits;
// those positions are distinct (base-(d-1) digits), so nothing carries, and
// position l * d holds exactly bit l (the j = l term). A mask keeps those.
struct MortonSpread {
    uint32_t magic, mask;
    __device__ __forceinline__ MortonSpread(int d, int mbits) : magic(0u), mask(0u)
    {
        if (d - 1 >= mbits) {
            for (int j = 0; j < mbits; ++j) {
                magic |= 1u << (j * (d - 1));
                mask |= 1u << (j * d);
            }
        }
    }
    __device__ __forceinline__ bool fast() const { return mask != 0u; }
};

// Where the occupancy bits go. All of them keep every bit; they differ in how
// many atomics hit one word.
//   MarkGlobal  fire-and-forget atomicOr on the bitmap
//   MarkPrivate a block-private copy of a small bitmap in shared memory
//   MarkCheck   the bitmap, but a mark whose bits are already set (read
//               through L1; stale is fine: bits are only ever set) sends no
//               atomic. Many rows of clustered data land on few cells, whose
//               words then take no further atomics. A block looks only when
//               the rows of its first chunk repeat words inside their warps
//               (clustered data); for spread data the extra load per row
//               would only add latency.
//   MarkNone    no marking (a pass that only needs the keys again)
// (A shared-memory cache of bitmap words measured slower on clustered data
// than both global variants.)
struct MarkGlobal {
    static constexpr bool kNone = false;
    static constexpr bool kByte = false;
    uint32_t* occ;
    __device__ __forceinline__ void mark(uint32_t word, uint32_t bits) const { atomicOr(occ + word, bits); }
};
// The private marker looks before it ORs: a bit already set costs one shared
// load, not a serialised atomic on the same address.
struct MarkPrivate {
    static constexpr bool kNone = false;
    static constexpr bool kByte = false;
    uint32_t* s_occ;   // shared memory
    __device__ __forceinline__ void mark(uint32_t word, uint32_t bits) const
    {
        if ((s_occ[word] & bits) != bits) atomicOr(s_occ + word, bits);
    }
};
struct MarkNone {
    static constexpr bool kNone = true;
    static constexpr bool kByte = false;
    __device__ __forceinline__ void mark(uint32_t, uint32_t) const {}
};
// MarkByte: one byte per cell, set by a plain store (no read-modify-write
// at L2); k_occ_pack builds the bitmap from the bytes after the pass.
struct MarkByte {
    static constexpr bool kNone = false;
    static constexpr bool kByte = true;
    uint8_t* occb;
    bool check;        // block-uniform: look before storing (clustered data)
    __device__ __forceinline__ void mark_key(uint32_t key) const
    {
        if (check && __ldca(occb + key) != 0) return;
        occb[key] = 1;
    }
    __device__ __forceinline__ void mark(uint32_t, uint32_t) const {}
};
struct MarkCheck {
    static constexpr bool kNone = false;
    static constexpr bool kByte = false;
    uint32_t* occ;
    bool check;        // block-uniform
    __device__ __forceinline__ void mark(uint32_t word, uint32_t bits) const
    {
        if (check && (__ldca(occ + word) & bits) == bits) return;
        atomicOr(occ + word, bits);
    }
};

// The key is built as key * G + c (G a runtime power of two: an integer
// multiply-add, off the integer ALU pipe that the clamps and masks use).
// EXACT: d == DP (no per-dimension guards); COARSE: the Morton grid is no
// finer than the cell grid, so the Morton column is the cell column shifted.
template <int DP, bool EXACT, bool COARSE>
__device__ __forceinline__ void map_keys(const float (&x)[DP], int d, int log2g, int mbits, const MortonSpread& ms,
                                         const float* s_off, const float* s_sc, const float* s_ms,
                                         uint32_t& key_out, uint32_t& code_out, bool& bad)
{
    const int dd = EXACT ? DP : d;
    const uint32_t G = 1u << log2g;
    const uint32_t M = 1u << mbits;
    uint32_t key = 0;
    uint32_t mq[DP];
    float nanacc = 0.0f;   // x * 0 is NaN exactly when x is infinite or NaN
#pragma unroll
    for (int k = DP - 1; k >= 0; --k) {
        mq[k] = 0;
        if (k < dd) {
            nanacc = fmaf(x[k], 0.0f, nanacc);
            const uint32_t c = column_of(x[k], s_off[k], s_sc[k], G);
            key = key * G + c;
            mq[k] = COARSE ? (c >> (log2g - mbits)) : column_of(x[k], s_off[k], s_ms[k], M);
        }
    }
    bad |= nanacc != nanacc;
    uint32_t code = 0;
    if (ms.fast()) {
#pragma unroll
        for (int k = 0; k < DP; ++k)
            if (k < dd) code += ((mq[k] * ms.magic) & ms.mask) << k;   // disjoint bits: + is |
    } else {
        for (int l = mbits - 1; l >= 0; --l)
#pragma unroll
            for (int k = DP - 1; k >= 0; --k)
                if (k < dd) code = (code << 1) | ((mq[k] >> l) & 1u);
    }
    key_out = key;
    code_out = code;
}

// `converged`: every lane of the warp calls together (no activemask query).
// The two shape tests are uniform across the grid, so each call runs one
// specialised body.
// Writes a row's keys and marks its cell.
// Marks a row's cell; when a whole warp hits one word the bits are merged
// first and one lane issues the mark.
template <bool converged, class Marker>
__device__ __forceinline__ void mark_cell(uint32_t key, const Marker& marker, uint32_t* dups = nullptr)
{
    const uint32_t word = key >> 5;
    if (dups) *dups += __popc(__match_any_sync(kFull, word)) > 1 ? 1u : 0u;   // converged callers only
    if constexpr (Marker::kByte) {
        marker.mark_key(key);
        return;
    }
    const uint32_t bit = 1u << (key & 31u);
    const uint32_t am = converged ? kFull : __activemask();
    const int leader = converged ? 0 : __ffs(am) - 1;
    const uint32_t w0 = __shfl_sync(am, word, leader);
    if (__all_sync(am, word == w0)) {
        const uint32_t bits = __reduce_or_sync(am, bit);
        if ((int)(threadIdx.x & 31) == leader) marker.mark(word, bits);
    } else {
        marker.mark(word, bit);
    }
}

// Writes a row's keys (when the pass keeps keys) and marks its cell.
template <bool converged, class Marker>
__device__ __forceinline__ void store_mark(uint32_t key, uint32_t code, int64_t row, uint32_t* __restrict__ ckey,
                                           uint32_t* __restrict__ mkey, const Marker& marker,
                                           uint32_t* dups = nullptr)
{
    if (ckey) {   // a marking pass that needs no keys passes none
        ckey[row] = key;
        mkey[row] = code;
    }
    if (!Marker::kNone) mark_cell<converged>(key, marker, dups);
}

template <int DP, bool converged, class Marker>
__device__ __forceinline__ void map_one(const float (&x)[DP], int d, int log2g, int mbits, const MortonSpread& ms,
                                        const float* s_off, const float* s_sc, const float* s_ms, int64_t row,
                                        uint32_t* __restrict__ ckey, uint32_t* __restrict__ mkey,
                                        Marker marker, bool& bad, uint32_t* dups = nullptr)
{
    uint32_t key, code;
    if (d == DP) {
        if (mbits <= log2g) map_keys<DP, true, true>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, key, code, bad);
        else map_keys<DP, true, false>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, key, code, bad);
    } else {
        if (mbits <= log2g) map_keys<DP, false, true>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, key, code, bad);
        else map_keys<DP, false, false>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, key, code, bad);
    }
    store_mark<converged>(key, code, row, ckey, mkey, marker, dups);
}

// Unit-cube map (offset 0, scale G in every dimension; Eq. 1 as printed),
// d == DP a multiple of 4, multiply-spread Morton keys: the keys of one row
// read from its shared-memory stage. The four-float pieces of the row are
// visited starting at piece `rot`, so that the eight threads of a 128-byte
// shared-memory phase read eight different bank groups (rows of 32 or 64
// bytes would otherwise collide 2- or 4-way); the key and the Morton key are
// ORs of shifted per-piece values, so the visiting order does not matter.
// x * G here equals (x - 0) * G of the general map bit for bit.
//
// One conversion per dimension: the column in the finer of the two grids
// (2^fb columns, fb = max(log2g, mbits)), clamped to 2^fb - 1; the column in
// the coarser grid is that column shifted right by the difference s. Exact:
// x * 2^fb and x * 2^(fb-s) are both exact products (power-of-two scales),
// so floor(x * 2^fb) >> s == floor(x * 2^(fb-s)); clamping commutes with the
// shift (2^fb - 1 >> s == 2^(fb-s) - 1); negative, NaN and overflowing
// values convert to 0 or saturate in both grids alike.
template <int DP, bool COARSE>
__device__ __forceinline__ void map_keys_unit(const float* __restrict__ r, int rot, int log2g, int mbits,
                                              const MortonSpread& ms, uint32_t& key_out, uint32_t& code_out,
                                              bool& bad)
{
    constexpr int NQ = DP / 4;
    const int fbits = COARSE ? log2g : mbits;
    const int sh = COARSE ? log2g - mbits : mbits - log2g;
    const float F = (float)(1u << fbits);
    const uint32_t Fm1 = (1u << fbits) - 1u;
    const uint32_t G = 1u << log2g;
    // Morton spread of dimension 4q + i: (mq * (magic << i)) & (mask << i)
    const uint32_t mg[4] = {ms.magic, ms.magic << 1, ms.magic << 2, ms.magic << 3};
    const uint32_t mk[4] = {ms.mask, ms.mask << 1, ms.mask << 2, ms.mask << 3};
    uint32_t key = 0, code = 0;
    float nanacc = 0.0f;   // x * 0 is NaN exactly when x is infinite or NaN
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        const int q = (j + rot) % NQ;
        const float4 v = *reinterpret_cast<const float4*>(r + 4 * q);
        const float xs[4] = {v.x, v.y, v.z, v.w};
        uint32_t kq = 0, cq = 0;
#pragma unroll
        for (int i = 3; i >= 0; --i) {
            nanacc = fmaf(xs[i], 0.0f, nanacc);
            uint32_t f = __float2uint_rd(__fmul_rn(xs[i], F));
            f = f < Fm1 ? f : Fm1;
            const uint32_t c = COARSE ? f : f >> sh;
            const uint32_t mq = COARSE ? f >> sh : f;
            kq = kq * G + c;                      // dimension 4q + 3 most significant
            cq |= (mq * mg[i]) & mk[i];
        }
        key |= kq << (log2g * 4 * q);
        code |= cq << (4 * q);
    }
    bad |= nanacc != nanacc;
    key_out = key;
    code_out = code;
}

// Small grids (at most kPrivWords words) are marked in a private copy of the
// bitmap in shared memory -- many rows share few words there, and global
// atomics on them would serialise -- which each block then writes to its row
// of `stage`; k_occ_merge ORs the rows into the bitmap.
// Marking modes of the map kernels: the bitmap itself (through the word cache
// in the streaming kernel), a private shared-memory copy of a small bitmap,
// or no marking at all (a second pass that only needs the keys again).
enum MapMark { kMarkCheck = 0, kMarkSmall = 1, kMarkNone = 2, kMarkByte = 3 };

template <int DP, int MODE>
__global__ void __launch_bounds__(kThreads) k_map_mark_plain(const float* __restrict__ pts, int64_t n,
                                                             int d, int64_t ld, bool vec4, int log2g, int mbits,
                                                             const float* params, uint32_t* ckey,
                                                             uint32_t* mkey, uint32_t* occ, uint32_t* err,
                                                             uint32_t* stage, int64_t words)
{
    extern __shared__ __align__(16) uint32_t s_occ[];   // [words] in kMarkSmall mode
    __shared__ float s_off[kMaxDim], s_sc[kMaxDim], s_ms[kMaxDim];
    if (threadIdx.x < kMaxDim) {
        s_off[threadIdx.x] = params[threadIdx.x];
        s_sc[threadIdx.x] = params[16 + threadIdx.x];
        s_ms[threadIdx.x] = params[48 + threadIdx.x];
    }
    if (MODE == kMarkSmall)
        for (int64_t w = threadIdx.x; w < words; w += blockDim.x) s_occ[w] = 0u;
    __syncthreads();
    const MortonSpread ms(d, mbits);
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_round = ((n + 31) / 32) * 32;   // whole warps stay in the loop together
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        if (i < n) {
            float x[DP];
            load_row<DP>(pts + i * ld, d, vec4, x);
            if (MODE == kMarkSmall)
                map_one<DP, false>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, i, ckey, mkey, MarkPrivate{s_occ}, bad);
            else if (MODE == kMarkNone)
                map_one<DP, false>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, i, ckey, mkey, MarkNone{}, bad);
            else if (MODE == kMarkByte)
                map_one<DP, false>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, i, ckey, mkey,
                                   MarkByte{reinterpret_cast<uint8_t*>(occ), false}, bad);
            else
                map_one<DP, false>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, i, ckey, mkey, MarkGlobal{occ}, bad);
        }
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, SKY_DEV_ERR_NONFINITE);
    if (MODE == kMarkSmall) {
        __syncthreads();
        for (int64_t w = threadIdx.x; w < words; w += blockDim.x) stage[blockIdx.x * words + w] = s_occ[w];
    }
}

// Bulk-copy streaming version: rows are contiguous (ld == d) and the base is
// 16-byte aligned. Chunks of kThreads rows (kThreads*d*4 bytes, a multiple of
// 16) go through kStages shared-memory buffers; one thread issues the copies.
// A thread reads its row from shared memory as float4s when d is a multiple
// of 4 (eight rows per quarter-warp phase: at most 4-way bank conflicts at
// d = 16 instead of 16-way for scalar reads).
constexpr int kMapStages = 4;

// Rows per thread and stage: a stage holds kThreads * map_rpt(DP) rows, at
// most 16 KB (four rows of four floats per thread at d <= 4, two at d <= 8),
// so that small rows keep as many bytes in flight as 16-float rows.
__host__ __device__ constexpr int map_rpt(int DP) { return DP >= 16 ? 1 : 16 / DP; }

template <int DP, int MODE>
__global__ void __launch_bounds__(kThreads) k_map_mark_tma(const float* __restrict__ pts, int64_t n,
                                                           int d, int log2g, int mbits, const float* params,
                                                           uint32_t* ckey, uint32_t* mkey, uint32_t* occ,
                                                           uint32_t* err, uint32_t* stage, int64_t words,
                                                           bool look)
{
    // [kMapStages][kThreads * map_rpt(DP) * d] row stages, then the private
    // bitmap [words] (kMarkSmall)
    extern __shared__ __align__(128) float s_buf[];
    __shared__ float s_off[kMaxDim], s_sc[kMaxDim], s_ms[kMaxDim];
    __shared__ __align__(8) uint64_t s_bar[kMapStages];
    __shared__ uint32_t s_dups, s_check;
    const int tid = threadIdx.x;
    uint32_t* s_tail = reinterpret_cast<uint32_t*>(s_buf + kMapStages * kThreads * map_rpt(DP) * d);
    if (tid < kMaxDim) {
        s_off[tid] = params[tid];
        s_sc[tid] = params[16 + tid];
        s_ms[tid] = params[48 + tid];
    }
    if (MODE == kMarkSmall)
        for (int64_t w = tid; w < words; w += kThreads) s_tail[w] = 0u;
    if (tid == 0) {
        for (int s = 0; s < kMapStages; ++s) mbar_init(&s_bar[s], 1);
        mbar_fence_init();
        s_dups = 0u;
        s_check = look ? 1u : 0u;
    }
    __syncthreads();
    const MortonSpread ms(d, mbits);
    const bool v4 = (d == DP);      // DP is d rounded up to a multiple of 4
    // the unit-cube map with whole float4 rows: the piece-rotated fast path
    bool unit = v4 && ms.fast();
    for (int k = 0; k < d && unit; ++k)
        unit = s_off[k] == 0.0f && s_sc[k] == (float)(1u << log2g) &&
               (mbits <= log2g || s_ms[k] == (float)(1u << mbits));
    constexpr int NQ = DP / 4;
    const int rot = NQ == 4 ? (tid >> 1) & 3 : (NQ == 2 ? (tid >> 2) & 1 : 0);

    constexpr int RPT = map_rpt(DP);
    constexpr int CR = kThreads * RPT;             // rows per stage
    const int64_t nfull = n / CR;
    const uint32_t chunk_bytes = (uint32_t)(CR * d * sizeof(float));
    const int64_t my_chunks = (nfull > blockIdx.x) ? (nfull - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    if (tid == 0) {
        for (int64_t i = 0; i < my_chunks && i < kMapStages; ++i) {
            const int64_t c = blockIdx.x + i * gridDim.x;
            mbar_arrive_expect_tx(&s_bar[i], chunk_bytes);
            bulk_g2s(s_buf + i * CR * d, pts + c * CR * d, chunk_bytes, &s_bar[i]);
        }
    }
    bool bad = false;
    bool timed_out = false;
    uint32_t dups = 0;   // rows of the first chunk whose word another lane of the warp has too
    for (int64_t i = 0; i < my_chunks; ++i) {
        const int s = (int)(i % kMapStages);
        const uint32_t parity = (uint32_t)((i / kMapStages) & 1);
        // one thread waits on the stage (the TMA writes become visible to it),
        // the block barrier passes them on to the others
        if (tid == 0 && !mbar_wait(&s_bar[s], parity, err)) timed_out = true;
        if (__syncthreads_or(timed_out)) {
            // Let every copy already issued land before the block goes on.
            if (tid == 0) {
                for (int64_t j = i; j < my_chunks && j < i + kMapStages; ++j)
                    mbar_wait(&s_bar[j % kMapStages], (uint32_t)((j / kMapStages) & 1), nullptr);
            }
            timed_out = true;
            __syncthreads();
            break;
        }
        const int64_t c = blockIdx.x + i * gridDim.x;
        if (unit) {
            // the stage's rows of this thread: keys first, then the marks
            uint32_t key[RPT], code[RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const float* r = s_buf + s * CR * d + (j * kThreads + tid) * d;
                if (mbits <= log2g) map_keys_unit<DP, true>(r, rot, log2g, mbits, ms, key[j], code[j], bad);
                else map_keys_unit<DP, false>(r, rot, log2g, mbits, ms, key[j], code[j], bad);
            }
            if (ckey) {
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const int64_t row = c * CR + j * kThreads + tid;
                    ckey[row] = key[j];
                    mkey[row] = code[j];
                }
            }
            if (MODE == kMarkSmall) {
#pragma unroll
                for (int j = 0; j < RPT; ++j) mark_cell<true>(key[j], MarkPrivate{s_tail});
            } else if (MODE == kMarkByte) {
                uint8_t* ob = reinterpret_cast<uint8_t*>(occ);
                if (s_check != 0u && i > 0) {
                    uint8_t v[RPT];
#pragma unroll
                    for (int j = 0; j < RPT; ++j) v[j] = __ldca(ob + key[j]);
#pragma unroll
                    for (int j = 0; j < RPT; ++j)
                        if (!v[j]) ob[key[j]] = 1;
                } else {
#pragma unroll
                    for (int j = 0; j < RPT; ++j)
                        mark_cell<true>(key[j], MarkByte{ob, false}, (i == 0 && j == 0) ? &dups : nullptr);
                }
            } else if (MODE == kMarkCheck) {
                if (s_check != 0u && i > 0) {
                    // looking: every bitmap read of the thread in flight at
                    // once; a mark is sent only when its bit is not set yet
                    uint32_t w[RPT];
#pragma unroll
                    for (int j = 0; j < RPT; ++j) w[j] = __ldca(occ + (key[j] >> 5));
#pragma unroll
                    for (int j = 0; j < RPT; ++j)
                        if (!((w[j] >> (key[j] & 31u)) & 1u)) atomicOr(occ + (key[j] >> 5), 1u << (key[j] & 31u));
                } else {
#pragma unroll
                    for (int j = 0; j < RPT; ++j)
                        mark_cell<true>(key[j], MarkCheck{occ, s_check != 0u}, (i == 0 && j == 0) ? &dups : nullptr);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < RPT && !unit; ++j) {
            const int rr = j * kThreads + tid;          // row of the stage
            const float* r = s_buf + s * CR * d + rr * d;
            const int64_t row = c * CR + rr;
            uint32_t* dp = (i == 0 && j == 0) ? &dups : nullptr;
            {
                float x[DP];
                if (v4) {
#pragma unroll
                    for (int k = 0; k < DP; k += 4) {
                        const float4 q = *reinterpret_cast<const float4*>(r + k);
                        x[k] = q.x; x[k + 1] = q.y; x[k + 2] = q.z; x[k + 3] = q.w;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < DP; ++k) x[k] = (k < d) ? r[k] : 0.0f;
                }
                if (MODE == kMarkSmall)
                    map_one<DP, true>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, row, ckey, mkey, MarkPrivate{s_tail},
                                      bad);
                else if (MODE == kMarkNone)
                    map_one<DP, true>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, row, ckey, mkey, MarkNone{}, bad);
                else if (MODE == kMarkByte)
                    map_one<DP, true>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, row, ckey, mkey,
                                      MarkByte{reinterpret_cast<uint8_t*>(occ), s_check != 0u}, bad, dp);
                else
                    map_one<DP, true>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, row, ckey, mkey,
                                      MarkCheck{occ, s_check != 0u}, bad, dp);
            }
        }
        if ((MODE == kMarkCheck || MODE == kMarkByte) && i == 0) {
            const uint32_t h = __reduce_add_sync(kFull, dups);
            if ((tid & 31) == 0 && h) atomicAdd(&s_dups, h);
        }
        __syncthreads();  // every thread is done with stage s
        if (tid == 0) {
            // look before marking from the second chunk on when at least
            // 1/16 of the first chunk's first rows shared their word inside a warp
            if ((MODE == kMarkCheck || MODE == kMarkByte) && i == 0 && s_dups >= (uint32_t)(kThreads / 16))
                s_check = 1u;
            if (i + kMapStages < my_chunks) {
                const int64_t c2 = blockIdx.x + (i + kMapStages) * gridDim.x;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&s_bar[s], chunk_bytes);
                bulk_g2s(s_buf + s * CR * d, pts + c2 * CR * d, chunk_bytes, &s_bar[s]);
            }
        }
    }
    // Tail rows (fewer than one stage): the last block loads them directly.
    if (!timed_out && blockIdx.x == gridDim.x - 1) {
        for (int64_t i = nfull * CR + tid; i < n; i += kThreads) {
            float x[DP];
            load_row<DP>(pts + i * d, d, false, x);
            if (MODE == kMarkSmall)
                map_one<DP, false>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, i, ckey, mkey, MarkPrivate{s_tail}, bad);
            else if (MODE == kMarkNone)
                map_one<DP, false>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, i, ckey, mkey, MarkNone{}, bad);
            else if (MODE == kMarkByte)
                map_one<DP, false>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, i, ckey, mkey,
                                   MarkByte{reinterpret_cast<uint8_t*>(occ), false}, bad);
            else
                map_one<DP, false>(x, d, log2g, mbits, ms, s_off, s_sc, s_ms, i, ckey, mkey, MarkGlobal{occ}, bad);
        }
    }
    if (__any_sync(kFull, bad) && (tid & 31) == 0) atomicOr(err, SKY_DEV_ERR_NONFINITE);
    __syncthreads();
    if (MODE == kMarkSmall) {
        for (int64_t w = tid; w < words; w += kThreads) stage[blockIdx.x * words + w] = s_tail[w];
    }
}

// ORs the blocks' private bitmaps (rows of `stage`) into the bitmap: block
// (c, r) takes 32 words and every kMergeSplit-th row from r on; the bitmap
// was zeroed before the map pass.
constexpr int kMergeSplit = 8;

__global__ void __launch_bounds__(kThreads) k_occ_merge(const uint32_t* __restrict__ stage, int rows,
                                                        int64_t words, uint32_t* occ)
{
    __shared__ uint32_t s_acc[kThreads / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t w = (int64_t)(blockIdx.x / kMergeSplit) * 32 + lane;
    const int r0 = (int)(blockIdx.x % kMergeSplit);
    uint32_t acc = 0;
    if (w < words)
        for (int r = r0 + warp * kMergeSplit; r < rows; r += kMergeSplit * (kThreads / 32))
            acc |= __ldg(stage + (int64_t)r * words + w);
    s_acc[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        for (int k = 1; k < kThreads / 32; ++k) acc |= s_acc[k][lane];
        if (w < words && acc) atomicOr(occ + w, acc);
    }
}

// ---------------------------------------------------------------------------
// One dimension of the prefix-OR over the whole grid (global memory).
// Bitmap word w from the 32 bytes of cells 32w .. 32w + 31 (each 0 or 1):
// ((x & 0x01010101) * 0x01020408) >> 24 gathers the low bits of four bytes
// into a nibble (the partial products land on distinct bits, no carries).
__global__ void __launch_bounds__(kThreads) k_occ_pack(const uint8_t* __restrict__ occb, uint32_t* occ, int64_t words)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += stride) {
        const uint4* src = reinterpret_cast<const uint4*>(occb + 32 * w);
        const uint4 a = __ldcs(src), b = __ldcs(src + 1);
        const uint32_t x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint32_t r = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) r |= (((x[q] & 0x01010101u) * 0x01020408u) >> 24) << (4 * q);
        occ[w] = r;
    }
}

__global__ void __launch_bounds__(kThreads) k_prefix_or_dim(uint32_t* R, int64_t words, int log2g, int k)
{
    prefix_or_dim(R, words, log2g, k, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                  (int64_t)gridDim.x * blockDim.x);
}

// Prefix-OR in two launches. The low kl dimensions (the low S = log2g * kl
// bits of a cell key, S >= 5) are done per aligned block of 2^S bits in
// shared memory; the high kh = d - kl dimensions by a second kernel that
// holds, for a run of wc consecutive words of the low block, all G^kh rows
// of the high grid in shared memory. Both are the per-dimension prefix-OR of
// prefix_or_dim applied in dimension order.
constexpr int kPrefixThreads = 1024;   // bound of k_prefix_low's launch
// Tiling of the two-launch prefix-OR (see prefix_split)
#ifndef SKY_PREFIX_LOW_BITS
#define SKY_PREFIX_LOW_BITS 16
#endif
#ifndef SKY_PREFIX_LOW_THREADS
#define SKY_PREFIX_LOW_THREADS 512
#endif
#ifndef SKY_PREFIX_WORDS_PER_THREAD
#define SKY_PREFIX_WORDS_PER_THREAD 4
#endif
#ifndef SKY_PREFIX_HIGH_WORDS
#define SKY_PREFIX_HIGH_WORDS 2048
#endif
constexpr int kPrefixLowBits = SKY_PREFIX_LOW_BITS;            // bits per low block
constexpr int kPrefixLowThreads = SKY_PREFIX_LOW_THREADS;      // at most, per low block
constexpr int kPrefixWordsPerThread = SKY_PREFIX_WORDS_PER_THREAD;
constexpr int kPrefixHighWords = SKY_PREFIX_HIGH_WORDS;        // shared words per high block
static_assert(kPrefixLowBits >= 5 && kPrefixLowBits <= 20, "low blocks of whole words, at most 128 KB");

__global__ void __launch_bounds__(kPrefixThreads) k_prefix_low(const uint32_t* __restrict__ occ, uint32_t* pre,
                                                               int64_t block_words, int log2g, int kl)
{
    extern __shared__ uint4 s_w4[];
    uint32_t* s_w = reinterpret_cast<uint32_t*>(s_w4);
    const int64_t base = (int64_t)blockIdx.x * block_words;
    const uint32_t bw = (uint32_t)block_words;
    if ((bw & 3u) == 0u) {   // 16-byte pieces (blocks of >= 128 cells)
        for (uint32_t w = threadIdx.x; w < bw / 4u; w += blockDim.x) cp_async16(s_w4 + w, occ + base + 4 * w);
    } else {
        for (uint32_t w = threadIdx.x; w < bw; w += blockDim.x) cp_async4(s_w + w, occ + base + w);
    }
    cp_async_wait_all();
    __syncthreads();
    // the dimensions inside one word in one pass, the others one pass each
    int kin = 0;
    while (kin < kl && log2g * (kin + 1) <= 5) ++kin;
    if (kin > 0) {
        prefix_or_inword(s_w, block_words, log2g, kin, threadIdx.x, blockDim.x);
        __syncthreads();
    }
    for (int k = kin; k < kl; ++k) {
        prefix_or_dim(s_w, block_words, log2g, k, threadIdx.x, blockDim.x);
        __syncthreads();
    }
    if ((bw & 3u) == 0u) {
        uint4* dst = reinterpret_cast<uint4*>(pre + base);
        for (uint32_t w = threadIdx.x; w < bw / 4u; w += blockDim.x) dst[w] = s_w4[w];
    } else {
        for (uint32_t w = threadIdx.x; w < bw; w += blockDim.x) pre[base + w] = s_w[w];
    }
}

// rows, wc and every stride are powers of two (log2: lrows, lwc); indices
// fit in 32 bits (at most 2^22 words).
__global__ void __launch_bounds__(kThreads) k_prefix_high(uint32_t* pre, int64_t row_words, int lrows, int lwc,
                                                          int log2g, int kh)
{
    extern __shared__ __align__(16) uint32_t s_t[];   // [rows][wc]
    const uint32_t wc = 1u << lwc;
    const uint32_t c0 = blockIdx.x << lwc;
    const uint32_t cells = 1u << (lrows + lwc);
    const uint32_t rw = (uint32_t)row_words;
    if (lwc >= 2) {   // rows of >= 4 words: 16-byte pieces (row starts are 16-byte aligned)
        for (uint32_t t = 4 * threadIdx.x; t < cells; t += 4 * blockDim.x)
            cp_async16(s_t + t, pre + (t >> lwc) * rw + c0 + (t & (wc - 1u)));
    } else {
        for (uint32_t t = threadIdx.x; t < cells; t += blockDim.x)
            cp_async4(s_t + t, pre + (t >> lwc) * rw + c0 + (t & (wc - 1u)));
    }
    cp_async_wait_all();
    __syncthreads();
    const uint32_t G = 1u << log2g;
    for (int j = 0; j < kh; ++j) {
        const int lsr = log2g * j;                          // row stride of high dimension j: 2^lsr
        const uint32_t lines = 1u << (lrows - log2g + lwc);
        for (uint32_t L = threadIdx.x; L < lines; L += blockDim.x) {
            const uint32_t w = L & (wc - 1u), l = L >> lwc;
            const uint32_t r = ((l >> lsr) << (lsr + log2g)) + (l & ((1u << lsr) - 1u));
            or_scan_strided(s_t + (r << lwc) + w, G, (1u << lsr) << lwc, 0u);
        }
        __syncthreads();
    }
    for (uint32_t t = threadIdx.x; t < cells; t += blockDim.x)
        pre[(t >> lwc) * rw + c0 + (t & (wc - 1u))] = s_t[t];
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
// row: the packed (ordered sum, row) minimum. Each thread keeps its running
// minimum per proposal in registers over its grid-stride rows; the block
// combines them by warp shuffles and shared-memory atomics and issues one
// global 64-bit atomic min per proposal, so the global traffic is
// blocks x proposals however many rows qualify.
template <int DP>
__global__ void __launch_bounds__(kThreads) k_snap(const float* __restrict__ pts, int64_t n, int d,
                                                   int64_t ld, bool vec4, const float* __restrict__ prop,
                                                   int n_prop, unsigned long long* snap)
{
    constexpr int NP = 16;
    // proposals padded to DP with +inf (a padded dimension never rejects),
    // read back as float4s; proposals past n_prop are -inf (never pass)
    __shared__ __align__(16) float s_f[NP * DP];
    __shared__ unsigned long long s_best[NP];
    for (int t = threadIdx.x; t < NP * DP; t += blockDim.x) {
        const int j = t / DP, k = t % DP;
        s_f[t] = j >= n_prop ? -INFINITY : (k < d ? prop[j * d + k] : INFINITY);
    }
    if (threadIdx.x < NP) s_best[threadIdx.x] = ~0ull;
    __syncthreads();
    // F = the proposals' componentwise maximum: a row above F in some
    // dimension is <= no proposal and skips the per-proposal tests
    float F[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) {
        F[k] = -INFINITY;
        for (int j = 0; j < NP; ++j) F[k] = fmaxf(F[k], s_f[j * DP + k]);
    }
    unsigned long long best[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) best[j] = ~0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float x[DP];
        load_row<DP>(pts + i * ld, d, vec4, x);
        // padded dimensions of x are 0 (load_row) and compare <= +inf
        bool under = true;
#pragma unroll
        for (int k = 0; k < DP; ++k) under &= x[k] <= F[k];
        if (!under) continue;
        uint32_t pass = 0;   // bit j: x <= proposal j in every dimension
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            bool le = true;
#pragma unroll
            for (int k = 0; k < DP; k += 4) {
                const float4 f = *reinterpret_cast<const float4*>(&s_f[j * DP + k]);
                le &= (x[k] <= f.x) & (x[k + 1] <= f.y) & (x[k + 2] <= f.z) & (x[k + 3] <= f.w);
            }
            pass |= (le ? 1u : 0u) << j;
        }
        if (pass == 0u) continue;   // most rows, when few proposals reach the data
        float sum = 0.0f;
#pragma unroll
        for (int k = 0; k < DP; ++k)
            if (k < d) sum = __fadd_rn(sum, x[k]);
        // + 0.0f turns a sum of -0.0 into +0.0, so that equal sums compare
        // equal in the packed order (ties then go to the lower row)
        const unsigned long long packed =
            ((unsigned long long)float_to_ordered(__fadd_rn(sum, 0.0f)) << 32) | (unsigned long long)(uint32_t)i;
#pragma unroll
        for (int j = 0; j < NP; ++j)
            if (((pass >> j) & 1u) && packed < best[j]) best[j] = packed;
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        if (j < n_prop) {
            unsigned long long v = best[j];
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long w = __shfl_xor_sync(kFull, v, o);
                v = w < v ? w : v;
            }
            if ((threadIdx.x & 31) == 0 && v != ~0ull) atomicMin(&s_best[j], v);
        }
    }
    __syncthreads();
    if (threadIdx.x < n_prop && s_best[threadIdx.x] != ~0ull) atomicMin(&snap[threadIdx.x], s_best[threadIdx.x]);
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
// Survivors of step (c), compacted in row order with their Morton keys, in
// two passes over the same fixed split of the rows: block b owns the
// contiguous tiles [b * tpb, (b + 1) * tpb) of kSurvTile rows. Row
// tile * kSurvTile + j * kThreads + tid is item j of thread tid, so the warp
// ballot of item j is exactly flag word row / 32.
//   k_surv_flags    reads the cell keys of its tiles (16-byte streaming
//                   loads, the next tile's in flight while a tile is
//                   decided), probes the prefix-OR bitmap at key - (1, ..., 1)
//                   (Corollary 4: a cell is dominated iff that cell is
//                   covered), applies the optional snapped proposals, writes
//                   the flag words and the block's survivor count
//   k_surv_scatter  sums the counts of the blocks before it, counts the
//                   survivors of each of its tiles from the flag words and
//                   scans them, then for the tiles that keep a row loads the
//                   Morton keys of the set rows and writes (Morton key, row)
//                   pairs, coalesced per warp
// No look-back chain and no global atomics. (Staging the keys through a
// shared-memory ring of 1-D bulk copies measured no faster: these passes are
// short and bound by the latency of their first loads, not by issue.)
constexpr int kSurvItems = 8;
constexpr int kSurvTile = kSurvItems * kThreads;   // 2048 rows
constexpr int kSurvMaxTpb = 2048;                  // tiles per block (n < 2^31 needs at most 1,772)
constexpr int kTileWords = kSurvTile / 32;         // flag words per tile
static_assert(kTileWords == 64, "one warp scans a tile's flag words two per lane");

// True when some lg-bit field of key is zero: (key - ones) borrows into the
// top bit of a field only below a zero field, and ~key keeps it only there.
__device__ __forceinline__ bool has_zero_column(uint32_t key, uint32_t ones, uint32_t highs)
{
    return ((key - ones) & ~key & highs) != 0u;
}

// Keys of rows tile * kSurvTile + h * 4 * kThreads + 4 * tid + (0..3) into
// k[h], one 16-byte streaming load each (rows past n read the arrays' slack
// and are ignored by the caller; steps starting past n load nothing).
template <int H>
__device__ __forceinline__ void surv_load_keys(const uint32_t* __restrict__ keys, int64_t tile, int64_t n, int tid,
                                               uint4 (&k)[H])
{
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int64_t r = tile * kSurvTile + (int64_t)h * 4 * kThreads + 4 * tid;
        k[h] = r < n ? __ldcs(reinterpret_cast<const uint4*>(keys + r)) : make_uint4(0u, 0u, 0u, 0u);
    }
}

// Four consecutive rows per thread and step (one 16-byte load); a tile is
// two steps of 1,024 rows. The eight lanes 8q .. 8q+7 of a
// warp hold the 32 rows of one flag word as nibbles, OR-ed together in three
// shuffles. The bitmap is probed only when some lane of the warp needs it.
template <int DP>
__global__ void __launch_bounds__(kThreads) k_surv_flags(
    const float* __restrict__ pts, int64_t n, int d, int64_t ld, bool vec4, int log2g,
    const uint32_t* __restrict__ ckey, const uint32_t* __restrict__ pre, const float* __restrict__ filt,
    int n_filter_max, DevResult* res, int64_t tpb, uint32_t* __restrict__ flags, uint32_t* __restrict__ counts,
    uint8_t* __restrict__ keep_bytes)
{
    __shared__ float s_f[16 * kMaxDim];
    __shared__ uint32_t s_cnt[kThreads / 32];
    __shared__ uint32_t s_diag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ntiles = (n + kSurvTile - 1) / kSurvTile;
    const int64_t t0 = (int64_t)blockIdx.x * tpb;
    const int64_t my = (t0 + tpb < ntiles ? t0 + tpb : ntiles) - t0;
    constexpr int H = kSurvTile / (4 * kThreads);   // steps per tile
    static_assert(H == 2, "two steps of four rows per thread");
    // this thread's keys of the block's first tile, in flight while the
    // block looks for D
    uint4 nk[H];
    surv_load_keys<H>(ckey, t0, n, tid, nk);
    const int nf = n_filter_max ? (int)res->n_filter_used : 0;
    for (int t = tid; t < nf * kMaxDim; t += kThreads) s_f[t] = filt[t];
    // With log2g = 0 the grid is one cell, which nothing dominates (and the
    // field masks below would be empty): no row probes the bitmap then.
    const bool can_dominate = log2g > 0;
    const uint32_t ones = ones_key(log2g, d);
    const uint32_t highs = can_dominate ? ones << (log2g - 1) : 0u;
    const int sub = lane & 7;                  // nibble of this lane in its flag word
    // D = the first t whose diagonal cell (t, .., t) has its prefix-OR bit
    // set: some occupied cell lies in [0, t]^d, so every cell whose columns
    // all exceed D is dominated (Def. 3) without a probe. D = 0 (the origin
    // cell is occupied) settles every row that would probe.
    if (warp == 0) {
        const uint32_t G = 1u << log2g;
        uint32_t first = G;
        for (uint32_t t0 = 0; t0 < G && can_dominate; t0 += 32) {
            const uint32_t t = t0 + lane;
            bool set = false;
            if (t < G) {
                const uint32_t c = t * ones;
                set = (__ldg(pre + (c >> 5)) >> (c & 31u)) & 1u;
            }
            const uint32_t b = __ballot_sync(kFull, set);
            if (b) { first = t0 + (uint32_t)(__ffs(b) - 1); break; }
        }
        if (lane == 0) s_diag = first;
    }
    __syncthreads();
    const uint32_t D = s_diag;
    const uint32_t cmask = (1u << log2g) - 1u;
    // Every key the map pass writes is below 2^(log2g d), so masking a probe
    // with the grid changes nothing; it keeps the probe inside the bitmap
    // when the map pass gave up (a bounded wait ran out) before writing some
    // rows' keys and those rows hold whatever the workspace held.
    const uint32_t gridmask = (uint32_t)((uint64_t(1) << (log2g * d)) - 1u);
    uint32_t cnt = 0;                          // rows kept by this thread
    for (int64_t i = 0; i < my; ++i) {
        const int64_t tile = t0 + i;
        const int64_t row0 = tile * kSurvTile;
        // rows of this tile: all kSurvTile but in the last tile
        const uint32_t valid = (uint32_t)(n - row0 < kSurvTile ? n - row0 : kSurvTile);
        uint32_t* fl = flags + tile * kTileWords;
        if (keep_bytes) {   // the refinement's keep bytes start at zero (4 rows a store; the array has slack)
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const uint32_t r = (uint32_t)(h * 4 * kThreads + 4 * tid);
                if (r < valid) *reinterpret_cast<uint32_t*>(keep_bytes + row0 + r) = 0u;
            }
        }
        uint32_t ks[H][4], keep[H], need[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            ks[h][0] = nk[h].x; ks[h][1] = nk[h].y; ks[h][2] = nk[h].z; ks[h][3] = nk[h].w;
        }
        // the next tile's keys in flight (a deeper register ring of three
        // tiles measured no faster)
        if (i + 1 < my) surv_load_keys<H>(ckey, tile + 1, n, tid, nk);
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const uint32_t r = (uint32_t)(h * 4 * kThreads + 4 * tid);   // first of this thread's 4 rows
            keep[h] = 0u;
            need[h] = 0u;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (r + e < valid) {
                    if (can_dominate && !has_zero_column(ks[h][e], ones, highs)) {
                        // every column >= 1; dominated outright when every
                        // column exceeds D, else the bitmap decides
                        bool above = D == 0u;
                        if (!above && DP <= 8) {
                            above = true;
#pragma unroll
                            for (int k = 0; k < DP; ++k)
                                if (k < d) above &= ((ks[h][e] >> (log2g * k)) & cmask) > D;
                        }
                        if (!above) need[h] |= 1u << e;
                    } else {
                        keep[h] |= 1u << e;
                    }
                }
            }
        }
        // every bitmap probe of the tile in flight at once
        if (__any_sync(kFull, (need[0] | need[1]) != 0u)) {
            uint32_t wd[H][4];
#pragma unroll
            for (int h = 0; h < H; ++h)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    wd[h][e] = ((need[h] >> e) & 1u) ? __ldg(pre + (((ks[h][e] - ones) & gridmask) >> 5)) : 0u;
#pragma unroll
            for (int h = 0; h < H; ++h)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (((need[h] >> e) & 1u) && !((wd[h][e] >> ((ks[h][e] - ones) & 31u)) & 1u))
                        keep[h] |= 1u << e;
        }
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const uint32_t r = (uint32_t)(h * 4 * kThreads + 4 * tid);
            if (nf && keep[h]) {
#pragma unroll 1
                for (int e = 0; e < 4; ++e) {
                    if (!((keep[h] >> e) & 1u)) continue;
                    float x[DP];
                    load_row<DP>(pts + (row0 + r + e) * ld, d, vec4, x);
                    bool filtered = false;
                    for (int q = 0; q < nf && !filtered; ++q) {
                        bool le = true, lt = false;
#pragma unroll
                        for (int k = 0; k < DP; ++k) {
                            if (k < d) {
                                const float v = s_f[q * kMaxDim + k];
                                le &= v <= x[k];
                                lt |= v < x[k];
                            }
                        }
                        filtered = le && lt;  // Definition 1: the snapped point dominates x
                    }
                    if (filtered) keep[h] &= ~(1u << e);
                }
            }
            cnt += (uint32_t)__popc(keep[h]);
            uint32_t v = keep[h] << (4 * sub);
            v |= __shfl_xor_sync(kFull, v, 1);
            v |= __shfl_xor_sync(kFull, v, 2);
            v |= __shfl_xor_sync(kFull, v, 4);
            // words past the end of the flag array only hold rows >= n
            const uint32_t wr = r - 4u * (uint32_t)sub;   // first row of this lane's flag word
            if (sub == 0 && wr < valid) fl[wr >> 5] = v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    if (lane == 0) s_cnt[warp] = cnt;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += s_cnt[w];
        counts[blockIdx.x] = t;
    }
}

// The block's output offset and every tile's offset come from the counts and
// flag words first; then each warp loads the Morton keys of its set rows (all
// eight items' loads in flight together) and writes (key, row) pairs,
// coalesced per warp. Tiles that keep no row are skipped.
__global__ void __launch_bounds__(kThreads) k_surv_scatter(int64_t n, const uint32_t* __restrict__ mkey,
                                                           const uint32_t* __restrict__ flags,
                                                           const uint32_t* __restrict__ counts, int64_t tpb,
                                                           DevResult* res, uint32_t* __restrict__ surv_key,
                                                           uint32_t* __restrict__ surv_idx)
{
    // per tile of this block: its survivor count [tpb] and exclusive offset [tpb]
    extern __shared__ __align__(16) uint32_t s_dyn[];
    uint32_t* s_tc = s_dyn;
    uint32_t* s_to = s_tc + tpb;
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ uint32_t s_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ntiles = (n + kSurvTile - 1) / kSurvTile;
    const int64_t t0 = (int64_t)blockIdx.x * tpb;
    const int my = (int)((t0 + tpb < ntiles ? t0 + tpb : ntiles) - t0);
    const int64_t nwords = (n + 31) / 32;
    // rows kept by the blocks before this one
    uint32_t part = 0;
    for (int b = tid; b < (int)blockIdx.x; b += kThreads) part += counts[b];
    part = __reduce_add_sync(kFull, part);
    if (lane == 0) s_warp[warp] = part;
    for (int i = tid; i < my; i += kThreads) s_tc[i] = 0u;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += s_warp[w];
        s_off = t;
    }
    // survivors per tile: the 32 lanes of a warp read 32 words of one tile
    for (int w = tid; w < my * kTileWords; w += kThreads) {
        const int64_t gw = t0 * kTileWords + w;
        uint32_t c = gw < nwords ? (uint32_t)__popc(__ldg(flags + gw)) : 0u;
        c = __reduce_add_sync(kFull, c);
        if (lane == 0) atomicAdd(&s_tc[w / kTileWords], c);
    }
    __syncthreads();
    // exclusive offsets of the tiles: each thread scans a contiguous run
    const int per = (my + kThreads - 1) / kThreads;
    const int i0 = tid * per;
    uint32_t run = 0;
    for (int i = i0; i < i0 + per && i < my; ++i) run += s_tc[i];
    uint32_t total;
    uint32_t before = block_excl_scan<kThreads>(run, s_warp, total);
    for (int i = i0; i < i0 + per && i < my; ++i) {
        s_to[i] = before;
        before += s_tc[i];
    }
    __syncthreads();
    const uint32_t base_off = s_off;
    const uint32_t below = lanemask_lt();
    for (int i = 0; i < my; ++i) {
        if (s_tc[i] == 0u) continue;   // block-uniform
        const int64_t tile = t0 + i;
        // every warp scans the tile's 64 flag words itself (lane l: words l
        // and 32 + l)
        const int64_t gw = tile * kTileWords + lane;
        const uint32_t fa = gw < nwords ? __ldg(flags + gw) : 0u;
        const uint32_t fb = gw + 32 < nwords ? __ldg(flags + gw + 32) : 0u;
        const uint32_t pa = (uint32_t)__popc(fa), pb = (uint32_t)__popc(fb);
        uint32_t xa = pa, xb = pb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t ya = __shfl_up_sync(kFull, xa, o), yb = __shfl_up_sync(kFull, xb, o);
            if (lane >= o) { xa += ya; xb += yb; }
        }
        const uint32_t ta = __shfl_sync(kFull, xa, 31);
        const uint32_t oa = xa - pa, ob = ta + xb - pb;   // exclusive offsets of words l and 32 + l
        const uint32_t tile_base = base_off + s_to[i];
        const uint32_t row0 = (uint32_t)(tile * kSurvTile);
        uint32_t fw[kSurvItems], ow[kSurvItems], key[kSurvItems];
#pragma unroll
        for (int j = 0; j < kSurvItems; ++j) {
            const int wi = j * (kThreads / 32) + warp;   // flag word of item j of this warp
            fw[j] = __shfl_sync(kFull, wi < 32 ? fa : fb, wi & 31);
            ow[j] = __shfl_sync(kFull, wi < 32 ? oa : ob, wi & 31);
        }
#pragma unroll
        for (int j = 0; j < kSurvItems; ++j)
            key[j] = ((fw[j] >> lane) & 1u) ? __ldcs(mkey + row0 + j * kThreads + tid) : 0u;
#pragma unroll
        for (int j = 0; j < kSurvItems; ++j) {
            if ((fw[j] >> lane) & 1u) {
                const uint32_t pos = tile_base + ow[j] + (uint32_t)__popc(fw[j] & below);
                surv_key[pos] = key[j];
                surv_idx[pos] = row0 + (uint32_t)(j * kThreads + tid);
            }
        }
    }
    if (blockIdx.x == gridDim.x - 1 && tid == 0) res->survivors = base_off + total;
}

// Result of a survivors-only call: the survivor row ids (already ascending)
// into the caller's buffer; count = survivors, nothing written past capacity.
__global__ void __launch_bounds__(kThreads) k_copy_survivors(const uint32_t* __restrict__ surv_idx, DevResult* res,
                                                             int32_t* out, int64_t capacity)
{
    const uint32_t m = res->survivors;
    if (blockIdx.x == 0 && threadIdx.x == 0) res->count = m;
    if ((int64_t)m > capacity) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)surv_idx[i];
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

// Upper bound of the map pass's block count (sizes the private-bitmap rows).
int map_blocks_bound(int64_t n)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, kMapMaxBlocks);
}

template <int DP, int MODE>
static void map_tma(const Plan& p, int& blocks, size_t smem, int smem_max, int64_t pw, cudaStream_t s)
{
    // look before marking from the start when the rows outnumber the cells
    // four to one: most marks then find their bit set already
    const bool look = p.n >= 4 * (int64_t(1) << (p.log2g * p.d));
    cudaFuncSetAttribute(k_map_mark_tma<DP, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    // one wave: as many blocks as fit on the SMs at once (a partial second
    // wave would run its blocks at a fraction of the occupancy)
    // (asked once per kernel instance and shared-memory size)
    static thread_local size_t cached_smem = ~size_t(0);
    static thread_local int cached_per_sm = 0;
    if (cached_smem != smem) {
        cached_per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cached_per_sm, k_map_mark_tma<DP, MODE>, kThreads, smem) !=
                cudaSuccess || cached_per_sm < 1) {
            cudaGetLastError();
            cached_per_sm = 1;
        }
        cached_smem = smem;
    }
    const int per_sm = cached_per_sm;
    blocks = std::min(blocks, per_sm * num_sms());
    uint32_t* occ = MODE == kMarkByte ? reinterpret_cast<uint32_t*>(p.occb) : p.occ;
    k_map_mark_tma<DP, MODE><<<blocks, kThreads, smem, s>>>(p.pts, p.n, p.d, p.log2g, p.morton_bits, p.params,
                                                            p.ckey, p.mkey, occ, &p.res->err,
                                                            MODE == kMarkSmall ? p.occ_stage : nullptr, pw, look);
}

template <int DP, int MODE>
static void map_plain(const Plan& p, int blocks, size_t smem, int64_t pw, bool v, cudaStream_t s)
{
    uint32_t* occ = MODE == kMarkByte ? reinterpret_cast<uint32_t*>(p.occb) : p.occ;
    k_map_mark_plain<DP, MODE><<<blocks, kThreads, smem, s>>>(p.pts, p.n, p.d, p.ld, v, p.log2g, p.morton_bits,
                                                              p.params, p.ckey, p.mkey, occ, &p.res->err,
                                                              MODE == kMarkSmall ? p.occ_stage : nullptr, pw);
}

// Steps (a)+(b) over p.pts with the parameters already in p.params. With
// mark = false only the keys are written (the bitmap is left alone).
cudaError_t launch_map_pass(const Plan& p, bool mark, cudaStream_t s)
{
    if (p.n == 0) return cudaGetLastError();
    const int mode = !mark ? kMarkNone
                           : (p.occ_stage != nullptr ? kMarkSmall : (p.occb != nullptr ? kMarkByte : kMarkCheck));
    const int64_t pw = mode == kMarkSmall ? p.words : 0;
    int blocks = 0;
    const int rpt = map_rpt(pad4(p.d));
    if (p.tma_ok && p.n >= (int64_t)kThreads * rpt) {
        const size_t tail = mode == kMarkSmall ? (size_t)pw * sizeof(uint32_t) : 0;
        const size_t smem = (size_t)kMapStages * kThreads * rpt * p.d * sizeof(float) + tail;
        const int smem_max = kMapStages * kThreads * 16 * (int)sizeof(float) +
                             (int)kPrivWords * (int)sizeof(uint32_t);
        const int64_t nchunks = p.n / ((int64_t)kThreads * rpt);
        blocks = grid_for(nchunks, 1, kMapMaxBlocks);   // capped at one wave by map_tma
        SKY_DISPATCH_DP(p.d, {
            if (mode == kMarkSmall) map_tma<DP, kMarkSmall>(p, blocks, smem, smem_max, pw, s);
            else if (mode == kMarkNone) map_tma<DP, kMarkNone>(p, blocks, smem, smem_max, pw, s);
            else if (mode == kMarkByte) map_tma<DP, kMarkByte>(p, blocks, smem, smem_max, pw, s);
            else map_tma<DP, kMarkCheck>(p, blocks, smem, smem_max, pw, s);
        });
    } else {
        blocks = grid_for(p.n, kThreads * 4, std::min(num_sms() * 8, kMapMaxBlocks));
        const bool v = vec4_ok(p);
        const size_t smem = (size_t)pw * sizeof(uint32_t);
        SKY_DISPATCH_DP(p.d, {
            if (mode == kMarkSmall) map_plain<DP, kMarkSmall>(p, blocks, smem, pw, v, s);
            else if (mode == kMarkNone) map_plain<DP, kMarkNone>(p, blocks, smem, pw, v, s);
            else if (mode == kMarkByte) map_plain<DP, kMarkByte>(p, blocks, smem, pw, v, s);
            else map_plain<DP, kMarkCheck>(p, blocks, smem, pw, v, s);
        });
    }
    if (mode == kMarkSmall) {
        const int64_t cols = (p.words + 31) / 32;
        k_occ_merge<<<(unsigned)(cols * kMergeSplit), kThreads, 0, s>>>(p.occ_stage, blocks, p.words, p.occ);
    }
    if (mode == kMarkByte)
        k_occ_pack<<<grid_for(p.words, kThreads, num_sms() * 8), kThreads, 0, s>>>(p.occb, p.occ, p.words);
    return cudaGetLastError();
}

void launch_mm_reset(const Plan& p, cudaStream_t s)
{
    cudaMemsetAsync(p.mm_min, 0xff, sizeof(uint32_t) * kMaxDim, s);
    cudaMemsetAsync(p.mm_max, 0x00, sizeof(uint32_t) * kMaxDim, s);
}

// Min / max of p's rows folded into p.mm_min / p.mm_max (reset beforehand).
cudaError_t launch_minmax_accumulate(const Plan& p, cudaStream_t s)
{
    if (p.n == 0) return cudaGetLastError();
    const int blocks = grid_for(p.n, kThreads * 8, num_sms() * 8);
    const bool v = vec4_ok(p);
    SKY_DISPATCH_DP(p.d, k_minmax<DP><<<blocks, kThreads, 0, s>>>(p.pts, p.n, p.d, p.ld, v, p.mm_min, p.mm_max,
                                                                   &p.res->err));
    return cudaGetLastError();
}

// p.params for p.map_mode: min / max scales from p.mm_* (mode 2), the unit
// cube (mode 1), or the automatic rule over p's rows (mode 0).
// The automatic map's sample kernel (eight CTAs) also zeroes the result
// block and a bitmap of at most this many words (32 KB), saving the k_clear
// launch; a 2 MB bitmap cleared by those eight CTAs measured slower than a
// separate wide k_clear.
constexpr int64_t kFoldClearWords = int64_t(1) << 13;

// Words the call's first kernel zeroes: the bitmap, or the byte map
int64_t clear_words(const Plan& p) { return p.occb ? p.words * 8 : p.words; }

bool clear_folded(const Plan& p)
{
    return p.map_mode == kMapAuto && p.n > 0 && clear_words(p) <= kFoldClearWords;
}

ClearSet clear_of(const Plan& p)
{
    ClearSet c;
    c.res = p.res;
    c.occ = p.occb ? reinterpret_cast<uint32_t*>(p.occb) : p.occ;   // the pack rewrites every bitmap word
    c.words = clear_words(p);
    c.digit_total = p.digit_total;
    c.lb_counter = p.lb_counter;
    c.lb_states = p.lb_states;
    c.lb_tiles = p.lb_states ? p.lb_tiles : 0;
    if (p.cidx != nullptr && !p.survivors_only) {   // only the refinement reads it
        c.cidx = p.cidx;
        c.cidx_words = int64_t(2) << p.d;
        c.pre_states = p.pre_states;
    }
    return c;
}

cudaError_t launch_params(const Plan& p, cudaStream_t s, bool clear)
{
    if (p.map_mode == kMapMinMax) {
        k_params<<<1, 32, 0, s>>>(p.mm_min, p.mm_max, p.d, p.log2g, p.morton_bits, 1, p.params);
    } else if (p.map_mode == kMapUnit || p.n == 0) {
        k_params<<<1, 32, 0, s>>>(p.mm_min, p.mm_max, p.d, p.log2g, p.morton_bits, 0, p.params);
    } else {
        const bool v = vec4_ok(p);
        const ClearSet cs = clear && clear_folded(p) ? clear_of(p) : ClearSet{};
        SKY_DISPATCH_DP(p.d, k_sample_params<DP><<<kDecideCluster, kDecideThreads, 0, s>>>(
                                 p.pts, p.n, p.d, p.ld, v, p.log2g, p.morton_bits, p.mm_min, p.mm_max, p.params,
                                 cs));
    }
    return cudaGetLastError();
}

// Cleared result block and bitmap, and the value map's parameters (min / max
// pass in mode 2).
cudaError_t launch_build_params(const Plan& p, cudaStream_t s)
{
    if (!clear_folded(p))
        k_clear<<<grid_for(clear_words(p), kThreads * 16, num_sms() * 4), kThreads, 0, s>>>(clear_of(p));
    if (p.map_mode == kMapMinMax) launch_mm_reset(p, s);
    if (p.n == 0) return cudaGetLastError();
    if (p.map_mode == kMapMinMax) launch_minmax_accumulate(p, s);
    return launch_params(p, s, true);
}

cudaError_t launch_build(const Plan& p, cudaStream_t s)
{
    const cudaError_t e = launch_build_params(p, s);
    if (e != cudaSuccess || p.n == 0) return e;
    return launch_map_pass(p, true, s);
}

int build_kernel_count(const Plan& p)
{
    if (p.n == 0) return 1;
    const int merge = (p.occ_stage || p.occb) ? 1 : 0;   // merge of private bitmaps, or pack of the byte map
    if (p.map_mode == kMapMinMax) return 4 + merge;
    return (clear_folded(p) ? 2 : 3) + merge;   // (clear,) parameters, map pass (+ merge)
}

// Split of the prefix-OR: kl low dimensions per shared-memory block (at most
// 2^kPrefixLowBits bits, as many dimensions as fit), the rest in rows of the
// high grid (at most 2^14 rows). Grids of at most 2^16 bits are one block.
// kl = 0 selects the fallback of one launch per dimension.
struct PrefixSplit {
    int kl = 0, kh = 0;
    int64_t block_words = 0, rows = 0;
    int wc = 0;
    int64_t high_blocks = 0, low_blocks = 0;
};

PrefixSplit prefix_split(const Plan& p)
{
    PrefixSplit ps;
    const int lg = p.log2g, d = p.d, B = lg * d;
    if (B <= 16) {                       // the whole grid (at most 8 KB) in one block
        ps.kl = d;
        ps.block_words = p.words;
        ps.low_blocks = 1;
        return ps;
    }
    int kl = 0;
    while (kl + 1 < d && lg * (kl + 1) <= kPrefixLowBits) ++kl;
    if (kl < 1 || lg * kl < 5 || B - lg * kl > 14) return PrefixSplit{};
    ps.kl = kl;
    ps.kh = d - kl;
    ps.block_words = 1ll << (lg * kl - 5);
    ps.low_blocks = p.words / ps.block_words;
    ps.rows = 1ll << (B - lg * kl);
    int64_t wc = kPrefixHighWords / ps.rows;   // words of shared memory per block: coalesced rows
    if (wc < 1) wc = 1;
    // long lines leave few lines per block: widen the block (up to 64 KB)
    while ((ps.rows >> lg) * wc < 32 && ps.rows * wc * 2 <= 16384 && wc * 2 <= ps.block_words) wc *= 2;
    if (wc > ps.block_words) wc = ps.block_words;
    ps.wc = (int)wc;
    ps.high_blocks = ps.block_words / wc;
    return ps;
}

// At most two columns per dimension the survivor pass needs no prefix-OR:
// a cell with no zero column is then the all-ones cell, whose one-down
// neighbour is the origin, and the inclusive prefix-OR at the origin is the
// origin's occupancy bit. The pass's diagonal shortcut also reads the
// all-ones cell; with the occupancy bit there (not the OR of the whole grid)
// its threshold only moves between values >= 1, for which every such row
// still probes the origin. So the survivor pass reads the bitmap itself
// (log2g = 0: one cell, nothing is dominated and nothing is read).
bool prefix_trivial(const Plan& p)
{
    return p.log2g <= 1;
}

int prefix_kernel_count(const Plan& p)
{
    const PrefixSplit ps = prefix_split(p);
    if (ps.kl == 0) return p.d;
    return ps.kh > 0 ? 2 : 1;
}

cudaError_t launch_prefix_or(const Plan& p, cudaStream_t s)
{
    const PrefixSplit ps = prefix_split(p);
    if (ps.kl == 0) {
        cudaMemcpyAsync(p.pre, p.occ, sizeof(uint32_t) * p.words, cudaMemcpyDeviceToDevice, s);
        for (int k = 0; k < p.d; ++k) {
            const int blocks = grid_for(p.words, kThreads, num_sms() * 8);
            k_prefix_or_dim<<<blocks, kThreads, 0, s>>>(p.pre, p.words, p.log2g, k);
        }
        return cudaGetLastError();
    }
    const int smem_low = (int)(ps.block_words * sizeof(uint32_t));
    // about two words per thread, whole warps
    const int thr = (int)std::min<int64_t>(kPrefixLowThreads,
                                           std::max<int64_t>(64, ps.block_words / kPrefixWordsPerThread));
    cudaFuncSetAttribute(k_prefix_low, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_low);
    k_prefix_low<<<(unsigned)ps.low_blocks, thr, smem_low, s>>>(p.occ, p.pre, ps.block_words, p.log2g, ps.kl);
    if (ps.kh > 0) {
        const int smem_high = (int)(ps.rows * ps.wc * sizeof(uint32_t));
        int lrows = 0, lwc = 0;
        while ((1ll << lrows) < ps.rows) ++lrows;
        while ((1 << lwc) < ps.wc) ++lwc;
        cudaFuncSetAttribute(k_prefix_high, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_high);
        k_prefix_high<<<(unsigned)ps.high_blocks, kThreads, smem_high, s>>>(p.pre, ps.block_words, lrows, lwc,
                                                                             p.log2g, ps.kh);
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

void survivor_split(int64_t n, int64_t* tpb, int* blocks)
{
    const int64_t ntiles = (n + kSurvTile - 1) / kSurvTile;
    // six blocks per SM (4, 8 and 12 measured the same within a microsecond)
    int64_t target = (int64_t)num_sms() * 6;
    if (target > kSurvMaxBlocks) target = kSurvMaxBlocks;
    int64_t t = (ntiles + target - 1) / target;
    if (t < 1) t = 1;
    if (t > kSurvMaxTpb) t = kSurvMaxTpb;
    int64_t b = (ntiles + t - 1) / t;
    if (b < 1) b = 1;
    *tpb = t;
    *blocks = (int)b;
}

cudaError_t launch_survivors(const Plan& p, int n_filter, cudaStream_t s, uint32_t* idx_out)
{
    if (p.n == 0) return cudaGetLastError();
    int64_t tpb = 1;
    int blocks = 1;
    survivor_split(p.n, &tpb, &blocks);
    const bool v = vec4_ok(p);
    SKY_DISPATCH_DP(p.d, k_surv_flags<DP><<<blocks, kThreads, 0, s>>>(p.pts, p.n, p.d, p.ld, v, p.log2g, p.ckey,
                                                                        p.pre, p.filt, n_filter, p.res, tpb,
                                                                        p.sflags, p.scount,
                                                                        p.survivors_only ? nullptr : p.keep));
    const int smem = 2 * (int)tpb * (int)sizeof(uint32_t);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_surv_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_surv_scatter<<<blocks, kThreads, smem, s>>>(p.n, p.mkey, p.sflags, p.scount, tpb, p.res, p.surv_key,
                                                  idx_out ? idx_out : p.surv_idx);
    return cudaGetLastError();
}

cudaError_t launch_copy_survivors(const Plan& p, int32_t* out, int64_t capacity, cudaStream_t s)
{
    const int blocks = grid_for(p.n, kThreads * 4, num_sms() * 4);
    k_copy_survivors<<<blocks, kThreads, 0, s>>>(p.surv_idx, p.res, out, capacity);
    return cudaGetLastError();
}

cudaError_t launch_cell_stats(const Plan& p, cudaStream_t s)
{
    return launch_dominated(p, s);
}

// Automatic layer: the largest log2_g <= min(8, 24 / d) with 2^(log2_g d)
// <= 32 n. At most 256 columns per dimension (the paper's default layer is
// 6): finer layers of 2- and 3-dimensional sets prune little more and make
// every line of the prefix-OR long.
int auto_log2g(int64_t n, int d)
{
    int r = 24 / d;
    if (r < 1) r = 1;
    if (r > kMaxAutoLayer) r = kMaxAutoLayer;
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
