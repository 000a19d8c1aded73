// sky_seq.cu -- the paper's sequential SkyCell (Alg. 1 driving the sequential
// ShrinkKeyCells of Alg. 2) on the host: the CPU baseline the GPU path is
// timed against. Host code only; no GPU entry point calls it, and it shares
// no code with the test oracle.
//
// Structure (Sec. 4, Alg. 1, Alg. 2), with the readings stated in the header:
//   1. every point's Layer-rho cell (Eq. 1) and the occupancy of Layers
//      rho .. 0 (a Layer-i cell is non-empty iff one of its 2^d children is);
//   2. Layer by layer, i = 0 .. rho, the cells of a layer are enumerated
//      slice by slice: a slice bb = [cl_{d-1}, .., cl_1] in the paper's
//      order (dimension d-1 outermost), and inside it cl_0 upward from a
//      start bound GS[bb] up to an end bound GE[bb]:
//        - GS[bb] = 2 * (first non-empty column of the parent slice bb / 2
//          in Layer i-1): a lower column of this slice would lie in an empty
//          Layer-(i-1) cell (the role of step (a) of Alg. 2);
//        - GE[bb] = min over the slices bb - e_k (one lower in dimension k)
//          of their inclusive minimum M (the role of MinGE): a cell at or
//          above it is partially dominated by a non-empty cell of a lower
//          slice, so the scan stops there;
//        - the first non-empty cell below GE[bb] is a key cell (Def. 4).
//      M[bb] = min(first non-empty column of bb, min_k M[bb - e_k]) is the
//      minimum column of a non-empty cell over the slices <= bb.
//   3. Layer rho: cell [bb, c] is dominated (Def. 3) iff some non-empty cell
//      lies strictly below it in every dimension, i.e. iff c > M[bb - 1]
//      (every slice dimension >= 1); the points of the other cells are the
//      candidates;
//   4. RefineSkyline across candidate cells (a point of one candidate cell
//      can dominate a point of another): sort-first skyline, points ordered
//      by their coordinate sum, each tested against the skyline points found
//      so far and against the points of equal sum.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/sky.h"

namespace {

thread_local std::string s_err;

sky_status seq_fail(sky_status s, const char* msg)
{
    s_err = msg;
    return s;
}

// Eq. 1 on the unit cube (mode 1) or after the min / max of all rows: the
// same binary32 expressions as the GPU path's value map (subtract, multiply,
// floor, clamp), written here independently.
struct ValueMap {
    float off[16], scale[16];
    int d;
    uint32_t G;
    uint32_t column(float x, int k) const
    {
        volatile float t = (x - off[k]);   // two roundings, no contraction
        t = t * scale[k];
        const float f = std::floor(t);
        if (!(f > 0.0f)) return 0u;   // negative, zero or NaN
        if (f >= (float)(G - 1u)) return G - 1u;
        return (uint32_t)f;
    }
};

bool make_map(const float* P, int64_t n, int d, int64_t ld, int log2g, bool unit, ValueMap& m)
{
    m.d = d;
    m.G = 1u << log2g;
    for (int k = 0; k < d; ++k) {
        if (unit) {
            m.off[k] = 0.0f;
            m.scale[k] = (float)m.G;
            continue;
        }
        float lo = INFINITY, hi = -INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            const float x = P[i * ld + k];
            lo = std::min(lo, x);
            hi = std::max(hi, x);
        }
        volatile float range = hi - lo;
        m.off[k] = lo;
        if (range == 0.0f) m.scale[k] = 0.0f;
        else if (std::isinf((float)range)) m.scale[k] = (float)m.G / FLT_MAX;
        else m.scale[k] = (float)m.G / range;
    }
    return true;
}

// One layer's slice tables: F = first non-empty column found (or the bound
// the scan stopped at: no non-empty column below it), M = inclusive minimum.
struct Layer {
    int log2g = 0;
    uint32_t G = 1;
    int64_t slices = 1;              // G^(d-1)
    std::vector<uint8_t> occ;        // G^d cells, key = sum c[k] G^k
    std::vector<uint32_t> F, M;
};

// Slice index of bb = [cl_{d-1}, .., cl_1]: sum_{k>=1} cl_k G^(k-1); the cell
// key of [bb, c] is slice * G + c.
void shrink_layer(Layer& L, const Layer* parent, int d, std::vector<int64_t>* keys_out)
{
    const uint32_t G = L.G;
    L.F.assign((size_t)L.slices, G);
    L.M.assign((size_t)L.slices, G);
    std::vector<uint32_t> bb(d > 1 ? d - 1 : 1, 0u);   // bb[k-1] = cl_k
    std::vector<int64_t> stride(d > 1 ? d - 1 : 1, 1);
    for (int k = 1; k < d - 1; ++k) stride[k] = stride[k - 1] * G;
    for (int64_t s = 0; s < L.slices; ++s) {
        // GE: partial domination from the slices one lower in each dimension
        uint32_t ge = G;
        for (int k = 0; k < d - 1; ++k)
            if (bb[k] > 0) ge = std::min(ge, L.M[(size_t)(s - stride[k])]);
        // GS: the parent slice's first non-empty column, doubled
        uint32_t gs = 0;
        if (parent) {
            int64_t ps = 0, pstride = 1;
            for (int k = 0; k < d - 1; ++k) {
                ps += (int64_t)(bb[k] >> 1) * pstride;
                pstride *= parent->G;
            }
            gs = 2u * parent->F[(size_t)ps];
        }
        uint32_t first = ge;   // nothing found below ge
        const uint8_t* row = L.occ.data() + s * (int64_t)G;
        for (uint32_t c = gs; c < ge; ++c) {
            if (row[c]) {
                first = c;
                if (keys_out) keys_out->push_back(s * (int64_t)G + c);   // key cell (Def. 4)
                break;
            }
        }
        L.F[(size_t)s] = first;
        L.M[(size_t)s] = std::min(first, ge);
        // next slice in the paper's order (dimension 1 fastest)
        for (int k = 0; k < d - 1; ++k) {
            if (++bb[k] < G) break;
            bb[k] = 0;
        }
    }
}

// Layers rho .. 0 and their tables; cell keys of the points at Layer rho.
bool build_layers(const float* P, int64_t n, int d, int64_t ld, int rho, bool unit, std::vector<Layer>& layers,
                  std::vector<uint32_t>& cell, std::vector<int64_t>* keys_rho)
{
    ValueMap vm;
    make_map(P, n, d, ld, rho, unit, vm);
    layers.assign((size_t)rho + 1, Layer{});
    for (int i = 0; i <= rho; ++i) {
        Layer& L = layers[(size_t)i];
        L.log2g = i;
        L.G = 1u << i;
        L.slices = (int64_t)1 << (i * (d - 1));
        L.occ.assign((size_t)1 << (i * d), 0u);
    }
    cell.resize((size_t)n);
    for (int64_t r = 0; r < n; ++r) {
        uint32_t key = 0;
        for (int k = d - 1; k >= 0; --k) key = (key << rho) | vm.column(P[r * ld + k], k);
        cell[(size_t)r] = key;
        layers[(size_t)rho].occ[key] = 1u;
    }
    // Layer i-1 cell of a Layer-i cell: every column halved
    for (int i = rho; i > 0; --i) {
        const Layer& C = layers[(size_t)i];
        Layer& Pn = layers[(size_t)i - 1];
        const uint32_t mask = (1u << i) - 1u;
        for (size_t key = 0; key < C.occ.size(); ++key) {
            if (!C.occ[key]) continue;
            uint32_t pk = 0;
            for (int k = d - 1; k >= 0; --k) pk = (pk << (i - 1)) | (((uint32_t)(key >> (i * k)) & mask) >> 1);
            Pn.occ[pk] = 1u;
        }
    }
    for (int i = 0; i <= rho; ++i)
        shrink_layer(layers[(size_t)i], i ? &layers[(size_t)i - 1] : nullptr, d, i == rho ? keys_rho : nullptr);
    return true;
}

bool dominates(const float* a, const float* b, int d)
{
    bool lt = false;
    for (int k = 0; k < d; ++k) {
        if (a[k] > b[k]) return false;
        if (a[k] < b[k]) lt = true;
    }
    return lt;
}

sky_status check_args(const float* P, int64_t n, int32_t d, int64_t ld, int rho)
{
    if (d < 1 || d > 16) return seq_fail(SKY_ERR_INVALID_ARGUMENT, "d outside [1, 16]");
    if (n < 0 || n >= (int64_t(1) << 31)) return seq_fail(SKY_ERR_INVALID_ARGUMENT, "n outside [0, 2^31)");
    if (ld < d) return seq_fail(SKY_ERR_INVALID_ARGUMENT, "ld < d");
    if (n > 0 && !P) return seq_fail(SKY_ERR_INVALID_ARGUMENT, "points pointer is NULL");
    if (rho < 0 || rho * d > 24) return seq_fail(SKY_ERR_TOO_LARGE, "layer tables above 2^24 cells (rho * d > 24)");
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < d; ++k)
            if (!std::isfinite(P[i * ld + k])) return seq_fail(SKY_ERR_NONFINITE, "input holds NaN or infinity");
    return SKY_OK;
}

int default_layer(int64_t n, int d)
{
    // the GPU path's automatic rule (largest rho <= min(8, 24 / d) with
    // 2^(rho d) <= 32 n), restated
    int r = std::min(8, std::max(1, 24 / d));
    while (r > 1 && std::ldexp(1.0, r * d) > 32.0 * (double)std::max<int64_t>(n, 1)) --r;
    return r;
}

}  // namespace

extern "C" {

SKY_API sky_status sky_baseline_sequential(const float* h_pts, int64_t n, int32_t d, int64_t ld, int32_t log2_g,
                                           int32_t assume_unit, int32_t* h_out, int64_t capacity,
                                           int64_t* h_count, int64_t* h_candidates)
{
    if (!h_count) return seq_fail(SKY_ERR_INVALID_ARGUMENT, "h_count is NULL");
    *h_count = 0;
    if (assume_unit != 0 && assume_unit != 1) return seq_fail(SKY_ERR_INVALID_ARGUMENT, "assume_unit outside {0, 1}");
    const int rho = log2_g >= 0 ? log2_g : default_layer(n, d);
    sky_status st = check_args(h_pts, n, d, ld, rho);
    if (st != SKY_OK) return st;
    if (capacity < 0 || (capacity > 0 && !h_out)) return seq_fail(SKY_ERR_INVALID_ARGUMENT, "bad output buffer");
    if (n == 0) return SKY_OK;
    try {
        std::vector<Layer> layers;
        std::vector<uint32_t> cell;
        build_layers(h_pts, n, d, ld, rho, assume_unit == 1, layers, cell, nullptr);
        const Layer& L = layers[(size_t)rho];
        // candidates: points whose cell is not dominated (Def. 3)
        const uint32_t G = L.G, mask = G - 1u;
        std::vector<int32_t> cand;
        for (int64_t r = 0; r < n; ++r) {
            const uint32_t key = cell[(size_t)r];
            const uint32_t c0 = key & mask;
            bool below = c0 > 0;   // every column >= 1: a cell one step down the diagonal exists
            int64_t sp = 0, str = 1;
            for (int k = 1; k < d && below; ++k) {
                const uint32_t ck = (key >> (rho * k)) & mask;
                if (ck == 0) below = false;
                sp += (int64_t)(ck - 1) * str;
                str *= G;
            }
            // (d = 1: the one slice; dominated iff a lower column is non-empty)
            const bool dominated = below && c0 > L.M[(size_t)sp];
            if (!dominated) cand.push_back((int32_t)r);
        }
        if (h_candidates) *h_candidates = (int64_t)cand.size();
        // RefineSkyline: sort-first skyline over the candidates
        std::vector<double> sum(cand.size());
        for (size_t i = 0; i < cand.size(); ++i) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += (double)h_pts[(int64_t)cand[i] * ld + k];
            sum[i] = s;
        }
        std::vector<size_t> order(cand.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return sum[a] < sum[b]; });
        std::vector<int32_t> sky;      // skyline rows found so far (all of smaller sum)
        size_t g0 = 0;
        while (g0 < order.size()) {
            size_t g1 = g0 + 1;
            while (g1 < order.size() && sum[order[g1]] == sum[order[g0]]) ++g1;
            // a dominator has a sum <= its victim's (sums are monotone):
            // test each point of the group against the earlier skyline and
            // against the other points of the group
            std::vector<int32_t> keep;
            for (size_t a = g0; a < g1; ++a) {
                const int32_t ra = cand[order[a]];
                const float* pa = h_pts + (int64_t)ra * ld;
                bool dom = false;
                for (size_t j = 0; j < sky.size() && !dom; ++j) dom = dominates(h_pts + (int64_t)sky[j] * ld, pa, d);
                for (size_t b = g0; b < g1 && !dom; ++b)
                    if (b != a) dom = dominates(h_pts + (int64_t)cand[order[b]] * ld, pa, d);
                if (!dom) keep.push_back(ra);
            }
            sky.insert(sky.end(), keep.begin(), keep.end());
            g0 = g1;
        }
        std::sort(sky.begin(), sky.end());
        *h_count = (int64_t)sky.size();
        if ((int64_t)sky.size() > capacity) return seq_fail(SKY_ERR_CAPACITY, "skyline larger than the output buffer");
        std::memcpy(h_out, sky.data(), sky.size() * sizeof(int32_t));
    } catch (const std::bad_alloc&) {
        return seq_fail(SKY_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    return SKY_OK;
}

SKY_API sky_status sky_baseline_key_cells(const float* h_pts, int64_t n, int32_t d, int64_t ld, int32_t log2_g,
                                          int32_t assume_unit, int64_t* h_keys, int64_t capacity, int64_t* h_count)
{
    if (!h_count) return seq_fail(SKY_ERR_INVALID_ARGUMENT, "h_count is NULL");
    *h_count = 0;
    if (assume_unit != 0 && assume_unit != 1) return seq_fail(SKY_ERR_INVALID_ARGUMENT, "assume_unit outside {0, 1}");
    if (log2_g < 0) return seq_fail(SKY_ERR_INVALID_ARGUMENT, "log2_g must be given");
    sky_status st = check_args(h_pts, n, d, ld, log2_g);
    if (st != SKY_OK) return st;
    if (capacity < 0 || (capacity > 0 && !h_keys)) return seq_fail(SKY_ERR_INVALID_ARGUMENT, "bad output buffer");
    if (n == 0) return SKY_OK;
    try {
        std::vector<Layer> layers;
        std::vector<uint32_t> cell;
        std::vector<int64_t> keys;
        build_layers(h_pts, n, d, ld, log2_g, assume_unit == 1, layers, cell, &keys);
        *h_count = (int64_t)keys.size();
        if ((int64_t)keys.size() > capacity) return seq_fail(SKY_ERR_CAPACITY, "more key cells than the buffer holds");
        std::memcpy(h_keys, keys.data(), keys.size() * sizeof(int64_t));
    } catch (const std::bad_alloc&) {
        return seq_fail(SKY_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    return SKY_OK;
}

SKY_API const char* sky_baseline_last_error(void) { return s_err.c_str(); }

}  // extern "C"
