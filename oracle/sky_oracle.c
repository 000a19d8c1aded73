/*
 * sky_oracle.c -- CPU oracle for the SkyCell skyline path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
 * this file; only the tests, the smoke check and the bench's CPU-baseline leg
 * do. It shares no source with the CUDA library: every function here is written
 * straight from the definitions in the paper, in plain C, favouring obviousness
 * over speed (loops over points may be spread over OpenMP threads; that does
 * not change what is computed).
 *
 * Contents (paper = Li, Gu, Qi, Yu, "SkyCell: A Space-Pruning Based Parallel
 * Skyline Algorithm", arXiv 2107.09993):
 *   orc_dominates         Definition 1 (point domination).
 *   orc_skyline_brute     Definition 2 (skyline set), literal double loop.
 *   orc_skyline_sfs       Sort-first skyline (Sec. 2.1, SFS): presort by the
 *                         Manhattan norm, test each point only against earlier
 *                         skyline points; blocks of equal-norm-free ranges run
 *                         in parallel.
 *   orc_dominator         first j with P_j dominating P_i (single-point check).
 *   orc_cell_params       per-dimension offset and scale of the value->column
 *                         map (Eq. 1 on the unit cube; min/max normalisation
 *                         for general data, see the reading below).
 *   orc_cell_keys         Eq. 1: column numbers of each point in Layer rho,
 *                         packed with dimension d-1 most significant.
 *   orc_cell_classes      Definitions 3-5 and 6 (auxiliary key cells) by
 *                         direct enumeration over all cells of one layer.
 *
 * Readings of points the paper leaves open:
 *   - Eq. 1 assumes data in [0,1)^d. General data is mapped with
 *     t = (x - min_k) * s_k, s_k = G / (max_k - min_k), both operations in
 *     IEEE binary32 round-to-nearest with no fused multiply-add, then
 *     column = clamp(floor(t), 0, G-1). With the unit-cube assumption,
 *     min_k = 0 and s_k = G. Range 0 gives s_k = 0 (every point in column 0);
 *     an infinite range gives s_k = G / FLT_MAX. Every such map is monotone
 *     non-decreasing in x, which is all that cell pruning needs. The
 *     automatic choice looks at a strided sample of at most 4096 rows: it
 *     keeps Eq. 1 when every sampled dimension lies in [0,1] and spans at
 *     least half of it, and normalises by the sample's range otherwise.
 *   - Non-finite inputs are outside the method (they break the order); callers
 *     of the oracle must not pass them.
 *   - Cell keys: key = sum_k column_k << (log2G * k), i.e. dimension d-1 is
 *     the most significant, matching the paper's L[cl_{d-1}, ..., cl_0].
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fno-fast-math -shared -fPIC
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* ---------------------------------------------------------------------- */
/* Definition 1: p dominates q iff p[k] <= q[k] for all k and p[l] < q[l]  */
/* for some l ("smaller is better").                                      */
/* ---------------------------------------------------------------------- */
ORC_API int orc_dominates(const float* p, const float* q, int d)
{
    int strictly_better_somewhere = 0;
    for (int k = 0; k < d; ++k) {
        if (p[k] > q[k]) return 0;
        if (p[k] < q[k]) strictly_better_somewhere = 1;
    }
    return strictly_better_somewhere;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

ORC_API int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Definition 2: the skyline is every point not dominated by another      */
/* point. Writes the skyline's row indices in ascending order to `out`    */
/* (capacity n) and returns how many there are.                           */
/* ---------------------------------------------------------------------- */
ORC_API int64_t orc_skyline_brute(const float* P, int64_t n, int d, int64_t ld,
                                  int32_t* out, int nthreads)
{
    unsigned char* is_sky = (unsigned char*)malloc((size_t)(n > 0 ? n : 1));
    if (!is_sky) return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int dominated = 0;
        for (int64_t j = 0; j < n && !dominated; ++j) {
            if (j == i) continue;
            if (orc_dominates(P + j * ld, P + i * ld, d)) dominated = 1;
        }
        is_sky[i] = (unsigned char)!dominated;
    }
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i)
        if (is_sky[i]) out[s++] = (int32_t)i;
    free(is_sky);
    return s;
}

/* First j (ascending) whose point dominates point i, or -1 when i is a
 * skyline point. O(n d). */
ORC_API int64_t orc_dominator(const float* P, int64_t n, int d, int64_t ld, int64_t i)
{
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        if (orc_dominates(P + j * ld, P + i * ld, d)) return j;
    }
    return -1;
}

/* Many independent single-point checks, spread over threads. */
ORC_API void orc_dominators(const float* P, int64_t n, int d, int64_t ld,
                            const int64_t* idx, int64_t m, int64_t* witness,
                            int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < m; ++t) witness[t] = orc_dominator(P, n, d, ld, idx[t]);
}

/* ---------------------------------------------------------------------- */
/* Sort-first skyline (SFS, Sec. 2.1): order the points by Manhattan norm */
/* (sum of coordinates). A point can only be dominated by a point whose   */
/* norm is not larger (the rounded float64 sum is monotone in each        */
/* coordinate, so rounding can at most make the two norms equal), and if  */
/* any point dominates p then a skyline point does (transitivity). So p   */
/* is tested against the skyline points found in earlier norm blocks and  */
/* against every point of its own block. Block boundaries never split a   */
/* run of equal norms.                                                    */
/* ---------------------------------------------------------------------- */
typedef struct { double norm; int64_t idx; } orc_norm_t;

static int cmp_norm(const void* a, const void* b)
{
    const orc_norm_t* x = (const orc_norm_t*)a;
    const orc_norm_t* y = (const orc_norm_t*)b;
    if (x->norm < y->norm) return -1;
    if (x->norm > y->norm) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

ORC_API int64_t orc_skyline_sfs(const float* P, int64_t n, int d, int64_t ld,
                                int32_t* out, int nthreads)
{
    if (n <= 0) return 0;
    orc_norm_t* ord = (orc_norm_t*)malloc(sizeof(orc_norm_t) * (size_t)n);
    int64_t* window = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    unsigned char* keep = (unsigned char*)malloc((size_t)n);
    if (!ord || !window || !keep) { free(ord); free(window); free(keep); return -1; }
    set_threads(nthreads);
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += (double)P[i * ld + k];
        ord[i].norm = s;
        ord[i].idx = i;
    }
    qsort(ord, (size_t)n, sizeof(orc_norm_t), cmp_norm);

    int64_t nwin = 0;
    const int64_t block = 4096;
    int64_t pos = 0;
    while (pos < n) {
        int64_t end = pos + block < n ? pos + block : n;
        while (end < n && ord[end].norm == ord[end - 1].norm) ++end;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t t = pos; t < end; ++t) {
            const float* p = P + ord[t].idx * ld;
            int dominated = 0;
            for (int64_t w = 0; w < nwin && !dominated; ++w)
                if (orc_dominates(P + window[w] * ld, p, d)) dominated = 1;
            for (int64_t u = pos; u < end && !dominated; ++u) {
                if (u == t) continue;
                if (orc_dominates(P + ord[u].idx * ld, p, d)) dominated = 1;
            }
            keep[t] = (unsigned char)!dominated;
        }
        for (int64_t t = pos; t < end; ++t)
            if (keep[t]) window[nwin++] = ord[t].idx;
        pos = end;
    }
    for (int64_t w = 0; w < nwin; ++w) out[w] = (int32_t)window[w];
    qsort(out, (size_t)nwin, sizeof(int32_t), cmp_i32);
    free(ord); free(window); free(keep);
    return nwin;
}

/* ---------------------------------------------------------------------- */
/* Value -> column map (Eq. 1 and its min/max reading, see header).       */
/* mode 1: unit cube, Eq. 1 as printed (offset 0, scale G).               */
/* mode 2: min/max normalisation of every dimension over all n rows.      */
/* mode 0: automatic, from the strided sample S of rows 0, t, 2t, ... < n */
/*         with t = ceil(n / 4096) (at most 4096 rows): Eq. 1 when every  */
/*         dimension of S lies in [0,1] and spans at least half of it     */
/*         (max - min >= 0.5 in binary32), otherwise normalisation by S's */
/*         per-dimension min / max. Rows outside S's range land in the   */
/*         first / last column; the map is still monotone.                */
/* `offset` and `scale` receive d floats each.                            */
/* ---------------------------------------------------------------------- */
#define ORC_DECIDE_SAMPLE 4096

ORC_API void orc_cell_params(const float* P, int64_t n, int d, int64_t ld,
                             int log2g, int mode, float* offset, float* scale)
{
    const float G = (float)(1u << log2g);
    float mn[64], mx[64];
    int unit = (mode == 1) || n <= 0;
    if (!unit) {
        /* rows visited: all of them (mode 2) or the sample (mode 0) */
        int64_t step = 1;
        if (mode == 0) step = (n + ORC_DECIDE_SAMPLE - 1) / ORC_DECIDE_SAMPLE;
        if (step < 1) step = 1;
        for (int k = 0; k < d; ++k) {
            mn[k] = P[k];
            mx[k] = P[k];
            for (int64_t i = step; i < n; i += step) {
                float v = P[i * ld + k];
                if (v < mn[k]) mn[k] = v;
                if (v > mx[k]) mx[k] = v;
            }
        }
        if (mode == 0) {
            unit = 1;
            for (int k = 0; k < d; ++k) {
                volatile float span = mx[k] - mn[k];
                if (!(mn[k] >= 0.0f && mx[k] <= 1.0f && span >= 0.5f)) unit = 0;
            }
        }
    }
    for (int k = 0; k < d; ++k) {
        if (unit) { offset[k] = 0.0f; scale[k] = G; continue; }
        volatile float range = mx[k] - mn[k];  /* binary32, round to nearest */
        offset[k] = mn[k];
        if (range == 0.0f) scale[k] = 0.0f;
        else if (isinf(range)) scale[k] = G / FLT_MAX;
        else scale[k] = G / range;             /* correctly rounded binary32 division */
    }
}

static inline uint32_t column_of(float x, float off, float s, int log2g)
{
    const uint32_t G = 1u << log2g;
    if (s == 0.0f) return 0u;
    volatile float diff = x - off;             /* no contraction with the multiply */
    volatile float t = diff * s;
    if (!(t > 0.0f)) return 0u;                /* negative (unit assumption) or zero */
    if (t >= (float)G) return G - 1u;
    uint32_t c = (uint32_t)floorf(t);
    return c > G - 1u ? G - 1u : c;
}

/* Eq. 1: key of the Layer-log2g cell of every point. */
ORC_API void orc_cell_keys(const float* P, int64_t n, int d, int64_t ld, int log2g,
                           const float* offset, const float* scale, uint64_t* keys)
{
    for (int64_t i = 0; i < n; ++i) {
        uint64_t key = 0;
        for (int k = d - 1; k >= 0; --k)
            key = (key << log2g) | column_of(P[i * ld + k], offset[k], scale[k], log2g);
        keys[i] = key;
    }
}

/* ---------------------------------------------------------------------- */
/* Definitions 3-6 by enumeration over the G^d cells of one layer.        */
/*   occ[c]        1 if cell c holds a point (input, G^d bytes)           */
/*   dominated[c]  some non-empty c' has c'[k] < c[k] for every k (Def. 3)*/
/*   key[c]        non-empty, and no other non-empty cell c' has          */
/*                 c'[k] <= c[k] for all k (neither dominates nor         */
/*                 partially dominates it; Def. 4)                        */
/*   candidate[c]  Def. 5 with the auxiliary key cells of Def. 6 / Lemma 2*/
/*                 counted as key cells (footnote to Theorem 1): c is a   */
/*                 key cell, or it is partially dominated by a key cell   */
/*                 (an auxiliary one when some c[j] = G-1) and dominated  */
/*                 by no key cell.                                        */
/* Cells are numbered by their key (dimension d-1 most significant).      */
/* Returns the number of candidate cells. O(G^(2d) d): tiny grids only.   */
/* ---------------------------------------------------------------------- */
static void decode_cell(uint64_t c, int d, int log2g, int* col)
{
    const uint64_t mask = (1ull << log2g) - 1ull;
    for (int k = 0; k < d; ++k) { col[k] = (int)(c & mask); c >>= log2g; }
}

ORC_API int64_t orc_cell_classes(const unsigned char* occ, int d, int log2g,
                                 unsigned char* dominated, unsigned char* key,
                                 unsigned char* candidate)
{
    const int G = 1 << log2g;
    const uint64_t ncell = 1ull << (log2g * d);
    int a[64], b[64];
    /* key cells (Def. 4) and dominated cells (Def. 3) */
    for (uint64_t c = 0; c < ncell; ++c) {
        decode_cell(c, d, log2g, a);
        int dom = 0, below = 0;
        for (uint64_t e = 0; e < ncell; ++e) {
            if (e == c || !occ[e]) continue;
            decode_cell(e, d, log2g, b);
            int all_lt = 1, all_le = 1;
            for (int k = 0; k < d; ++k) {
                if (!(b[k] < a[k])) all_lt = 0;
                if (!(b[k] <= a[k])) all_le = 0;
            }
            if (all_lt) dom = 1;
            if (all_le) below = 1;
        }
        dominated[c] = (unsigned char)dom;
        key[c] = (unsigned char)(occ[c] && !below);
    }
    /* candidate cells (Def. 5) with the auxiliary key cells of Def. 6:   */
    /* Lambda_j has column G-1 in dimension j and -1 elsewhere, so it     */
    /* partially dominates exactly the cells with c[j] = G-1 (Lemma 2)    */
    /* and dominates no cell of the layer.                                */
    int64_t count = 0;
    for (uint64_t c = 0; c < ncell; ++c) {
        decode_cell(c, d, log2g, a);
        int cand = key[c];
        if (!cand) {
            int dom_by_key = 0, pdom_by_key = 0;
            for (uint64_t e = 0; e < ncell; ++e) {
                if (!key[e]) continue;
                decode_cell(e, d, log2g, b);
                int all_lt = 1, all_le = 1, some_eq = 0;
                for (int k = 0; k < d; ++k) {
                    if (!(b[k] < a[k])) all_lt = 0;
                    if (!(b[k] <= a[k])) all_le = 0;
                    if (b[k] == a[k]) some_eq = 1;
                }
                if (all_lt) dom_by_key = 1;
                if (all_le && some_eq) pdom_by_key = 1;
            }
            for (int j = 0; j < d; ++j)
                if (a[j] == G - 1) pdom_by_key = 1;   /* auxiliary key cell Lambda_j */
            cand = pdom_by_key && !dom_by_key;
        }
        candidate[c] = (unsigned char)cand;
        count += cand;
    }
    return count;
}
