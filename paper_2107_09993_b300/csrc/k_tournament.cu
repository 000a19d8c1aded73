// k_tournament.cu -- the paper's tournament-tree ShrinkKeyCells (Algorithm 3,
// Sec. 5.2) on one grid layer, as a comparison variant of step (c): it
// produces the same dominated / key / candidate classes as the prefix-OR path
// (Theorem 2), by a different parallel schedule.
//
// Structure kept from Algorithm 3: the cells are the leaves of a complete
// binary tree, in the enumeration order of the current rotation of the
// dimensions; each pass runs an up-sweep that sets every node's pointer u
// from its two children, then a down-sweep that sets every node's pointer l
// (k = 0: its own u; k odd: its parent's l; k even: the combination of the l
// of the node before its parent and its own u); between passes the
// dimensions rotate (dimension k + 1 becomes k, dimension 0 the last) and
// every leaf's u takes the previous pass's l. Each level is one parallel
// step ("par-do"), one kernel launch.
//
// Reading (the printed form does not reproduce Definitions 4-5: a single
// pointer per node cannot hold a two-dimensional staircase, and the proof's
// mixed cells mu(c', c) must exist as leaves):
//   * leaves are all cells of the layer, so every mixed cell is a leaf;
//   * a pass compares in ONE dimension (the rotated dimension 0): two
//     pointers combine only within a line of cells that differ in that
//     dimension alone, and the earlier pointer wins ("1-domination"); d
//     passes cover the d dimensions;
//   * a pointer is a non-empty cell (a witness) or none; at the first pass a
//     leaf points to its own cell when the cell is non-empty.
// After pass m a leaf c points to a non-empty cell e != c with e[k] <= c[k]
// for the dimensions passed so far and e[k] = c[k] for the others, if there
// is one, else to c itself when c is non-empty, else to none. After the d
// passes (Theorem 2, as read here):
//   key        l(c) = c                                        (Def. 4)
//   dominated  every c[k] >= 1 and l(c - (1, ..., 1)) is a cell (Def. 3)
//   candidate  not dominated, and l(c) is a cell or c lies on the upper
//              boundary (the auxiliary key cells of Def. 6)      (Def. 5)
#include <cstdint>

#include "sky_common.cuh"
#include "sky_internal.h"

namespace sky {

namespace {

constexpr int kTT = 256;
constexpr int32_t kNone = -1;

// Cell (row-major key: dimension d-1 most significant) of the leaf at
// position pos under rotation m: rotated dimension k is dimension (k + m) % d.
__device__ __forceinline__ uint32_t leaf_cell(uint32_t pos, int d, int lg, int m)
{
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t cell = 0;
    for (int k = 0; k < d; ++k) {
        const uint32_t col = (pos >> (lg * k)) & mask;
        int dim = k + m;
        if (dim >= d) dim -= d;
        cell |= col << (lg * dim);
    }
    return cell;
}

// Combine the pointer of an earlier range (a) with that of a later range (b)
// whose last leaves are last_a < last_b: the earlier pointer wins when both
// ranges end on the same line of the rotated dimension 0 (positions in one
// line share pos >> lg) and the later range lies inside that line.
__device__ __forceinline__ int32_t combine(int32_t a, int32_t b, uint32_t first_b, uint32_t last_a, uint32_t last_b,
                                           int lg)
{
    const bool same_line = (last_a >> lg) == (last_b >> lg) && (first_b >> lg) == (last_b >> lg);
    if (a != kNone && same_line) return a;
    return b;
}

// Leaves: u = the previous pass's l (pass 0: the cell itself if occupied).
__global__ void __launch_bounds__(kTT) k_tt_leaves(const uint32_t* __restrict__ occ, const int32_t* __restrict__ prev,
                                                   int32_t* u0, uint32_t N, int d, int lg, int m)
{
    const uint32_t pos = blockIdx.x * kTT + threadIdx.x;
    if (pos >= N) return;
    const uint32_t cell = leaf_cell(pos, d, lg, m);
    int32_t v;
    if (m == 0) v = ((occ[cell >> 5] >> (cell & 31u)) & 1u) ? (int32_t)cell : kNone;
    else v = prev[cell];
    u0[pos] = v;
}

// Up-sweep, level j >= 1: node k covers leaves [k 2^j, (k + 1) 2^j).
__global__ void __launch_bounds__(kTT) k_tt_up(const int32_t* __restrict__ below, int32_t* up, uint32_t nodes, int j,
                                               int lg)
{
    const uint32_t k = blockIdx.x * kTT + threadIdx.x;
    if (k >= nodes) return;
    const uint32_t span = 1u << j, half = span >> 1;
    const uint32_t first_r = k * span + half;
    up[k] = combine(below[2 * k], below[2 * k + 1], first_r, first_r - 1u, k * span + span - 1u, lg);
}

// Down-sweep, level j (from the top): l of node k from its parent level's l
// (level j + 1) and its own u.
__global__ void __launch_bounds__(kTT) k_tt_down(const int32_t* __restrict__ u, const int32_t* __restrict__ lpar,
                                                 int32_t* l, uint32_t nodes, int j, int lg, int top)
{
    const uint32_t k = blockIdx.x * kTT + threadIdx.x;
    if (k >= nodes) return;
    if (j == top || k == 0) {
        l[k] = u[k];
    } else if (k & 1u) {
        l[k] = lpar[(k - 1) >> 1];
    } else {
        const uint32_t span = 1u << j;
        // the node before the parent ends just before this node starts
        l[k] = combine(lpar[k / 2 - 1], u[k], k * span, k * span - 1u, k * span + span - 1u, lg);
    }
}

// Leaf l pointers back to cell order for the next pass / the classes.
__global__ void __launch_bounds__(kTT) k_tt_scatter(const int32_t* __restrict__ l0, int32_t* by_cell, uint32_t N, int d,
                                                    int lg, int m)
{
    const uint32_t pos = blockIdx.x * kTT + threadIdx.x;
    if (pos >= N) return;
    by_cell[leaf_cell(pos, d, lg, m)] = l0[pos];
}

// Classes per cell: bit 0 dominated, bit 1 key, bit 2 candidate.
__global__ void __launch_bounds__(kTT) k_tt_classes(const int32_t* __restrict__ l, uint8_t* cls, uint32_t N, int d,
                                                    int lg)
{
    const uint32_t c = blockIdx.x * kTT + threadIdx.x;
    if (c >= N) return;
    const uint32_t G = 1u << lg, mask = G - 1u;
    bool pos_all = lg > 0, boundary = false;
    for (int k = 0; k < d; ++k) {
        const uint32_t col = (c >> (lg * k)) & mask;
        pos_all &= col >= 1u;
        boundary |= col == G - 1u;
    }
    const bool dominated = pos_all && l[c - ones_key(lg, d)] != kNone;
    const bool key = l[c] == (int32_t)c;
    const bool cand = !dominated && (l[c] != kNone || boundary);
    cls[c] = (uint8_t)((dominated ? 1u : 0u) | (key ? 2u : 0u) | (cand ? 4u : 0u));
}

unsigned blocks(uint32_t n) { return (n + kTT - 1) / kTT; }

}  // namespace

size_t tournament_workspace_bytes(int d, int log2g)
{
    const size_t N = size_t(1) << (log2g * d);
    // u and l for all levels (2N each) + the cell-ordered pointers (N)
    return sizeof(int32_t) * (4 * N + N) + 1024;
}

// Runs the d passes on the occupancy bitmap `occ` of one layer and writes the
// classes to cls[2^(log2g d)]. ws: tournament_workspace_bytes(d, log2g).
cudaError_t launch_tournament(const uint32_t* occ, int d, int log2g, uint8_t* cls, void* ws, cudaStream_t s)
{
    const int h = log2g * d;
    const uint32_t N = 1u << h;
    int32_t* U = static_cast<int32_t*>(ws);   // level j at U + (2N - 2^(h - j + 1)), 2^(h - j) nodes
    int32_t* L = U + 2 * (size_t)N;
    int32_t* byc = L + 2 * (size_t)N;
    auto lev = [&](int32_t* base, int j) { return base + (2 * (size_t)N - (size_t(2) << (h - j))); };
    for (int m = 0; m < d; ++m) {
        k_tt_leaves<<<blocks(N), kTT, 0, s>>>(occ, byc, lev(U, 0), N, d, log2g, m);
        for (int j = 1; j <= h; ++j) {
            const uint32_t nodes = N >> j;
            k_tt_up<<<blocks(nodes), kTT, 0, s>>>(lev(U, j - 1), lev(U, j), nodes, j, log2g);
        }
        for (int j = h; j >= 0; --j) {
            const uint32_t nodes = N >> j;
            k_tt_down<<<blocks(nodes), kTT, 0, s>>>(lev(U, j), j == h ? lev(L, j) : lev(L, j + 1), lev(L, j), nodes, j,
                                                    log2g, h);
        }
        k_tt_scatter<<<blocks(N), kTT, 0, s>>>(lev(L, 0), byc, N, d, log2g, m);
    }
    k_tt_classes<<<blocks(N), kTT, 0, s>>>(byc, cls, N, d, log2g);
    return cudaGetLastError();
}

int tournament_kernel_count(int d, int log2g)
{
    const int h = log2g * d;
    return d * (2 + h + (h + 1)) + 1;
}

}  // namespace sky
