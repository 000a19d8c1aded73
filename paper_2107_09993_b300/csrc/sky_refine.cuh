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
// of 32, plus a producer warp. The producer scans the q-tiles up to the last
// one that can hold a dominator (the p-tile itself first, then the rest in
// ascending Morton order), keeps those whose byte-wise minimum code is <= the
// byte-wise maximum
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
// Only the codes of a q-tile are streamed (1-2 KB a tile); the rare exact
// test reads q's coordinates from global memory (the survivor layout is
// L2-resident). Small stages allow a deep ring: the tile stream, not the
// tests, bounds sets whose points die early.
#ifndef SKY_REFINE_STAGES
#define SKY_REFINE_STAGES 8
#endif
#ifndef SKY_REFINE_SUMMARY
#define SKY_REFINE_SUMMARY 32
#endif
#ifndef SKY_REFINE_UNROLL
#define SKY_REFINE_UNROLL 1
#endif
constexpr int kRingStages = SKY_REFINE_STAGES;
constexpr uint32_t kSummaryEvery = SKY_REFINE_SUMMARY;   // issued tiles between refreshes of the group maxima
constexpr int kPUnroll = SKY_REFINE_UNROLL;              // listed p's tested per loop step (1 or 2)
static_assert(kPUnroll == 1 || kPUnroll == 2, "one or two p's per step");
// 1: the listed p's of a group are compacted into a per-warp list in shared
// memory and tested branch-free four at a time (hits collected as bits and
// resolved afterwards); 0: a bit-scan loop over the ballot, one branch per p
// When at most this many p's of a CTA are still live at the start of a
// super-tile, the ring stops and the rest of the scan runs in sparse mode:
// all five warps walk the remaining q-tiles themselves, 32 tiles at a time
// (one lane per tile tests the tile's minimum code against each live p),
// and test each relevant tile's 128 q's, four per lane, against only the
// live p's that tile can reach -- no producer, no stage handshakes. 0: off.
// SKY_REFINE_SPARSE applies below padded dimension 12, SKY_REFINE_SPARSE_HIGH
// from 12 up (where the sparse walk has the layer-1 cell index): measured on
// B300 with the index, 10 instead of 6 took 10^7 x 12 independent 41.3 ->
// 40.5 ms (10^7 x 16 anti-correlated unchanged) but 10^6 x 8 independent
// 0.72 -> 0.75 ms.
#ifndef SKY_REFINE_SPARSE
#define SKY_REFINE_SPARSE 6
#endif
#ifndef SKY_REFINE_SPARSE_HIGH
#define SKY_REFINE_SPARSE_HIGH 10
#endif
template <int DP>
struct SparseLive {
    static constexpr uint32_t value = DP >= 12 ? SKY_REFINE_SPARSE_HIGH : SKY_REFINE_SPARSE;
    static_assert(value <= 32, "the sparse list is one lane mask wide");
};
#ifndef SKY_REFINE_LIST
#define SKY_REFINE_LIST 1
#endif
// The single-set producer tests relevance against register copies of the
// group maxima up to this padded dimension (beyond it, against shared memory)
#ifndef SKY_REFINE_REGMAX_DP
#define SKY_REFINE_REGMAX_DP 16
#endif
// 1: the producer holds one sub-tile minimum in registers at a time (fewer
// registers at high d); 0: all five minima of a tile at once
// Fast codes: the list probe first compares 3-bit codes (the top three bits
// of the 7-bit codes, eight dimensions to a 32-bit word with a guard bit per
// nibble) and runs the 7-bit test only on the pairs that pass -- a necessary
// condition, so nothing is lost. Used from this padded dimension up; beyond
// the compile-time maximum, off.
#ifndef SKY_REFINE_FAST_MIN_DP
#define SKY_REFINE_FAST_MIN_DP 16
#endif
// Windows of 32 q-tiles whose sub-tile minima the producer has in flight
// (bulk copies into a ring of shared-memory buffers): the producer's scan
// over the windows waits on one of these copies per window, so at high d,
// where few tiles of a window are relevant, the depth of this ring sets the
// pace of the stream.
#ifndef SKY_REFINE_WINDOWS
#define SKY_REFINE_WINDOWS 2
#endif
// One buffer (no copy in flight ahead of the window being examined) ended a
// launch with an unspecified launch failure on B300 whose cause was not
// found by reading the code; it is not built.
static_assert(SKY_REFINE_WINDOWS >= 2, "at least two window buffers");
// 1: the CTA's own p coordinates are staged in shared memory for the exact
// tests; 0: the exact tests read them from global memory (rare, and the
// shared memory goes to deeper rings)
#ifndef SKY_REFINE_PX_SMEM
#define SKY_REFINE_PX_SMEM 1
#endif
// 1: with fast codes, a block of listed entries is first reduced to one
// "any pass" word (a running minimum) and the per-entry hit bits are formed
// only for the rare blocks that hold a pass. Measured on B300 at d = 16: no
// gain (10^7 x 16 anti-correlated 124.6 -> 125.7 ms), so off
#ifndef SKY_REFINE_MIN_PROBE
#define SKY_REFINE_MIN_PROBE 0
#endif
constexpr bool kMinProbe = SKY_REFINE_MIN_PROBE != 0;
// 1: the (sub-tile, group) pairs of a stage are dealt to the consumer warps
// in turn; 0: consumer warp w takes sub-tile w of every stage. Clock
// counters (a copy outside the tree) showed the consumer warps waiting 27 %
// and the producer 46 % of their time at 2*10^6 x 16, but dealing the pairs
// measured slower on B300 (10^7 x 16 anti-correlated 124.6 -> 155.5 ms,
// 4,096-query batch 525 -> 631 ms): more sub-tile reloads per warp.

#ifndef SKY_REFINE_BALANCE
#define SKY_REFINE_BALANCE 0
#endif
constexpr bool kBalance = SKY_REFINE_BALANCE == 1;
// listed p's tested per step of the list probe (2, 4 or 8; entries past the
// list's end hold stale codes and their bits are dropped)
#ifndef SKY_REFINE_PROBE_UNROLL
#define SKY_REFINE_PROBE_UNROLL 4
#endif
#ifndef SKY_REFINE_SLIM_PRODUCER
#define SKY_REFINE_SLIM_PRODUCER 0
#endif
// Layer-1 cell index (see cellwin_next): the producer of the single-set
// kernel takes its windows from the index from padded dimension
// SKY_REFINE_INDEX_RING_MIN_DP up, and the sparse mode from
// SKY_REFINE_INDEX_SPARSE_MIN_DP up, whenever the index pays (index_pays);
// otherwise both scan consecutive windows. Measured on B300 (ms, seed 1):
// the ring index took 10^7 x 16 anti-correlated 124.6 -> 112.4, 10^7 x 12
// independent 46.1 -> 44.5, 2*10^6 x 12 anti-correlated 9.12 -> 8.32,
// 10^6 x 8 anti-correlated / independent 1.224 / 0.734 -> 1.21 / 0.72; the
// sparse-mode index then 112.4 -> 107.5 and 44.5 -> 41.3, but at d = 8 it
// cost 6 % (the five warps each walk every window of the index to deal them
// out, and at 256 cells the windows are nearly as many as without it).
#ifndef SKY_REFINE_INDEX_RING_MIN_DP
#define SKY_REFINE_INDEX_RING_MIN_DP 8
#endif
#ifndef SKY_REFINE_INDEX_SPARSE_MIN_DP
#define SKY_REFINE_INDEX_SPARSE_MIN_DP 12
#endif
constexpr bool kListProbe = SKY_REFINE_LIST != 0;
constexpr uint32_t kEndTile = 0xffffffffu;

// ---- layer-1 cell index -------------------------------------------------
// A point's layer-1 cell (Eq. 1 at layer 1: two columns per dimension) is
// read off its 7-bit codes: bit k is set iff code k >= 64. If q dominates p
// (Definition 1), every code of q is <= p's (monotone map), so every column
// of q's layer-1 cell is <= p's (the cells are equal or one dominates or
// partially dominates the other, Definition 3): q's cell is a subset of p's.
// The cells that can hold a dominator of any live p of a tile are therefore
// the subsets of U, the union of the live p's cells. The index holds, per
// cell, the first and last q-tile holding one of its points (stored as
// ~first and last + 1 with atomicMax, so that a zeroed array means "no
// point"); the tiles are in Morton order, whose d top bits are the same
// layer-1 columns (the Morton and code grids are one monotone map at 2^b and
// 128 columns), so a cell's points are contiguous and its range is tight.
// The subsets of U are taken in ascending order, 32 at a time (one lane
// each), and their tile ranges are packed into windows of up to 32
// consecutive tiles: the tiles to examine, in ascending order, without
// visiting the tiles of any other cell. The box tests against the live
// groups' maxima still decide which of those tiles are streamed.

// The four layer-1 bits (bit 6 of each byte) of one word of 7-bit codes.
__device__ __forceinline__ uint32_t cell_bits4(uint32_t x)
{
    return ((((x >> 6) & 0x01010101u) * 0x01020408u) >> 24) & 0xfu;
}

template <int DW>
__device__ __forceinline__ uint32_t cell_of_codes(const uint32_t* c)
{
    uint32_t cell = 0;
#pragma unroll
    for (int w = 0; w < DW; ++w) cell |= cell_bits4(c[w]) << (4 * w);
    return cell;
}

// The j-th subset of U in ascending order: the bits of j deposited into the
// positions of U's set bits.
__device__ __forceinline__ uint32_t subset_of(uint32_t j, uint32_t U)
{
    uint32_t s = 0;
    for (uint32_t u = U; u != 0u && j != 0u; u &= u - 1u, j >>= 1)
        if (j & 1u) s |= u & (0u - u);
    return s;
}

// Windows (first tile, mask of tiles) over the tile ranges of the subsets of
// U, clipped to [first, last], produced one per call of next() by one warp.
// The state lives in shared memory (CellWinState, one per walking warp), so
// that it holds no registers between calls. A is the alignment of a window's
// first tile (its sub-tile minima are fetched by one 16-byte aligned bulk
// copy). If the ranges were not ascending (they are when the tile order
// groups the cells), a tile may fall into two windows: examined twice, never
// missed.
struct CellWinState {
    uint32_t U, nsub, batch, first, last;
    uint32_t pend;       // lanes of the batch whose range is not placed yet
    uint32_t clo, chi;   // the range being placed, while `have`
    uint32_t cursor;     // one past the last tile of the ranges placed so far (0: none)
    uint32_t have;
    uint32_t lo[32], hi[32];   // the current batch's ranges (lo > hi: none)
};

__device__ __forceinline__ void cellwin_init(CellWinState& st, uint32_t u, uint32_t f, uint32_t l)
{
    if ((threadIdx.x & 31) == 0) {
        st.U = u; st.nsub = 1u << __popc(u); st.batch = 0u; st.first = f; st.last = l;
        st.pend = 0u; st.clo = st.chi = 0u; st.cursor = 0u; st.have = 0u;
    }
    __syncwarp();
}

template <uint32_t A>
__device__ __forceinline__ bool cellwin_next(CellWinState& st, const uint32_t* __restrict__ mlo,
                                             const uint32_t* __restrict__ mhi, uint32_t& t0, uint32_t& wm)
{
    const int lane = threadIdx.x & 31;
    uint32_t pend = st.pend, clo = st.clo, chi = st.chi, cursor = st.cursor, batch = st.batch;
    bool have = st.have != 0u;
    wm = 0u;
    t0 = 0u;
    while (true) {
        if (!have) {
            if (pend == 0u) {
                if (batch * 32u >= st.nsub) break;
                const uint32_t j = batch * 32u + (uint32_t)lane;
                uint32_t lo = 1u, hi = 0u;
                if (j < st.nsub) {
                    const uint32_t s = subset_of(j, st.U);
                    const uint32_t a = __ldg(mlo + s), b = __ldg(mhi + s);
                    if (a != 0u && b != 0u) {
                        lo = max(~a, st.first);
                        hi = min(b - 1u, st.last);
                    }
                }
                pend = __ballot_sync(kFull, lo <= hi);
                st.lo[lane] = lo;
                st.hi[lane] = hi;
                __syncwarp();
                ++batch;
                continue;
            }
            const int b = __ffs(pend) - 1;
            pend &= pend - 1u;
            clo = st.lo[b];
            chi = st.hi[b];
            if (cursor != 0u && clo + 1u == cursor) clo = cursor;   // the previous range's last tile
            if (clo > chi) continue;
            have = true;
        }
        if (wm == 0u) t0 = clo & ~(A - 1u);
        else if (clo < t0 || clo > t0 + 31u) break;   // the range opens the next window
        const uint32_t end = min(chi, t0 + 31u);
        wm |= (0xffffffffu >> (31u - (end - t0))) & (0xffffffffu << (clo - t0));
        if (end == chi) {
            have = false;
            cursor = max(cursor, chi + 1u);
        } else {
            clo = t0 + 32u;   // the rest of the range opens the next window
            break;
        }
    }
    __syncwarp();   // every lane has read st.lo / st.hi
    if (lane == 0) {
        st.pend = pend; st.clo = clo; st.chi = chi; st.cursor = cursor; st.batch = batch;
        st.have = have ? 1u : 0u;
    }
    __syncwarp();
    return wm != 0u;
}

// Use the index when its subset batches are fewer than half the windows of
// 32 consecutive tiles that a scan of [first, last] would examine.
__device__ __forceinline__ bool index_pays(uint32_t U, uint32_t first, uint32_t last)
{
    return last >= first && (1ull << __popc(U)) <= 16ull * ((uint64_t)(last - first) / 32u + 1u);
}

// Mask probe (single-set kernel, padded dimensions 12 and 16): besides its
// 7-bit codes, every streamed q-tile carries threshold masks of its 32-point
// sub-tiles -- for each dimension k and level l of the 3-bit codes (the top
// three bits of the 7-bit codes), the 32-bit set of the sub-tile's q's whose
// 3-bit code in k is <= l (written by the gather). A group scan that lists
// at least SKY_REFINE_MASK_MIN_LIST p's gives every lane one p and ANDs the
// d masks at that p's levels: the q's of the sub-tile that pass the 3-bit
// test against it (necessary for dominance: the code map is monotone), 32
// pairs per lane in about 2.5 instructions per dimension, where the list
// probe spends about 10 warp instructions per listed p plus the list's
// construction. The rare passes get the 7-bit and exact tests of the list
// probe. Measured on B300 (ms, one sky_skyline call, seed 1; list probe ->
// mask probe from 3 / 2 / 1 listed p's): 10^7 x 16 anti-correlated 108.9 ->
// 92.9 / 91.2 / 83.7, 2*10^6 x 16 independent 14.2 -> 15.5 / 14.2 / 12.6,
// correlated 10.6 -> 10.1 / 10.4 / 11.0; at padded dimension 12 (from 1
// listed p) 10^7 x 12 independent 20.7 -> 17.3, 2*10^6 x 12 anti-correlated
// 8.19 -> 5.42, correlated (a one-point skyline) 1.09 -> 1.56. A per-stage
// flag that left the masks out once few p's were live measured 13 % slower
// on every set.
#ifndef SKY_REFINE_MASK_MIN_LIST
#define SKY_REFINE_MASK_MIN_LIST 1
#endif
// ring depth with the mask probe (its stages hold codes and masks: 4 KB a
// tile at d = 16, 3.5 KB at d = 12; 8 stages with four CTAs per SM measured
// 10^7 x 16 anti-correlated 83.6 -> 97.3 ms)
#ifndef SKY_REFINE_MASK_STAGES
#define SKY_REFINE_MASK_STAGES 6
#endif

// 1: a CTA whose p-tile holds 256 points (PG = 8 groups, see RefineSmem)
// stages its own p coordinates in shared memory as well; 0: its exact tests
// read them from global memory, which keeps the CTA at the shared memory of
// the 128-point form
#ifndef SKY_REFINE_PX_SMEM_WIDE
#define SKY_REFINE_PX_SMEM_WIDE 0
#endif

// Shared memory of one refinement CTA. S: ring stages; FAST: fast-code
// list probe (see SKY_REFINE_FAST_MIN_DP for the single-set default); PG:
// groups of 32 p's in the CTA's p-tile -- 4 (one 128-point tile, the q-tile
// size) or 8 (two consecutive tiles: every streamed q-tile and every stage
// hand-off then serves twice the p's); MASK: the mask probe -- 0 off, 1 the
// q-tiles' threshold masks streamed with their codes, 2 the masks only (with
// the mask probe taking every scan, SKY_REFINE_MASK_MIN_LIST <= 1, the
// staged codes serve only the rare 3-bit passes, which then read their q's
// 7-bit codes from global memory).
template <int DP, int S = kRingStages, bool FAST = (DP >= SKY_REFINE_FAST_MIN_DP), int PG = kTQ / 32,
          int MASK = 0>
struct RefineSmem {
    static_assert(PG == kTQ / 32 || PG == 2 * (kTQ / 32), "one or two tiles of p's");
    static_assert(MASK == 0 || DP >= 8, "the mask probe is built for padded dimensions 8 to 16");
    static_assert(MASK != 2 || SKY_REFINE_MASK_MIN_LIST <= 1, "masks only: the list probe never runs");
    static constexpr int DW = DP / 4;
    static constexpr int kStages = S;
    static constexpr bool kFast = FAST;
    static constexpr bool kMask = MASK != 0;
    static constexpr bool kMaskOnly = MASK == 2;
    static constexpr int kGroups = PG;               // groups of 32 p's
    static constexpr int kTP = PG * 32;              // p's of the CTA
    static constexpr int kTiles = kTP / kTQ;         // 128-point tiles of p's
    static constexpr bool kPxSmem = SKY_REFINE_PX_SMEM && (kTiles == 1 || SKY_REFINE_PX_SMEM_WIDE) && MASK == 0;
    static constexpr int FW = (DP + 7) / 8;        // fast-code words
    // list entry words (vector loads): fast codes, or the 7-bit codes
    static constexpr int DWL = kFast ? FW : (DW == 3 ? 4 : DW);
    // bulk-copy destinations: 16-byte aligned whatever the ring depth
    alignas(16) uint32_t qC[kMaskOnly ? 1 : S][kMaskOnly ? 4 : kTQ * DW];  // streamed q-tiles (codes)
    // streamed q-tiles' threshold masks: sub-tile q, dimension k, level l at
    // word q * 128 + k * 8 + l; each sub-tile's table 256-byte aligned (its
    // addresses are formed by replacing the low byte, see the mask probe)
    alignas(kMask ? 256 : 4) uint32_t qT[kMask ? S : 1][kMask ? kMaskWords : 1];
    // own p's byte offsets into a sub-tile table half: byte k % 4 of word
    // k / 4 = (k % 8) * 32 + 4 * (3-bit code of dimension k)
    alignas(16) uint32_t pO[kMask ? kTP : 1][4];
    static constexpr int kWindows = SKY_REFINE_WINDOWS;
    alignas(16) float pX[kPxSmem ? kTP * DP : 4];   // own p coordinates (exact tests)
    uint32_t pP[kTP * DW];               // own p codes | 0x80 per byte
    uint32_t pF[kFast ? kTP * FW : 1];   // own p fast codes | 0x8 per nibble
    uint32_t livemask[PG];               // bit l of word g: p g*32+l is still undominated
    uint32_t validmask[PG];              // the p's of the tile (split scans: the kills are merged)
    uint32_t gmax[PG][DW];               // byte-wise max code of each group's live p's | 0x80 per byte (producer)
    uint32_t glive[PG];                  // live p's per group (producer)
    uint32_t stage_tile[S];
    uint32_t stage_mask[S];              // bit PG*w+g: sub-tile w may dominate a live p of group g
    uint32_t stage_sub[S][kTQ / 32][DW];   // sub-tile minimum codes of the staged tile
    uint64_t full[S];
    uint64_t empty[S];
    alignas(16) uint32_t stc[kWindows][32 * kSubSlots * DW];   // producer: codes of the 32 tiles of a super-tile
    uint64_t cbar[kWindows];                 // producer: their bulk copies
    int32_t pend[kWindows];                  // producer: the first tile of the window held by each buffer
    uint32_t wmask[kWindows];                // producer: the window's tiles to examine (bit i: first tile + i)
    CellWinState cwin[kTQ / 32 + 1];         // layer-1 cell index walk of each warp (producer: the last)
    // consumer warp w: codes of the listed p's (in sparse mode, the whole
    // array holds one list of up to 32 entries of 7-bit codes)
    alignas(16) uint32_t plist[kTQ / 32][32 * (DWL > 1 ? DWL : 2)];
    static_assert((kTQ / 32) * 32 * (DWL > 1 ? DWL : 2) >= 32 * (DW == 3 ? 4 : DW), "sparse list fits");
    uint8_t pidx[kTQ / 32][32];                        // and their indices in the tile
    uint32_t live;                       // live p's of the CTA
    uint32_t sparse;                     // 1: the scan continues in sparse mode
    uint32_t resume;                     // first q-tile of the sparse scan
    uint32_t scan_end;                   // last q-tile to scan
    uint32_t nlist;                      // live p's listed for the sparse scan
    uint32_t failed;
    uint32_t lastpart;                   // split scans: this CTA finished the p-tile's last part
};

// Listed p entry j of a warp's list, DW words into c (16- or 8-byte loads).
template <int DW>
__device__ __forceinline__ void load_entry(const uint32_t* e, uint32_t (&c)[DW])
{
    if constexpr (DW == 4 || DW == 3) {
        const uint4 v = *reinterpret_cast<const uint4*>(e);
        c[0] = v.x; c[1] = v.y; c[2] = v.z;
        if constexpr (DW == 4) c[3] = v.w;
    } else if constexpr (DW == 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(e);
        c[0] = v.x; c[1] = v.y;
    } else {
        c[0] = e[0];
    }
}

// Fast code word f of a point from its 7-bit code words: nibble b of the
// low half-byte holds code(8f + b) >> 4, nibble b of the high half-byte
// code(8f + 4 + b) >> 4 (three bits each, bit 3 clear).
template <int DW>
__device__ __forceinline__ uint32_t fast_word(const uint32_t (&c)[DW], int f)
{
    const uint32_t lo = (c[2 * f] >> 4) & 0x07070707u;
    const uint32_t hi = (2 * f + 1 < DW) ? ((c[2 * f + 1] >> 4) & 0x07070707u) : 0u;
    return lo | (hi << 4);
}
constexpr uint32_t kHighNib = 0x88888888u;

__device__ __forceinline__ uint32_t has_zero_byte(uint32_t x)
{
    return (x - 0x01010101u) & ~x & 0x80808080u;
}

// every byte of lo <= the matching byte of hi (7-bit codes; hi with its
// guard bits 0x80 already set)
template <int DW>
__device__ __forceinline__ bool bytes_le(const uint32_t* lo, const uint32_t* hi)
{
    uint32_t r = kHigh;
#pragma unroll
    for (int w = 0; w < DW; ++w) r &= hi[w] - lo[w];
    return r == kHigh;
}

// Refines p-tile `ptile` (< ceil(m / SM::kTP)) of one point set: the
// SM::kTP = 128 or 256 survivors from ptile * SM::kTP on (one or two
// consecutive 128-point tiles). Called by all kTQ + 32 threads of the CTA
// with the CTA's shared memory; leaves the shared memory free for the next
// call (barriers invalidated).
// TEND (optional): per p-tile, the last q-tile that can hold a dominator of
// one of its points (the tiles are in Morton order, and a dominator's Morton
// key is never above its victim's: the column maps are monotone), so the
// scan stops there; NULL scans every tile. SUPMIN (optional): byte-wise
// minimum code of each run of 32 q-tiles ("super-tile"); a super-tile whose
// minimum exceeds every live group's maximum in some byte is skipped whole;
// NULL examines every super-tile.
// SPARSE (the single-set kernel): a p-tile whose live points drop to
// SparseLive<DP> finishes in sparse mode, and the producer tests relevance
// against register copies of the group maxima. The batched persistent kernel
// keeps the ring to the end and the maxima in shared memory (fewer registers:
// measured faster there).
// WIT (witness mode, a checking aid): every removal of a p by a q also writes
// wit[row of p] = row of q, a point that dominates p (Definition 1).
template <int DP, bool SPARSE = true, bool WIT = false, class SM = RefineSmem<DP>>
__device__ __forceinline__ void refine_ptile(SM& sm, const float* __restrict__ X,
                                             const uint32_t* __restrict__ C, const int32_t* __restrict__ ids,
                                             const uint32_t* __restrict__ SUB, const uint32_t* __restrict__ TEND,
                                             const uint32_t* __restrict__ SUPMIN, uint32_t m, uint32_t ptile,
                                             DevResult* res, uint8_t* keep, int32_t* wit = nullptr,
                                             const uint32_t* __restrict__ MLO = nullptr,
                                             const uint32_t* __restrict__ MHI = nullptr,
                                             const uint32_t* __restrict__ TM = nullptr, uint32_t part = 0,
                                             uint32_t nparts = 1, uint32_t* split = nullptr)
{
    constexpr int DW = DP / 4;
    constexpr int NG = SM::kGroups;   // groups of 32 p's
    constexpr int NQ = kTQ / 32;      // q sub-tiles of a streamed tile = consumer warps
    constexpr int NT = SM::kTiles;    // 128-point tiles of p's
    constexpr int kTP = SM::kTP;
    constexpr int S = SM::kStages;
    constexpr uint32_t kSparseLive = SparseLive<DP>::value;
    constexpr uint32_t kBytesC = SM::kMaskOnly ? 0u : kTQ * DW * sizeof(uint32_t);   // the tile's codes
    constexpr uint32_t kBytesT = SM::kMask ? kMaskWords * sizeof(uint32_t) : 0u;   // the tile's threshold masks
    const uint32_t T = (m + kTQ - 1) / kTQ;
    uint32_t* err = &res->err;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t pbase = (int64_t)ptile * kTP;
    const uint32_t tile0 = ptile * (uint32_t)NT;   // the first of the p-tile's own q-tiles
    // q-tile t is one of the p-tile's own (streamed first, skipped later)
    auto own = [&](uint32_t t) -> bool { return t - tile0 < (uint32_t)NT; };
    if (tid < kTQ) {
#pragma unroll
        for (int h = 0; h < NT; ++h) {
            const int pi = h * kTQ + tid;
            // the survivor layout ends with tile T - 1; a second tile past it holds no p
            const bool in_layout = tile0 + (uint32_t)h < T;
            const bool valid = pbase + pi < m;
            uint32_t pc[DW];
#pragma unroll
            for (int w = 0; w < DW; ++w) {
                pc[w] = in_layout ? C[(pbase + pi) * DW + w] : 0x7f7f7f7fu;
                sm.pP[pi * DW + w] = pc[w] | kHigh;
            }
            if constexpr (SM::kFast) {
#pragma unroll
                for (int f = 0; f < SM::FW; ++f) sm.pF[pi * SM::FW + f] = fast_word<DW>(pc, f) | kHighNib;
            }
            if constexpr (SM::kMask) {
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    uint32_t o = 0;
                    if (w < DW) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t l = (pc[w < DW ? w : 0] >> (8 * j + 4)) & 7u;
                            o |= ((uint32_t)(((4 * w + j) % 8) * 32) + 4u * l) << (8 * j);
                        }
                    }
                    sm.pO[pi][w] = o;
                }
            }
            if constexpr (SM::kPxSmem) {
#pragma unroll
                for (int k = 0; k < DP; k += 4)
                    *reinterpret_cast<float4*>(&sm.pX[pi * DP + k]) =
                        in_layout ? *reinterpret_cast<const float4*>(X + (pbase + pi) * DP + k)
                                  : make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
            }
            const uint32_t vm = __ballot_sync(kFull, valid);
            if ((tid & 31) == 0) {
                sm.livemask[pi >> 5] = vm;
                sm.validmask[pi >> 5] = vm;
            }
        }
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], NQ);
        }
        for (int b = 0; b < SM::kWindows; ++b) mbar_init(&sm.cbar[b], 1);
        mbar_fence_init();
        sm.live = (m - pbase) < (uint32_t)kTP ? (m - (uint32_t)pbase) : (uint32_t)kTP;
        sm.failed = 0;
        sm.sparse = 0;
        if constexpr (SM::kMask) {
            // the mask probe forms table addresses by replacing their low byte
            if (smem_addr(&sm.qT[0][0]) & 255u) {
                atomicOr(err, SKY_DEV_ERR_LAYOUT);
                sm.failed = 1u;
                sm.live = 0u;
            }
        }
    }
    __syncthreads();

    if (warp == NQ) {
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
                    if (lane == 0) sm.gmax[g][w] = c | kHigh;   // guard bits set for the box tests
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
        // last q-tile to scan (the last own tile's end: the ends are non-decreasing)
        const uint32_t E = TEND ? min(TEND[min(tile0 + (uint32_t)NT - 1u, T - 1u)], T - 1u) : T - 1u;
        if (lane == 0) sm.scan_end = E;
        const uint32_t SL = E / 32u;                                     // last super-tile
        // Streaming order: the p-tile itself first (its own points kill each
        // other early in anti-correlated sets), then the super-tiles in
        // ascending Morton order (tiles near the origin, whose points
        // dominate most, early). Relevant super-tiles are found 32 at a time
        // (lane = super-tile).
        uint32_t win = 0, smask = 0;
        auto next_super = [&]() -> int {
            while (true) {
                if (smask) {
                    const int b = __ffs(smask) - 1;
                    smask &= smask - 1;
                    return (int)(win - 32u) + b;
                }
                if (win > SL) return -1;
                const uint32_t sx = win + lane;
                bool rel = sx <= SL;
                // (a split scan's parts deal windows by their position in
                // this sequence, so for them it must not depend on which p's
                // are live: no super-tile test; the per-tile test still runs)
                if (rel && SUPMIN && nparts == 1u) {
                    uint32_t mn[DW];
#pragma unroll
                    for (int w = 0; w < DW; ++w) mn[w] = __ldg(SUPMIN + (int64_t)sx * DW + w);
                    rel = false;
#pragma unroll
                    for (int g = 0; g < NG; ++g) rel |= (sm.glive[g] != 0u) && bytes_le<DW>(mn, sm.gmax[g]);
                }
                smask = __ballot_sync(kFull, rel);
                win += 32u;
            }
        };
        // With the layer-1 cell index, the windows cover only the tiles of
        // the cells that can hold a dominator of a live p (cellwin_next);
        // otherwise they are the relevant super-tiles.
        constexpr uint32_t kWinAlign = DW == 4 ? 1u : DW == 2 ? 2u : 4u;   // 16-byte aligned copies
        bool use_idx = false;
        if (MLO != nullptr && DP >= SKY_REFINE_INDEX_RING_MIN_DP) {
            uint32_t U = 0;
#pragma unroll
            for (int g = 0; g < NG; ++g)
                if (sm.glive[g] != 0u) U |= cell_of_codes<DW>(sm.gmax[g]);
            use_idx = index_pays(U, 0u, E);
            if (use_idx) cellwin_init(sm.cwin[NQ], U, 0u, E);
        }
        auto next_window = [&](uint32_t& t0, uint32_t& wm) -> bool {
            if (use_idx) return cellwin_next<kWinAlign>(sm.cwin[NQ], MLO, MHI, t0, wm);
            const int sx = next_super();
            if (sx < 0) return false;
            t0 = (uint32_t)sx * 32u;
            wm = 0xffffffffu;
            return true;
        };
        // the p-tile's own q-tiles: every (sub-tile, group) pair whose
        // sub-tile minimum is within the group's reach (lane q * NG + g);
        // slot `issued` (< NT <= S) of the ring, not yet used
        static_assert(NQ * NG <= 32 && NT <= S, "one lane per (sub-tile, group) pair");
#pragma unroll
        for (int h = 0; h < NT; ++h) {
            const uint32_t ot = tile0 + (uint32_t)h;
            if (ot >= T || part != 0u) break;   // a split scan's first part streams them
            const int q = lane / NG, g = lane % NG;
            const int s = (int)issued;
            bool rel = false;
            if (lane < NQ * NG && sm.glive[g] != 0u) {
                uint32_t mn[DW];
#pragma unroll
                for (int w = 0; w < DW; ++w) mn[w] = __ldg(SUB + ((int64_t)ot * kSubSlots + q) * DW + w);
                rel = bytes_le<DW>(mn, sm.gmax[g]);
            }
            if (lane < NQ * DW) sm.stage_sub[s][lane / DW][lane % DW] = __ldg(SUB + (int64_t)ot * kSubSlots * DW + lane);
            const uint32_t bmask = __ballot_sync(kFull, rel);
            __syncwarp();   // the lanes' writes before lane 0's arrive on the slot
            if (lane == 0 && bmask) {
                sm.stage_tile[s] = ot;
                sm.stage_mask[s] = bmask;
                mbar_arrive_expect_tx(&sm.full[s], kBytesC + kBytesT);
                if constexpr (!SM::kMaskOnly) bulk_g2s(sm.qC[s], C + (int64_t)ot * kTQ * DW, kBytesC, &sm.full[s]);
                if constexpr (SM::kMask) bulk_g2s(sm.qT[s], TM + (int64_t)ot * kMaskWords, kBytesT, &sm.full[s]);
            }
            __syncwarp();
            if (bmask) { ++issued; ++since; }
        }
        // the sub-tile minima of the tiles of a window: one bulk copy (the
        // arrays carry 16 bytes of slack past their end); copy k goes to
        // buffer k % NB and is that buffer's (k / NB)-th use; up to NB
        // windows are in flight ahead of the one being examined
        constexpr uint32_t NB = (uint32_t)SM::kWindows;
        uint32_t kiss = 0, kcons = 0;   // copies issued / consumed
        auto fetch_window = [&](uint32_t t0, uint32_t wm) {
            const uint32_t nt = min(32u - (uint32_t)__clz(wm), T - t0);
            const uint32_t bytes = (nt * kSubSlots * DW * 4u + 15u) & ~15u;
            const int bb = (int)(kiss % NB);
            __syncwarp();
            if (lane == 0) {
                sm.pend[bb] = (int32_t)t0;
                sm.wmask[bb] = wm;
                fence_proxy_async_smem();   // generic reads of this buffer are done
                mbar_arrive_expect_tx(&sm.cbar[bb], bytes);
                bulk_g2s(sm.stc[bb], SUB + (int64_t)t0 * kSubSlots * DW, bytes, &sm.cbar[bb]);
            }
            __syncwarp();
            ++kiss;
        };
        // a split scan's part takes every nparts-th window from its part on
        uint32_t wseq = 0;
        auto refill = [&]() {
            while (kiss - kcons < NB) {
                uint32_t t0, wm;
                if (!next_window(t0, wm)) break;
                const bool mine = nparts == 1u || wseq % nparts == part;
                ++wseq;
                if (mine) fetch_window(t0, wm);
            }
        };
        refill();
        while (kcons < kiss && !stop) {
            if (all_dead()) break;
            const int bf = (int)(kcons % NB);
            const uint32_t t0 = (uint32_t)sm.pend[bf];
            const uint32_t wmk = sm.wmask[bf];
            if (SPARSE && kSparseLive > 0 && nparts == 1u && __shfl_sync(kFull, sm.live, 0) <= kSparseLive) {
                // few p's left: the rest of the scan runs in sparse mode,
                // from this (fetched, not yet examined) window on
                if (lane == 0) {
                    sm.sparse = 1u;
                    sm.resume = t0;
                }
                break;
            }
            bool ok = true;
            if (lane == 0) ok = mbar_wait(&sm.cbar[bf], (kcons / NB) & 1u, err);
            if (!__shfl_sync(kFull, ok ? 1 : 0, 0)) { if (lane == 0) sm.failed = 1u; stop = true; break; }
            __syncwarp();   // lane 0 observed the copy; the warp barrier orders the others' reads after it
            if (since >= kSummaryEvery) { summarise(); since = 0; }
            const uint32_t t = t0 + lane;
            const uint32_t* tc = &sm.stc[bf][lane * kSubSlots * DW];
            // relevance of each (sub-tile, group) pair of this q-tile; in the
            // single-set kernel with four groups the group maxima and the live
            // groups are read into registers once for the 4 + 16 box tests of
            // a lane; with eight groups, one group's maximum at a time
            constexpr bool kRegMax = SPARSE && DP <= SKY_REFINE_REGMAX_DP && NG == NQ;
            uint32_t gm[kRegMax ? NG : 1][DW];
            uint32_t gl = 0;
            if constexpr (kRegMax) {
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    if (sm.glive[g] != 0u) gl |= 1u << g;
#pragma unroll
                    for (int w = 0; w < DW; ++w) gm[g][w] = sm.gmax[g][w];
                }
            }
            auto le_g = [&](const uint32_t* lo, int g) -> bool {
                if constexpr (kRegMax) return ((gl >> g) & 1u) && bytes_le<DW>(lo, gm[g]);
                else return (sm.glive[g] != 0u) && bytes_le<DW>(lo, sm.gmax[g]);
            };
            uint32_t rmask = 0;
            if (t <= E && !own(t) && ((wmk >> lane) & 1u)) {   // the own tiles went first
#if SKY_REFINE_SLIM_PRODUCER
                // one sub-tile's minimum in registers at a time
                uint32_t cw[DW];
#pragma unroll
                for (int w = 0; w < DW; ++w) cw[w] = tc[NQ * DW + w];   // the tile minimum
                bool any = false;
#pragma unroll
                for (int g = 0; g < NG; ++g) any |= le_g(cw, g);
                if (any) {
#pragma unroll 1
                    for (int q = 0; q < NQ; ++q) {
#pragma unroll
                        for (int w = 0; w < DW; ++w) cw[w] = tc[q * DW + w];
#pragma unroll
                        for (int g = 0; g < NG; ++g)
                            if (le_g(cw, g)) rmask |= 1u << (q * NG + g);
                    }
                }
#else
                uint32_t cw[NQ + 1][DW];   // sub-tile minima, then the tile minimum
#pragma unroll
                for (int q = 0; q <= NQ; ++q)
#pragma unroll
                    for (int w = 0; w < DW; ++w) cw[q][w] = tc[q * DW + w];
                if constexpr (NG == NQ) {
                    bool any = false;
#pragma unroll
                    for (int g = 0; g < NG; ++g) any |= le_g(cw[NQ], g);
                    if (any) {
#pragma unroll
                        for (int q = 0; q < NQ; ++q)
#pragma unroll
                            for (int g = 0; g < NG; ++g)
                                if (le_g(cw[q], g)) rmask |= 1u << (q * NG + g);
                    }
                } else {
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        if (sm.glive[g] == 0u) continue;
                        uint32_t gg[DW];
#pragma unroll
                        for (int w = 0; w < DW; ++w) gg[w] = sm.gmax[g][w];
                        if (!bytes_le<DW>(cw[NQ], gg)) continue;   // the tile minimum first
#pragma unroll
                        for (int q = 0; q < NQ; ++q)
                            if (bytes_le<DW>(cw[q], gg)) rmask |= 1u << (q * NG + g);
                    }
                }
#endif
            }
            uint32_t mask = __ballot_sync(kFull, rmask != 0u);
            while (mask) {
                const int b = __ffs(mask) - 1;
                mask &= mask - 1;
                const uint32_t bmask = __shfl_sync(kFull, rmask, b);
                int s;
                if (!claim(s)) { if (lane == 0) sm.failed = 1u; stop = true; break; }
                // tile b's sub-tile minima to the slot; the warp barrier orders
                // these writes before lane 0's arrive on the slot
                if (lane < NQ * DW) sm.stage_sub[s][lane / DW][lane % DW] = sm.stc[bf][b * kSubSlots * DW + lane];
                __syncwarp();
                if (lane == 0) {
                    const uint32_t tt = t0 + b;
                    sm.stage_tile[s] = tt;
                    sm.stage_mask[s] = bmask;
                    mbar_arrive_expect_tx(&sm.full[s], kBytesC + kBytesT);
                    if constexpr (!SM::kMaskOnly)
                        bulk_g2s(sm.qC[s], C + (int64_t)tt * kTQ * DW, kBytesC, &sm.full[s]);
                    if constexpr (SM::kMask)
                        bulk_g2s(sm.qT[s], TM + (int64_t)tt * kMaskWords, kBytesT, &sm.full[s]);
                }
                __syncwarp();
                ++issued;
                ++since;
                // every fourth tile: has every p died (a few stages issued
                // after the last death cost the consumers one check each),
                // or are few enough left for sparse mode, from the next tile?
                if ((issued & 3u) == 0u) {
                    if (all_dead()) { stop = true; break; }
                    if (SPARSE && kSparseLive > 0 && nparts == 1u && __shfl_sync(kFull, sm.live, 0) <= kSparseLive) {
                        if (lane == 0) {
                            sm.sparse = 1u;
                            sm.resume = t0 + (uint32_t)b + 1u;
                        }
                        stop = true;
                        break;
                    }
                }
            }
            if (stop) break;
            ++kcons;    // buffer bf is free again
            refill();
        }
        // code copies that were not consumed land before the exit
        if (lane == 0)
            for (uint32_t k = kcons; k < kiss; ++k) mbar_wait(&sm.cbar[k % NB], (k / NB) & 1u, nullptr);
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
        int qi = warp * 32 + lane;   // this lane's q of the sub-tile being tested
        uint32_t listed = 0, gscans = 0;   // per warp (32-bit: a CTA lists far fewer than 2^32)
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
            const uint32_t smask = sm.stage_mask[s];
            const bool any_live = __shfl_sync(kFull, sm.live != 0u ? 1 : 0, 0) != 0;
            if (any_live && smask) {
                constexpr bool kFast = SM::kFast;
                constexpr int FW = SM::FW;
                uint32_t Mw[DW], Q[DW], QF[FW];
                // the codes of sub-tile q of the stage: this lane takes q's point lane
                auto load_sub = [&](int q) {
                    qi = q * 32 + lane;
#pragma unroll
                    for (int w = 0; w < DW; ++w) Mw[w] = sm.stage_sub[s][q][w];
                    if constexpr (!SM::kMaskOnly) {
#pragma unroll
                        for (int w = 0; w < DW; ++w) Q[w] = sm.qC[s][qi * DW + w];
                        if constexpr (kFast) {
#pragma unroll
                            for (int f = 0; f < FW; ++f) QF[f] = fast_word<DW>(Q, f);
                        }
                    }
                };
                // sub-tile (loaded) against the live p's of group g
                auto test_group = [&](int g) {
                    ++gscans;
                    const int pg = g * 32 + lane;
                    uint32_t r = kHigh;
#pragma unroll
                    for (int w = 0; w < DW; ++w) r &= sm.pP[pg * DW + w] - Mw[w];
                    uint32_t mask = __ballot_sync(kFull, r == kHigh) & sm.livemask[g];
                    listed += __popc(mask);

                    // q (this lane) against listed p pi
                    auto probe = [&](int pi) {
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
                                const float* qx = X + ((int64_t)tt * kTQ + qi) * DP;
                                const float* px = SM::kPxSmem ? &sm.pX[pi * DP] : X + (pbase + pi) * DP;
                                bool le = true, lt = false;
#pragma unroll
                                for (int kk = 0; kk < DP; kk += 4) {
                                    const float4 u = __ldg(reinterpret_cast<const float4*>(qx + kk));
                                    const float4 v = *reinterpret_cast<const float4*>(px + kk);
                                    le &= (u.x <= v.x) & (u.y <= v.y) & (u.z <= v.z) & (u.w <= v.w);
                                    lt |= (u.x < v.x) | (u.y < v.y) | (u.z < v.z) | (u.w < v.w);
                                }
                                dom = le && lt;
                            }
                            if (dom) {
                                const uint32_t bit = 1u << (pi & 31);
                                if (atomicAnd(&sm.livemask[pi >> 5], ~bit) & bit) atomicSub(&sm.live, 1u);
                                if constexpr (WIT) wit[ids[pbase + pi]] = ids[(int64_t)tt * kTQ + qi];
                            }
                        }
                    };
                    if constexpr (SM::kMask) {
                        if (__popc(mask) >= SKY_REFINE_MASK_MIN_LIST) {
                            // mask probe: this lane's p (pg, if listed) against
                            // the 32 q's of the sub-tile -- the AND of the
                            // sub-tile's masks at p's 3-bit levels is the set
                            // of q's whose 3-bit codes are <= p's everywhere
                            uint32_t mq = ((mask >> lane) & 1u) ? 0xffffffffu : 0u;
                            const uint4 po = *reinterpret_cast<const uint4*>(&sm.pO[pg][0]);
                            const uint32_t pw[4] = {po.x, po.y, po.z, po.w};
                            const uint32_t tb = smem_addr(&sm.qT[s][(qi >> 5) * 128]);   // 256-byte aligned
                            uint32_t v[DP];
#pragma unroll
                            for (int kd = 0; kd < DP; ++kd) {
                                // the table half's address with its low byte
                                // replaced by p's offset for dimension kd
                                const uint32_t a = __byte_perm(tb + (kd < 8 ? 0u : 256u), pw[kd >> 2],
                                                               0x3214u + (uint32_t)(kd & 3));
                                asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v[kd]) : "r"(a));
                            }
#pragma unroll
                            for (int kd = 0; kd < DP; ++kd) mq &= v[kd];
                            if (mq) {   // rare: the 7-bit and exact tests of each passing q
                                uint32_t pc[DW];
#pragma unroll
                                for (int w = 0; w < DW; ++w) pc[w] = sm.pP[pg * DW + w];
                                while (mq) {
                                    const int qj = (qi & ~31) + __ffs(mq) - 1;
                                    mq &= mq - 1u;
                                    uint32_t D[DW];
                                    uint32_t a = kHigh;
#pragma unroll
                                    for (int w = 0; w < DW; ++w) {
                                        const uint32_t qw = SM::kMaskOnly ? __ldg(C + ((int64_t)tt * kTQ + qj) * DW + w)
                                                                          : sm.qC[s][SM::kMaskOnly ? 0 : qj * DW + w];
                                        D[w] = pc[w] - qw;
                                        a &= D[w];
                                    }
                                    if (a != kHigh) continue;
                                    ++hits;
                                    uint32_t eq = 0;
#pragma unroll
                                    for (int w = 0; w < DW; ++w) eq |= has_zero_byte(D[w] ^ kHigh);
                                    bool dom = true;
                                    if (eq) {
                                        ++exact;
                                        const float* qx = X + ((int64_t)tt * kTQ + qj) * DP;
                                        const float* px = SM::kPxSmem ? &sm.pX[pg * DP] : X + (pbase + pg) * DP;
                                        bool le = true, lt = false;
#pragma unroll
                                        for (int kk = 0; kk < DP; kk += 4) {
                                            const float4 u = __ldg(reinterpret_cast<const float4*>(qx + kk));
                                            const float4 w4 = *reinterpret_cast<const float4*>(px + kk);
                                            le &= (u.x <= w4.x) & (u.y <= w4.y) & (u.z <= w4.z) & (u.w <= w4.w);
                                            lt |= (u.x < w4.x) | (u.y < w4.y) | (u.z < w4.z) | (u.w < w4.w);
                                        }
                                        dom = le && lt;
                                    }
                                    if (dom) {
                                        const uint32_t bit = 1u << lane;
                                        if (atomicAnd(&sm.livemask[g], ~bit) & bit) atomicSub(&sm.live, 1u);
                                        if constexpr (WIT) wit[ids[pbase + pg]] = ids[(int64_t)tt * kTQ + qj];
                                        break;
                                    }
                                }
                            }
                            return;
                        }
                    }
                    if constexpr (kListProbe && !SM::kMaskOnly) {
                        if (mask) {
                            // the listed p's of the group, in lane order, into
                            // this warp's list
                            constexpr int DWL = SM::DWL;
                            uint32_t* L = sm.plist[warp];
                            if ((mask >> lane) & 1u) {
                                const int rank = __popc(mask & ((1u << lane) - 1u));
                                if constexpr (kFast) {
#pragma unroll
                                    for (int f = 0; f < FW; ++f) L[rank * DWL + f] = sm.pF[pg * FW + f];
                                } else {
#pragma unroll
                                    for (int w = 0; w < DW; ++w) L[rank * DWL + w] = sm.pP[pg * DW + w];
                                }
                                sm.pidx[warp][rank] = (uint8_t)pg;
                            }
                            __syncwarp();
                            const int k = __popc(mask);
                            // q (this lane) against every listed p, four per
                            // step; entries past k hold stale codes and their
                            // bits are dropped below
                            uint32_t hb = 0;
                            constexpr int PU = SKY_REFINE_PROBE_UNROLL;
                            for (int j0 = 0; j0 < k; j0 += PU) {
                                if constexpr (kFast && kMinProbe) {
                                    // the block's entries first: H & ~(d0 & d1) is zero
                                    // exactly for an entry that passes, so the block
                                    // holds a pass iff the smallest such word is zero
                                    // (stale entries past k take part; a pass among
                                    // them only costs the exact pass below)
                                    uint32_t miss = 0xffffffffu;
#pragma unroll
                                    for (int u = 0; u < PU; ++u) {
                                        uint32_t c[FW];
                                        load_entry<FW>(L + (j0 + u) * DWL, c);
                                        uint32_t a = kHighNib;
#pragma unroll
                                        for (int f = 0; f < FW; ++f) a &= c[f] - QF[f];
                                        miss = min(miss, a ^ kHighNib);
                                    }
                                    if (miss != 0u) continue;
                                }
                                uint32_t nb = 0;   // hit bits of entries j0 .. j0 + PU - 1
#pragma unroll
                                for (int u = 0; u < PU; ++u) {
                                    if constexpr (kFast) {
                                        uint32_t c[FW];
                                        load_entry<FW>(L + (j0 + u) * DWL, c);
                                        uint32_t a = kHighNib;
#pragma unroll
                                        for (int f = 0; f < FW; ++f) a &= c[f] - QF[f];
                                        if (a == kHighNib) nb |= 1u << u;
                                    } else {
                                        uint32_t c[DW];
                                        load_entry<DW>(L + (j0 + u) * DWL, c);
                                        uint32_t a = kHigh;
#pragma unroll
                                        for (int w = 0; w < DW; ++w) a &= c[w] - Q[w];
                                        if (a == kHigh) nb |= 1u << u;
                                    }
                                }
                                hb |= nb << j0;
                            }
                            if (k < 32) hb &= (1u << k) - 1u;
                            // rare: code(q) <= code(p) in every dimension
                            while (hb) {
                                const int j = __ffs(hb) - 1;
                                hb &= hb - 1u;
                                probe((int)sm.pidx[warp][j]);
                            }
                            __syncwarp();   // the list is rewritten by the next group
                        }
                    } else if constexpr (!SM::kMaskOnly) {
                        while (mask) {
                            const int pa = g * 32 + __ffs(mask) - 1;
                            mask &= mask - 1;
                            if (kPUnroll == 2 && mask) {
                                const int pb = g * 32 + __ffs(mask) - 1;
                                mask &= mask - 1;
                                probe(pa);
                                probe(pb);
                            } else {
                                probe(pa);
                            }
                        }
                    }
                };
                if constexpr (kBalance && NG == NQ) {
                    // the stage's (sub-tile, group) pairs (bit q * NG + g),
                    // dealt to the consumer warps in turn, so that a stage
                    // whose work sits in one sub-tile still spreads over
                    // all warps
                    uint32_t rank = 0;
                    int curq = -1;
                    for (uint32_t mm = smask; mm; mm &= mm - 1u, ++rank) {
                        if ((int)(rank % (uint32_t)NG) != warp) continue;
                        const int bit = __ffs(mm) - 1;
                        const int q = bit / NG;
                        if (q != curq) {
                            load_sub(q);
                            curq = q;
                        }
                        test_group(bit % NG);
                    }
                } else {
                    // warp w takes sub-tile w (rotated by the stage number
                    // with SKY_REFINE_BALANCE = 2) and every group within its reach
                    const int q = SKY_REFINE_BALANCE == 2 ? (int)((warp + k) % (uint32_t)NQ) : warp;
                    const uint32_t gm = (smask >> (q * NG)) & ((1u << NG) - 1u);
                    if (gm) {
                        load_sub(q);
#pragma unroll
                        for (int g = 0; g < NG; ++g)
                            if ((gm >> g) & 1u) test_group(g);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[s]);
        }
        if (lane == 0 && listed) atomicAdd(&res->pairs, 32ull * listed);  // 32 q-lanes per listed p
        if (lane == 0 && gscans) atomicAdd(&res->groups, (unsigned long long)gscans);
        const uint32_t wh = __reduce_add_sync(kFull, hits), we = __reduce_add_sync(kFull, exact);
        if (lane == 0 && wh) atomicAdd(&res->hits, (unsigned long long)wh);
        if (lane == 0 && we) atomicAdd(&res->exact, (unsigned long long)we);
    }
    __syncthreads();
    if (SPARSE && kSparseLive > 0 && sm.sparse && !sm.failed && sm.live != 0u) {
        // ---------------------------------------------------------- sparse mode
        constexpr int NW = NQ + 1;                        // all five warps
        constexpr int DWL = DW == 3 ? 4 : DW;             // 7-bit code words per sparse-list entry
        uint32_t* LC = sm.plist[0];                       // the consumers' lists are free now
        uint8_t* LI = sm.pidx[0];
        if (warp == 0) {
            uint32_t nl = 0;
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const uint32_t lm = sm.livemask[g];
                if ((lm >> lane) & 1u) {
                    const uint32_t r = nl + __popc(lm & ((1u << lane) - 1u));
                    if (r < 32u) {
#pragma unroll
                        for (int w = 0; w < DW; ++w) LC[r * DWL + w] = sm.pP[(g * 32 + lane) * DW + w];
                        LI[r] = (uint8_t)(g * 32 + lane);
                    }
                }
                nl += __popc(lm);
            }
            if (lane == 0) sm.nlist = nl < 32u ? nl : 32u;
        }
        __syncthreads();
        const int nl = (int)sm.nlist;
        const uint32_t E = sm.scan_end;
        unsigned long long spairs = 0;
        uint32_t shits = 0, sexact = 0;
        // windows of up to 32 q-tiles from the resume point on, dealt to the
        // warps in turn: consecutive tiles, or, with the layer-1 cell index,
        // the tiles of the subsets of the listed p's cells (every warp runs
        // the same generator and takes every NW-th window)
        const uint32_t R = sm.resume;
        uint32_t Us = 0;
        constexpr bool kSparseIdx = DP >= SKY_REFINE_INDEX_SPARSE_MIN_DP;
        if (MLO != nullptr && kSparseIdx) {
            if (lane < nl) {
                uint32_t pc[DW];
                load_entry<DW>(LC + lane * DWL, pc);
                Us = cell_of_codes<DW>(pc);
            }
            Us = __reduce_or_sync(kFull, Us);
        }
        const bool sidx = MLO != nullptr && kSparseIdx && index_pays(Us, R, E);
        if (sidx) cellwin_init(sm.cwin[warp], Us, R, E);
        uint32_t wi = 0, wnext = R + (uint32_t)warp * 32u;
        while (true) {
            uint32_t wbase, wmk;
            if (sidx) {
                bool got;
                while ((got = cellwin_next<1u>(sm.cwin[warp], MLO, MHI, wbase, wmk))) {
                    const bool mine = wi % (uint32_t)NW == (uint32_t)warp;
                    ++wi;
                    if (mine) break;
                }
                if (!got) break;
            } else {
                if (wnext > E) break;
                wbase = wnext;
                wmk = 0xffffffffu;
                wnext += NW * 32u;
            }
            if (__shfl_sync(kFull, sm.live, 0) == 0u) break;
            const uint32_t t = wbase + (uint32_t)lane;
            uint32_t rm = 0;   // listed p's whose codes reach this tile's minimum
            if (t <= E && !own(t) && ((wmk >> lane) & 1u)) {
                uint32_t mn[DW];
#pragma unroll
                for (int w = 0; w < DW; ++w) mn[w] = __ldg(SUB + ((int64_t)t * kSubSlots + NQ) * DW + w);
                for (int i = 0; i < nl; ++i) {
                    uint32_t pc[DW];
                    load_entry<DW>(LC + i * DWL, pc);
                    uint32_t r = kHigh;
#pragma unroll
                    for (int w = 0; w < DW; ++w) r &= pc[w] - mn[w];
                    if (r == kHigh) rm |= 1u << i;
                }
            }
            uint32_t tiles = __ballot_sync(kFull, rm != 0u);
            while (tiles) {
                const int b = __ffs(tiles) - 1;
                tiles &= tiles - 1;
                const uint32_t tt = wbase + (uint32_t)b;
                uint32_t em = __shfl_sync(kFull, rm, b);
                uint32_t qc[4][DW];   // q's j * 32 + lane of tile tt
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int w = 0; w < DW; ++w) qc[j][w] = __ldg(C + ((int64_t)tt * kTQ + j * 32 + lane) * DW + w);
                if (tiles) {   // the next relevant tile's codes on their way into L1 while this one is tested
                    const uint32_t tn = wbase + (uint32_t)(__ffs(tiles) - 1);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(C + ((int64_t)tn * kTQ + j * 32 + lane) * DW));
                }
                while (em) {
                    const int i = __ffs(em) - 1;
                    em &= em - 1;
                    const int pi = (int)LI[i];
                    const bool alive = __shfl_sync(kFull, (sm.livemask[pi >> 5] >> (pi & 31)) & 1u, 0) != 0u;
                    if (!alive) continue;
                    spairs += 128;
                    uint32_t pc[DW];
                    load_entry<DW>(LC + i * DWL, pc);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        uint32_t D[DW];
                        uint32_t a = kHigh;
#pragma unroll
                        for (int w = 0; w < DW; ++w) {
                            D[w] = pc[w] - qc[j][w];
                            a &= D[w];
                        }
                        if (a == kHigh) {   // code(q) <= code(p) in every dimension (rare)
                            ++shits;
                            uint32_t eq = 0;
#pragma unroll
                            for (int w = 0; w < DW; ++w) eq |= has_zero_byte(D[w] ^ kHigh);
                            bool dom = true;
                            if (eq) {
                                ++sexact;
                                const float* qx = X + ((int64_t)tt * kTQ + j * 32 + lane) * DP;
                                const float* px = SM::kPxSmem ? &sm.pX[pi * DP] : X + (pbase + pi) * DP;
                                bool le = true, lt = false;
#pragma unroll
                                for (int kk = 0; kk < DP; kk += 4) {
                                    const float4 u = __ldg(reinterpret_cast<const float4*>(qx + kk));
                                    const float4 v = *reinterpret_cast<const float4*>(px + kk);
                                    le &= (u.x <= v.x) & (u.y <= v.y) & (u.z <= v.z) & (u.w <= v.w);
                                    lt |= (u.x < v.x) | (u.y < v.y) | (u.z < v.z) | (u.w < v.w);
                                }
                                dom = le && lt;
                            }
                            if (dom) {
                                const uint32_t bit = 1u << (pi & 31);
                                if (atomicAnd(&sm.livemask[pi >> 5], ~bit) & bit) atomicSub(&sm.live, 1u);
                                if constexpr (WIT) wit[ids[pbase + pi]] = ids[(int64_t)tt * kTQ + j * 32 + lane];
                            }
                        }
                    }
                }
            }
        }
        if (lane == 0 && spairs) atomicAdd(&res->pairs, spairs);
        const uint32_t wh = __reduce_add_sync(kFull, shits), we = __reduce_add_sync(kFull, sexact);
        if (lane == 0 && wh) atomicAdd(&res->hits, (unsigned long long)wh);
        if (lane == 0 && we) atomicAdd(&res->exact, (unsigned long long)we);
        __syncthreads();
    }
    if (nparts > 1u) {
        // split scan: this part's kills go into the p-tile's record; the
        // part that finishes last reads every part's kills and writes keep
        if (tid < NG) atomicOr(&split[tid], sm.validmask[tid] & ~sm.livemask[tid]);
        __threadfence();
        __syncthreads();
        if (tid == 0) sm.lastpart = atomicAdd(&split[4], 1u) == nparts - 1u ? 1u : 0u;
        __syncthreads();
        if (sm.lastpart) {
            __threadfence();
            if (tid < NG) sm.livemask[tid] = sm.validmask[tid] & ~atomicOr(&split[tid], 0u);
        }
        __syncthreads();
    }
    if (tid < kTQ && !sm.failed && (nparts == 1u || sm.lastpart)) {
#pragma unroll
        for (int h = 0; h < NT; ++h) {
            const int pi = h * kTQ + tid;
            if (pbase + pi < m && ((sm.livemask[pi >> 5] >> (pi & 31)) & 1u)) keep[ids[pbase + pi]] = 1;
        }
    }
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
