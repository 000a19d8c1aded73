// sky_internal.h -- kernel launchers and workspace layout of libsky (host side).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

struct sky_query;   // include/sky.h

namespace sky {

// Per-call result block, copied to the host once at the end of a call.
struct DevResult {
    uint32_t survivors;        // points left after step (c) (and the filter)
    uint32_t count;            // skyline size
    uint32_t err;              // SKY_DEV_ERR_* bits
    uint32_t n_filter_used;    // proposals that snapped to a data point
    unsigned long long pairs;  // candidate pairs examined by the refinement
    uint32_t occupied_cells;   // filled on request (grid statistics)
    uint32_t surviving_cells;
    uint32_t refine_m;         // survivors left for the full refinement after its pre-pass
    uint32_t pad1;
    unsigned long long tiles;  // q-tiles streamed by the refinement (all CTAs)
    unsigned long long groups; // (warp, p-group) list scans in the refinement
    unsigned long long hits;   // pairs with code(q) <= code(p) in every dimension
    unsigned long long exact;  // pairs that ran the float test
};



// Value -> column map of the map pass.
enum MapMode { kMapAuto = 0, kMapUnit = 1, kMapMinMax = 2 };

// Everything one skyline computation needs on the device.
struct Plan {
    // problem
    const float* pts = nullptr;
    int64_t n = 0;
    int d = 0;
    int64_t ld = 0;
    int log2g = 0;
    int map_mode = kMapAuto;   // MapMode
    bool tma_ok = false;       // 16-byte aligned and ld == d
    int morton_bits = 0;       // bits per dimension of the sort key
    bool survivors_only = false;   // stop after step (c)

    // workspace (device)
    uint32_t* mm_min = nullptr;      // [d] ordered-uint min
    uint32_t* mm_max = nullptr;      // [d] ordered-uint max
    float* params = nullptr;         // [4][16]: offset, cell scale, code scale, morton scale
    uint32_t* ckey = nullptr;        // [n] cell key per point (Eq. 1 columns packed)
    uint32_t* mkey = nullptr;        // [n] Morton key per point (spatial sort key)
    uint32_t* sflags = nullptr;      // [ceil(n / 32)] survivor flag bits of step (c)
    uint32_t* scount = nullptr;      // [kSurvMaxBlocks] survivors per block of step (c)
    uint32_t* occ = nullptr;         // [words] occupancy bitmap
    uint32_t* occ_stage = nullptr;   // [map blocks][words] private bitmaps (grids of <= kPrivWords words)
    uint8_t* occb = nullptr;         // [32 words] byte-per-cell occupancy of larger grids (byte-map marking)
    bool bytemap = false;            // layout: give grids above kPrivWords words a byte map
    uint32_t* pre = nullptr;         // [words] inclusive prefix-OR of occ
    uint32_t* dom = nullptr;         // [words] dominated bitmap (grid API only)
    int64_t words = 0;
    unsigned long long* lb_states = nullptr;  // look-back states (max of both scans)
    uint32_t* lb_counter = nullptr;           // [2] tile counters
    int64_t lb_tiles = 0;
    uint32_t* surv_key = nullptr;    // [n] morton key of survivors
    uint32_t* surv_idx = nullptr;    // [n] row id of survivors (ascending)
    uint32_t* sort_key2 = nullptr;   // [n] ping-pong buffers
    uint32_t* sort_val2 = nullptr;
    uint32_t* hist = nullptr;        // [256][sort_blocks]
    uint32_t* digit_total = nullptr; // [4][256] per-pass digit totals
    int64_t sort_blocks = 0;
    float* X = nullptr;              // [n_pad][dp] sorted survivor coordinates
    uint32_t* C = nullptr;           // [n_pad][dp/4] 7-bit codes
    int32_t* ids = nullptr;          // [n_pad] row id per sorted survivor
    uint32_t* tmax = nullptr;        // [tiles][dp/4] byte-wise max code of each tile
    uint32_t* tile_cost = nullptr;   // [tiles] cost estimate of each p-tile
    uint32_t* tile_order = nullptr;  // [tiles + kSplitExtra] p-tiles, largest cost first (split ones once per part)
    uint32_t* tile_part = nullptr;   // [tiles + kSplitExtra] part | parts << 8 | split slot << 16 of each entry
    uint32_t* split_state = nullptr; // [kSplitSlots][5] kills (4 words) and finished parts of each split p-tile,
                                     // then the number of order entries
    uint32_t* subcode = nullptr;     // [tiles][5][dp/4] byte-wise min code of each 32-point sub-tile, then of the tile
    uint32_t* tile_end = nullptr;    // [tiles] last q-tile whose first Morton key <= the tile's last key
    uint32_t* supmin = nullptr;      // [ceil(tiles / 32)][dp/4] byte-wise min code of each run of 32 tiles
    uint32_t* cidx = nullptr;        // [2][2^d] layer-1 cell index: ~first tile, last tile + 1 (0: no point)
    uint32_t* tend_pre = nullptr;    // [tiles] last q-tile of the refinement's pre-pass scan
    uint32_t* tmask = nullptr;       // [tiles][4][128] threshold masks of the 32-point sub-tiles (mask probe)
    unsigned long long* pre_states = nullptr;   // [lb_tiles] look-back states of the pre-pass compaction
    uint8_t* keep = nullptr;         // [n] 1 = skyline
    float* filt = nullptr;           // [16][16] snapped filter points
    unsigned long long* snap = nullptr;  // [16] packed (sum, row) argmin
    DevResult* res = nullptr;
    int32_t* witness = nullptr;      // witness mode: [n] dominating row of every dropped point (caller's)
    // last sort output
    const uint32_t* sorted_val = nullptr;
    const uint32_t* sorted_key = nullptr;
};

// One query of a batch (device copy; pointers resolved into the workspace).
struct QueryPlan {
    const float* base;        // table row row_begin
    int64_t n;                // rows of the query
    int64_t rs, cs;           // element (r, k) = base[r * rs + col[k] * cs]
    int64_t row_begin;
    int32_t d, dp, log2g, mbits, passes, dpclass;
    int32_t col[16];
    int32_t quadrant;         // 1: only rows >= origin (every column) take part
    int32_t invalid;          // planned on the device: 1 bad query, 2 beyond the workspace bound (n = 0)
    float origin[16];
    int64_t words, chunks, tiles;
    uint2* keys;
    uint32_t* occ;
    uint32_t* pre;
    unsigned long long* lb_a;
    unsigned long long* lb_b;
    uint32_t* surv_key;
    uint32_t* surv_idx;
    uint32_t* key2;
    uint32_t* val2;
    uint32_t* hist;
    uint32_t* digit_total;    // [4][256]
    float* X;
    uint32_t* C;
    int32_t* ids;
    uint32_t* sub;
    uint32_t* tend;           // [tiles] last q-tile whose first Morton key <= the tile's last key
    uint32_t* supmin;         // [ceil(tiles / 32)][dp / 4] byte-wise minimum code of each run of 32 tiles
    uint32_t* cidx;           // [2][2^d] layer-1 cell index: ~first tile, last tile + 1 (0: no point)
    uint8_t* keep;
    int32_t* stage;
    uint32_t* tmask;          // [tiles][4][128] threshold masks (dp >= 12: the mask probe); NULL below
    DevResult* res;
};

constexpr int kRefineTile = 128;   // points per refinement tile
// Split refinement scans: order entries beyond one per p-tile, and split
// p-tiles, at most (bounds of the rule in k_cost_order for up to 148 SMs x
// 9 CTAs)
constexpr int kSplitExtra = 2 * 148 * 9;
constexpr int kSplitSlots = 2 * 148 * 9;
// threshold masks per tile for the refinement's mask probe: 4 sub-tiles of
// 32 points x 16 dimensions x 8 levels of the 3-bit codes
constexpr int kMaskWords = 4 * 128;
constexpr int kSurvMaxBlocks = 4096;  // blocks of the survivor passes (at most 6 per SM)
constexpr int kMapMaxBlocks = 1024;   // blocks of the map pass
constexpr int64_t kPrivWords = 2048;  // grids of at most 2^16 cells are marked in shared memory first
constexpr int kScanItems = 8;      // items per thread in the look-back scans
constexpr int kScanThreads = 256;
constexpr int kScanTile = kScanItems * kScanThreads;
constexpr int kSortItems = 8;
constexpr int kSortThreads = 256;
constexpr int kSortTile = kSortItems * kSortThreads;

// Workspace bytes for a plan (all buffers, 256-byte aligned each).
size_t plan_workspace_bytes(int64_t n, int d, int log2g, bool grid_api);
// Carves `ws` into the plan's buffers.
void plan_carve(Plan& p, void* ws, bool grid_api);

// Launchers (k_grid.cu)
// Steps (a)+(b) in the plan's map mode (min/max pass, parameters, map pass,
// and in automatic mode the decision and the gated second map pass).
cudaError_t launch_build(const Plan& p, cudaStream_t s);
cudaError_t launch_build_params(const Plan& p, cudaStream_t s);   // launch_build without the map pass
int build_kernel_count(const Plan& p);
cudaError_t launch_prefix_or(const Plan& p, cudaStream_t s);
int prefix_kernel_count(const Plan& p);
bool prefix_trivial(const Plan& p);   // log2g <= 1: the survivor pass reads the bitmap itself
int map_blocks_bound(int64_t n);
void launch_mm_reset(const Plan& p, cudaStream_t s);
cudaError_t launch_minmax_accumulate(const Plan& p, cudaStream_t s);
// the value map's parameters; with `clear` (the first launch of a call) the
// automatic map's sample kernel also zeroes the result block and a small bitmap
cudaError_t launch_params(const Plan& p, cudaStream_t s, bool clear = false);
cudaError_t launch_map_pass(const Plan& p, bool mark, cudaStream_t s);
void set_last_error(const char* msg);   // the message sky_last_error() returns
cudaError_t launch_dominated(const Plan& p, cudaStream_t s);
cudaError_t launch_snap(const Plan& p, const float* d_prop, int n_prop, cudaStream_t s);
// idx_out: where the survivor row ids go (default: p.surv_idx; the caller's
// buffer of a survivors-only call that can hold n ids)
cudaError_t launch_survivors(const Plan& p, int n_filter, cudaStream_t s, uint32_t* idx_out = nullptr);
cudaError_t launch_copy_survivors(const Plan& p, int32_t* out, int64_t capacity, cudaStream_t s);
cudaError_t launch_cell_stats(const Plan& p, cudaStream_t s);
// k_sort.cu
cudaError_t launch_sort(Plan& p, cudaStream_t s);
// k_refine.cu
// mcount: the number of sorted survivors to lay out (default &p.res->survivors)
cudaError_t launch_gather(const Plan& p, cudaStream_t s, const uint32_t* mcount = nullptr);
// whether launch_refine runs the pre-pass (3 more kernels: refine, compaction, gather)
bool refine_prepass(const Plan& p);
// whether the refinement of d-dimensional points uses the mask probe (and
// the workspace holds p.tmask)
bool refine_mask_probe(int d);
cudaError_t launch_refine(const Plan& p, cudaStream_t s);
cudaError_t launch_emit(const Plan& p, int32_t* out, int64_t capacity, cudaStream_t s);
// k_tournament.cu: Algorithm 3 (tournament tree) classes of one layer
size_t tournament_workspace_bytes(int d, int log2g);
cudaError_t launch_tournament(const uint32_t* occ, int d, int log2g, uint8_t* cls, void* ws, cudaStream_t s);
int tournament_kernel_count(int d, int log2g);
// k_witness.cu: witnesses of the points step (c) dropped (rep: 2^(log2g d) ints of scratch)
cudaError_t launch_witness_cells(const Plan& p, int32_t* rep, int n_prop, cudaStream_t s);

// One batched launch (k_batched.cu): device pointers into the workspace.
struct BatchLaunch {
    const QueryPlan* qps = nullptr;
    int nq = 0;
    const int64_t* pchunk = nullptr;   // [nq+1] exclusive prefix of 2048-row chunks
    int64_t chunk_items = 0;
    const int64_t* ptile = nullptr;    // [nq+1] exclusive prefix of 128-point tiles
    int64_t tile_items = 0;
    const int2* items = nullptr;       // refinement (query, p-tile) items, grouped by class
    int class_begin[4] = {0, 0, 0, 0};
    int class_items[4] = {0, 0, 0, 0};
    uint32_t* claims = nullptr;        // [6] work counters (zeroed per launch)
    void* zero_base = nullptr;         // region cleared at the start of every launch
    size_t zero_bytes = 0;
    int max_passes = 0;
    int64_t max_words = 1;
    int refine_ctas_per_sm = 0;
    // per padded-dimension class (d <= 4, 8, 12, 16) refinement variant
    int class_ctas[4] = {0, 0, 0, 0};       // persistent CTAs per SM (0: refine_ctas_per_sm)
    int class_stages[4] = {8, 8, 8, 8};     // ring depth: 4 or 8
    int class_fast[4] = {0, 0, 0, 1};       // fast-code list probe
    bool concurrent_classes = false;        // class kernels as parallel branches
    cudaStream_t class_streams[4] = {};     // (owned by the batch)
    cudaEvent_t fork = nullptr, joins[4] = {};
    // planned on the device: [0..3] first item, [4..7] items of each class
    // (the counts above are then bounds, and chunk / tile counts are read
    // from pchunk[nq] / ptile[nq])
    const int* d_class = nullptr;
    int32_t* out = nullptr;
    int64_t capacity = 0;
    int64_t* offsets = nullptr;
    int32_t* status = nullptr;
};
cudaError_t launch_batched(const BatchLaunch& b, cudaStream_t s);
int batched_kernel_count(const BatchLaunch& b);
// k_bplan.cu: the batch planned on the device (sky_skyline_batched_device)
size_t batched_device_workspace_bytes(int n_cols, int nq, int64_t max_total_rows);
cudaError_t launch_batched_device(const float* table, int64_t n_rows, int n_cols, int64_t rs, int64_t cs,
                                  const ::sky_query* d_queries, int nq, int64_t max_total_rows, void* ws,
                                  size_t ws_bytes, int32_t* out, int64_t capacity, int64_t* offsets, int32_t* status,
                                  cudaStream_t s);

constexpr int kMaxAutoLayer = 8;   // the automatic layer never exceeds 8 (256 columns per dimension)
int auto_log2g(int64_t n, int d);
int morton_bits_for(int64_t n, int d);

}  // namespace sky
