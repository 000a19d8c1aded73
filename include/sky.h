/*
 * sky.h -- C ABI of libsky: exact grid-pruned skyline computation on one GPU.
 *
 * The method is SkyCell (Li, Gu, Qi, Yu, arXiv 2107.09993). Given n points
 * P in R^d, it returns the skyline S, the points that no other point
 * dominates (Definitions 1 and 2, Sec. 3): p dominates q when
 * p[k] <= q[k] in every dimension k and p[l] < q[l] in at least one
 * ("smaller is better").
 *
 * The hot path has four steps, each behind one of the calls below:
 *   (a) map every point to its cell of the finest grid layer (Eq. 1);
 *   (b) mark occupied cells in a bitmap;
 *   (c) prune every cell dominated by an occupied cell (Definition 3),
 *       which holds no skyline point (Sec. 3, cell types);
 *   (d) run exact point-vs-point dominance tests on the survivors and
 *       compact the skyline's row indices in ascending order.
 *
 * Conventions shared by every call
 *   Points     device pointer to float32, row-major, n rows of d values with
 *              a row stride of `ld` floats (ld >= d). The pointer must be
 *              4-byte aligned; 16-byte alignment with ld == d selects the
 *              bulk-copy (TMA) streaming path. 1 <= d <= 16, 0 <= n < 2^31.
 *              NaN or +-inf anywhere -> SKY_ERR_NONFINITE.
 *   Output     ascending 0-based int32 row indices. The set is unique and
 *              the order canonical, so results compare bit for bit.
 *   Ownership  the caller owns every buffer it passes and keeps it alive
 *              until the call (or, for a grid handle, sky_grid_destroy)
 *              returns; the library never frees caller memory. Handles own
 *              their device workspace.
 *   Streams    `stream` is a cudaStream_t passed as void* (NULL = legacy
 *              default stream). All device work is enqueued on it.
 *   Errors     every call returns a sky_status; no C++ exception crosses the
 *              boundary. sky_last_error() gives a thread-local detail string.
 *              Calls are re-entrant across distinct handles; one handle must
 *              not be used from two threads at once.
 */
#ifndef SKY_H_
#define SKY_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SKY_API __attribute__((visibility("default")))
#else
#define SKY_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sky_status {
    SKY_OK = 0,
    SKY_ERR_INVALID_ARGUMENT = 1, /* bad pointer, size, stride or option      */
    SKY_ERR_NONFINITE = 2,        /* NaN or infinity in the input              */
    SKY_ERR_CAPACITY = 3,         /* output buffer too small; count is set     */
    SKY_ERR_OUT_OF_MEMORY = 4,    /* device workspace allocation failed        */
    SKY_ERR_CUDA = 5,             /* a CUDA runtime call failed (or the        */
                                  /* refinement's shared memory was not        */
                                  /* 256-byte aligned; sky_last_error says)    */
    SKY_ERR_TOO_LARGE = 6,        /* grid of 2^(log2_g*d) cells above 2^27     */
    SKY_ERR_TIMEOUT = 7,          /* a bounded device-side wait ran out        */
    SKY_ERR_NO_DEVICE = 8         /* no CUDA device, or not an sm_103 device   */
} sky_status;

/* Options of one skyline computation. Zero-initialise, then set fields. */
typedef struct sky_options {
    /* Cells per dimension = 2^log2_g, i.e. the finest grid layer rho of
     * Sec. 3 / Algorithm 1. -1 picks it from n and d (automatic). The grid
     * must satisfy log2_g * d <= 27 (dense bitmap), else SKY_ERR_TOO_LARGE. */
    int32_t log2_g;
    /* Value -> column map of step (a). Any monotone map keeps the result
     * exact; the choice only changes how much step (c) prunes.
     * 1: Eq. 1 as printed, for data in the unit cube: column =
     *    floor(x * 2^log2_g), values outside [0,1) clamped to the first or
     *    last column.
     * 2: per-dimension min/max normalisation first (one extra read pass).
     * 0 (default): automatic, decided on the strided sample of rows 0, t,
     *    2t, ... with t = ceil(n / 4096): Eq. 1 when every sampled dimension
     *    lies in [0,1] and spans at least half of it, otherwise min/max
     *    scales from the sample (rows outside its range fall into the edge
     *    columns). One map pass. */
    int32_t assume_unit;
    /* Optional pre-filter proposals: n_filter points of d floats (device,
     * row-major). Any coordinates are accepted. Each proposal f is replaced by
     * the data point q <= f (every dimension) with the smallest coordinate
     * sum, or dropped when there is none; then every point dominated by such
     * a q is removed before step (d). Since every q is a real data point this
     * never changes the result, only the work. NULL / 0 = no filter. */
    const float* d_filter_pts;
    int32_t n_filter;             /* 0..16 */
    /* 1: stop after step (c) [Corollary 4]; the result is then the ascending
     * row ids of the points whose cell is not dominated (and that no snapped
     * proposal dominates) -- a superset of the skyline, the candidates of
     * step (d). 0 (default): the skyline. */
    int32_t survivors_only;
} sky_options;

/* Opaque grid handle: steps (a)-(c) for one point set. Owns its workspace. */
typedef struct sky_grid sky_grid;

/* Statistics of a grid handle (filled by sky_grid_stats). */
typedef struct sky_grid_stats_t {
    int32_t log2_g;               /* chosen layer: 2^log2_g cells per dimension */
    int32_t d;
    int64_t n;
    int64_t occupied_cells;       /* cells holding at least one point          */
    int64_t surviving_cells;      /* occupied cells not dominated (Def. 3)     */
    int64_t surviving_points;     /* points handed to step (d)                 */
    int32_t n_filter_used;        /* proposals that snapped to a data point    */
    int32_t error_flags;          /* device error bits (see sky_status)        */
} sky_grid_stats_t;

/* Device views into a grid handle, for inspection and tests. Valid until
 * sky_grid_destroy. All arrays live on the device. */
typedef struct sky_grid_view {
    const uint32_t* cell_key;     /* [n] cell key of point i: sum_k c[k] << (log2_g*k)      */
    const uint32_t* occupied;     /* [words] bit c set when cell c holds a point            */
    const uint32_t* dominated;    /* [words] bit c set when cell c is dominated (Def. 3)    */
    const int32_t* survivors;     /* [surviving_points] row ids after step (c), ascending    */
    const float* cell_offset;     /* [d] value -> column map: t = (x - offset) * scale      */
    const float* cell_scale;      /* [d]                                                    */
    int64_t words;                /* 32-bit words per bitmap = max(1, 2^(log2_g*d) / 32)    */
} sky_grid_view;

/*
 * Steps (a) and (b) [Eq. 1; Sec. 4, Algorithm 1 line 1]: map each point to
 * its cell of layer log2_g and mark occupied cells. Allocates the handle and
 * its workspace; enqueues the work on `stream` and returns without waiting.
 * `d_pts` is borrowed and must stay valid until sky_grid_destroy.
 */
SKY_API sky_status sky_build_grid(const float* d_pts, int64_t n, int32_t d, int64_t ld,
                          const sky_options* opt, void* stream, sky_grid** out);

/*
 * Step (c) [Definition 3; Sec. 3 "dominated cells"; Corollary 4]: mark every
 * cell dominated by an occupied cell and compact the rows of the remaining
 * points (survivors). A cell c is dominated iff some occupied cell c' has
 * c'[k] < c[k] in every dimension; computed as an inclusive prefix-OR of the
 * occupancy bitmap over all d dimensions, read one cell down the diagonal.
 * Optional proposals (see sky_options.d_filter_pts) additionally remove points
 * dominated by their snapped data points. Asynchronous on `stream`.
 */
SKY_API sky_status sky_prune_cells(sky_grid* grid, const float* d_filter_pts, int32_t n_filter,
                           void* stream);

/* Synchronises the grid's stream and reports its statistics. */
SKY_API sky_status sky_grid_stats(const sky_grid* grid, sky_grid_stats_t* out);

/* Device pointers into the handle (no synchronisation). */
SKY_API sky_status sky_grid_get_view(const sky_grid* grid, sky_grid_view* out);

/* Arrays of a grid handle that sky_grid_copy_out can copy. */
typedef enum sky_grid_array {
    SKY_GRID_CELL_KEY = 0,        /* uint32[n]                                  */
    SKY_GRID_OCCUPIED = 1,        /* uint32[words]                              */
    SKY_GRID_DOMINATED = 2,       /* uint32[words] (after sky_prune_cells)      */
    SKY_GRID_SURVIVORS = 3,       /* int32[surviving_points] (after pruning)    */
    SKY_GRID_CELL_MAP = 4,        /* float[32]: offset[16] then scale[16]       */
    SKY_GRID_SNAP = 5             /* uint64[16] (after pruning with proposals):
                                   * for proposal j, (ordered binary32 coordinate
                                   * sum << 32) | row of the data point it was
                                   * snapped to; all ones when no point is <= it */
} sky_grid_array;

/* Copies one array of the handle into caller memory d_dst (device) of
 * `bytes` bytes; synchronises the handle's stream. Returns SKY_ERR_CAPACITY
 * when `bytes` is smaller than the array. */
SKY_API sky_status sky_grid_copy_out(const sky_grid* grid, sky_grid_array which, void* d_dst, size_t bytes);

/* Frees the handle and its workspace (NULL is accepted). Synchronises the
 * handle's stream first. */
SKY_API void sky_grid_destroy(sky_grid* grid);

/*
 * Steps (a)-(d) [Algorithm 1; Definitions 1-3]: the skyline of the n points.
 * Writes the ascending row indices of the skyline to d_out_idx (device,
 * capacity out_capacity entries) and the skyline size to *h_out_count (host).
 * If out_capacity is smaller than the skyline, returns SKY_ERR_CAPACITY with
 * *h_out_count set to the size needed; the buffer's contents are then
 * undefined. Synchronises `stream` once, to read the count. The workspace is
 * taken from the device's stream-ordered pool and returned before the call
 * ends.
 */
SKY_API sky_status sky_skyline(const float* d_pts, int64_t n, int32_t d, int64_t ld,
                       const sky_options* opt, int32_t* d_out_idx, int64_t out_capacity,
                       int64_t* h_out_count, void* stream);

/*
 * Same as sky_skyline, with host buffers: copies the points to the device,
 * runs steps (a)-(d) and copies the indices back. h_pts (n*ld floats) and
 * h_out_idx (out_capacity ints) are host memory; page-locked memory makes the
 * copies asynchronous. Synchronises `stream` before returning.
 */
SKY_API sky_status sky_skyline_host(const float* h_pts, int64_t n, int32_t d, int64_t ld,
                            const sky_options* opt, int32_t* h_out_idx, int64_t out_capacity,
                            int64_t* h_out_count, void* stream);

/*
 * Witness mode of sky_skyline, a checking aid [Definitions 1-3]: the same
 * skyline (same arguments, same result in d_out_idx / *h_out_count), and for
 * every row i, d_witness[i] (device, n int32, caller-owned) =
 *   -1  when i is in the skyline;
 *   j   the row of a point that dominates point i (Definition 1), when the
 *       path dropped i: for a point of a dominated cell (step c, Def. 3), a
 *       point of an occupied cell that is below it in every dimension; for a
 *       point a snapped proposal removed (step c'), that proposal's row; for
 *       a point the refinement removed (step d), the survivor that did;
 *   -2  when step (c) dropped i and no such point was found (an error of the
 *       path; a correct run never writes it).
 * So a caller verifies every dropped point with one O(d) test each, without
 * computing the skyline itself. survivors_only must be 0. Slower than
 * sky_skyline and allocates per call: workspace plus 4 * 2^(log2_g * d)
 * bytes of cell scratch from the stream-ordered pool; no CUDA graph.
 * Synchronises `stream`.
 */
SKY_API sky_status sky_skyline_witness(const float* d_pts, int64_t n, int32_t d, int64_t ld,
                                       const sky_options* opt, int32_t* d_out_idx, int64_t out_capacity,
                                       int64_t* h_out_count, int32_t* d_witness, void* stream);

/*
 * The paper's tournament-tree ShrinkKeyCells [Algorithm 3, Sec. 5.2;
 * Theorem 2] on one grid layer, as a comparison variant of step (c): the
 * cells of the layer are the leaves of a complete binary tree in the
 * enumeration order of a rotation of the dimensions; each of d passes runs an
 * up-sweep of pointers u and a down-sweep of pointers l (one kernel per tree
 * level), then the dimensions rotate and every leaf's u takes its l. A
 * pointer is a non-empty cell. Reading (the printed form does not reproduce
 * Definitions 4-5): all cells are leaves, and a pass compares in one
 * dimension -- the earlier pointer wins within a line of cells that differ
 * only in the rotated dimension 0 -- so that after the d passes l(c) is a
 * non-empty cell e <= c (componentwise) other than c if one exists, else c
 * when c is non-empty, else none.
 *
 *   d_occupied  device bitmap of the layer: bit c of word c / 32 set when
 *               cell c (key sum_k c[k] << (log2_g k)) holds a point; at least
 *               max(1, 2^(log2_g d) / 32) words (sky_grid_copy_out's
 *               SKY_GRID_OCCUPIED array has this layout).
 *   d_classes   device, one byte per cell: bit 0 dominated (Def. 3: every
 *               c[k] >= 1 and l(c - (1, ..., 1)) is a cell), bit 1 key cell
 *               (Def. 4: l(c) = c), bit 2 candidate cell (Def. 5 with the
 *               auxiliary key cells of Def. 6: not dominated, and l(c) is a
 *               cell or some c[k] = 2^log2_g - 1).
 *   d_ws        device workspace of sky_tournament_workspace_size(d, log2_g)
 *               bytes (20 bytes a cell), 256-byte aligned, caller-owned.
 * 1 <= d <= 16, log2_g * d <= 27 (SKY_ERR_TOO_LARGE beyond). Asynchronous on
 * `stream`; allocates nothing. sky_tournament_workspace_size returns 0 for
 * arguments outside these limits.
 */
SKY_API size_t sky_tournament_workspace_size(int32_t d, int32_t log2_g);
SKY_API sky_status sky_tournament_cells(const uint32_t* d_occupied, int32_t d, int32_t log2_g,
                                        uint8_t* d_classes, void* d_ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Many independent point sets in one call (a project addition: the paper    */
/* computes one skyline at a time). Each set is steps (a)-(d) exactly as     */
/* sky_skyline computes it; the sets run concurrently on up to four          */
/* library-internal streams, so that one set's small phases overlap another  */
/* set's large ones.                                                          */
/* ------------------------------------------------------------------------ */
typedef struct sky_set {
    const float* pts;             /* in: n*ld floats, row-major (device or host, per entry point) */
    int64_t n;                    /* in: rows, [0, 2^31)                        */
    int32_t d;                    /* in: attributes, [1, 16]                    */
    int32_t reserved0;
    int64_t ld;                   /* in: row stride in floats, >= d             */
    int32_t* out_idx;             /* in: buffer of `capacity` ints (device or host) */
    int64_t capacity;             /* in: entries of out_idx                     */
    int64_t count;                /* out: skyline size (the size needed when status is
                                   * SKY_ERR_CAPACITY); -1 when the set did not complete */
    int32_t status;               /* out: sky_status of this set                */
    int32_t reserved1;
} sky_set;

/*
 * Device-resident sets: for every sets[i], the ascending row ids of its
 * skyline go to sets[i].out_idx and the size to sets[i].count, as sky_skyline
 * would write them. `opt` applies to every set; proposals (n_filter > 0)
 * belong to one set and are rejected here. Arguments of every set are checked
 * before any work starts (SKY_ERR_INVALID_ARGUMENT / SKY_ERR_TOO_LARGE name
 * the set in sky_last_error()). A run-time failure of one set (capacity,
 * non-finite input, timeout) is recorded in its status and does not stop the
 * others. Returns SKY_OK when every set succeeded, else the status of the
 * first failing set (in index order), described by sky_last_error(). Work
 * starts after the work already queued on `stream`; the call returns when
 * every set has completed. sky_last_run_stats() then reports the sums over
 * the sets (d and log2_g of the last set); sky_last_phase_times() is not
 * updated. Workspaces and graphs are cached per set as for sky_skyline.
 */
SKY_API sky_status sky_skyline_sets(sky_set* sets, int32_t count, const sky_options* opt, void* stream);

/*
 * Host-resident sets: pts and out_idx are host memory (page-locked memory
 * makes the copies asynchronous). The inputs are copied to per-slot device
 * buffers in set order on one copy stream, so the copy of set i+1 overlaps
 * the kernels of set i; the ids of a set are copied back as soon as its count
 * is known (at most `capacity` of them; SKY_ERR_CAPACITY with count = the
 * size needed when they do not fit). Same checks, statuses and return value
 * as sky_skyline_sets. The staging buffers grow to the largest set seen and
 * are kept for later calls on the same thread.
 */
SKY_API sky_status sky_skyline_host_sets(sky_set* sets, int32_t count, const sky_options* opt, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched skylines (a project addition; the paper has no batched form).     */
/* Many skyline queries over row ranges and attribute subsets of one table   */
/* run as one CUDA-graph launch: every phase of steps (a)-(d) is one kernel  */
/* over all queries, and step (d) is a persistent kernel that pulls          */
/* (query, tile) work items, largest queries first.                          */
/* ------------------------------------------------------------------------ */

/* One query: rows [row_begin, row_begin + row_count) of the table, with the
 * columns whose bits are set in dim_mask (1 to 16 columns) as attributes.
 * With SKY_QUERY_QUADRANT in flags it is a quadrant query (the query
 * experiments of Sec. 7): the point `origin` (one value per selected column,
 * in column order) becomes the origin and only the rows >= origin in every
 * selected column take part; their skyline is returned (shifting them by the
 * origin would not change it). */
#define SKY_QUERY_QUADRANT 1u
typedef struct sky_query {
    int64_t row_begin;
    int64_t row_count;
    uint32_t dim_mask;
    uint32_t flags;               /* 0 or SKY_QUERY_QUADRANT */
    float origin[16];             /* used with SKY_QUERY_QUADRANT */
} sky_query;

/* Tuning knobs (zero-initialise; paper_2107_09993_b300/tune.py chooses them
 * by timing). None changes a result, only the time. The refinement runs one
 * persistent kernel per padded-dimension class: class c holds the queries of
 * 4c+1 .. 4c+4 attributes. */
typedef struct sky_batch_tuning {
    const int32_t* h_log2g;       /* per-query grid layer (host array), or NULL:
                                     automatic; log2_g * d <= 18 in batches     */
    int32_t refine_ctas_per_sm;   /* persistent refinement CTAs per SM (0 = max
                                     resident), for classes without their own  */
    int32_t class_ctas[4];        /* per class CTAs per SM (0 = the value above) */
    int32_t class_stages[4];      /* per class ring depth of streamed q-tiles:
                                     4 or 8 (0 = 8)                             */
    int32_t class_code[4];        /* per class pair test of the list probe:
                                     0 = library default (3-bit fast codes first
                                     for class 3 only), 1 = 7-bit codes, 2 = 3-bit
                                     fast codes first                            */
    int32_t concurrent_classes;   /* 1: the class kernels run as parallel
                                     branches of the graph (their tails overlap);
                                     0: one after another                       */
} sky_batch_tuning;

typedef struct sky_batch sky_batch;

typedef struct sky_batch_stats_t {
    int32_t n_queries;
    int32_t kernels;              /* kernels in the captured graph              */
    int32_t graph_launches_per_call;
    int32_t reserved;
    int64_t points;               /* sum of row_count                           */
    int64_t survivors;            /* points left after step (c), all queries    */
    int64_t skyline;              /* indices returned, all queries              */
    int64_t pairs;                /* candidate pairs examined in step (d)       */
} sky_batch_stats_t;

/*
 * Plans a batch on the host. d_table: n_rows x n_cols float32 on the device,
 * element (r, c) at d_table[r * row_stride + c * col_stride]; the table is
 * row-major (col_stride 1) or column-major (row_stride 1, faster: each query
 * then reads only its own columns). h_queries: host array. Nothing runs on
 * the device. *ws_bytes receives the workspace size the batch needs. The
 * table must stay valid (and unchanged in layout) for the batch's lifetime;
 * its contents may change between launches.
 */
SKY_API sky_status sky_batch_create(const float* d_table, int64_t n_rows, int32_t n_cols, int64_t row_stride,
                                    int64_t col_stride, const sky_query* h_queries, int32_t n_queries,
                                    const sky_batch_tuning* tuning, sky_batch** out, size_t* ws_bytes);

/* Workspace bytes for a batch (same planning as sky_batch_create; 0 on error). */
SKY_API size_t sky_batched_workspace_size(int64_t n_rows, int32_t n_cols, int64_t row_stride, int64_t col_stride,
                                          const sky_query* h_queries, int32_t n_queries,
                                          const sky_batch_tuning* tuning);

/*
 * Binds the caller's buffers (all device memory, owned by the caller):
 * d_ws (ws_bytes >= the size from sky_batch_create, 256-byte aligned),
 * d_out_idx (out_capacity int32), d_out_offsets (n_queries + 1 int64, CSR:
 * query q's skyline is d_out_idx[offsets[q] .. offsets[q+1]), ascending
 * global row ids), d_query_status (n_queries int32 sky_status codes). Uploads
 * the plan, runs the batch once and captures its kernel sequence into a CUDA
 * graph. Synchronises `stream`.
 */
SKY_API sky_status sky_batch_bind(sky_batch* batch, void* d_ws, size_t ws_bytes, int32_t* d_out_idx,
                                  int64_t out_capacity, int64_t* d_out_offsets, int32_t* d_query_status,
                                  void* stream);

/*
 * Steps (a)-(d) for every query of a bound batch: one CUDA-graph launch on
 * `stream`. Never allocates and never synchronises; results are valid once
 * the stream reaches this point. Queries whose indices do not fit in
 * out_capacity report SKY_ERR_CAPACITY in d_query_status (offsets stay exact).
 */
SKY_API sky_status sky_skyline_batched(sky_batch* batch, void* stream);

/* Synchronises `stream` and sums the per-query work counters. */
SKY_API sky_status sky_batch_stats(const sky_batch* batch, void* stream, sky_batch_stats_t* out);

SKY_API void sky_batch_destroy(sky_batch* batch);        /* NULL accepted */
SKY_API const char* sky_batch_last_error(void);          /* thread-local detail */

/*
 * Batched skylines planned on the device. The query records stay in device
 * memory (d_queries: n_queries sky_query) and may be written by earlier work
 * on `stream`; the planning of sky_batch_create (validation, grid layer and
 * sort-key bits, per-query arrays in the workspace, work items grouped by
 * padded-dimension class with larger queries first) runs in a kernel, so the
 * call enqueues the whole batch without synchronising, allocating or copying,
 * and may be recorded in a CUDA graph. The grids of the batched kernels are
 * sized by the bounds; the kernels read the planned counts.
 *
 * Bounds: n_queries and max_total_rows (the largest sum of row_count over
 * the valid queries that a call will see). d_ws: at least
 * sky_batched_device_workspace_size(n_cols, n_queries, max_total_rows) bytes,
 * 256-byte aligned. Outputs as in sky_batch_bind (d_out_offsets n_queries + 1
 * int64 CSR, d_query_status n_queries int32), written by the device.
 * Per-query status: SKY_ERR_INVALID_ARGUMENT for a bad row range, flag or
 * dim_mask (the query returns no indices); SKY_ERR_TOO_LARGE for every query
 * when the valid queries hold more than max_total_rows rows (nothing runs);
 * otherwise as sky_skyline_batched. Grid layers are automatic (log2_g * d
 * <= 18) and the refinement uses the library's default variants (no tuning).
 * Returns SKY_ERR_INVALID_ARGUMENT / SKY_ERR_CAPACITY (workspace too small)
 * before enqueuing anything, SKY_ERR_CUDA when a launch fails; the detail is
 * in sky_batch_last_error().
 */
SKY_API size_t sky_batched_device_workspace_size(int32_t n_cols, int32_t n_queries, int64_t max_total_rows);
SKY_API sky_status sky_skyline_batched_device(const float* d_table, int64_t n_rows, int32_t n_cols,
                                              int64_t row_stride, int64_t col_stride, const sky_query* d_queries,
                                              int32_t n_queries, int64_t max_total_rows, void* d_ws, size_t ws_bytes,
                                              int32_t* d_out_idx, int64_t out_capacity, int64_t* d_out_offsets,
                                              int32_t* d_query_status, void* stream);

/* ------------------------------------------------------------------------ */
/* Learned proposal (a project addition; the paper has no counterpart). A    */
/* 3-layer perceptron (636 -> 64 -> 64 -> 264, ReLU, bfloat16 weights, fp32  */
/* accumulation) maps distribution features of a point set to a grid layer   */
/* and 16 filter points. Parameters are one flat array of SKY_MLP_PARAMS     */
/* values in the order W1[64][636], b1[64], W2[64][64], b2[64], W3[264][64], */
/* b3[264]; outputs 0..7 score log2_g = 1..8, outputs 8 + 16 j + k give      */
/* coordinate k (normalised to the sample's min/max) of filter point j.      */
/* ------------------------------------------------------------------------ */
#define SKY_MLP_FEATURES 636
#define SKY_MLP_OUTPUTS 264
#define SKY_MLP_PARAMS 62088

/* Features of n x d points (device): d_feat[636] = 16 x 32 histograms of the
 * min/max-normalised values, the 120 pairwise Pearson correlations (k < l),
 * d/16, log2(s)/32, 0, 0 -- over the strided sample of s <= 65,536 rows
 * (every ceil(n / 65,536)-th row). d_range[32] receives the sample's min[16]
 * and max[16]. d_work: sky_features_work_floats() floats, 8-byte aligned,
 * owned by the caller and not read before it is written. Asynchronous. */
SKY_API sky_status sky_features(const float* d_pts, int64_t n, int32_t d, int64_t ld, float* d_feat,
                                float* d_range, float* d_work, void* stream);
SKY_API size_t sky_features_work_floats(void);

/* Floats of scratch the forward/backward calls need for a batch. */
SKY_API size_t sky_mlp_work_floats(int32_t batch);

/* Forward pass for `batch` feature rows: d_out[batch][264]. Asynchronous. */
SKY_API sky_status sky_mlp_forward(const uint16_t* d_params_bf16, const float* d_feat, int32_t batch,
                                   float* d_out, float* d_work, void* stream);

/* Mean loss over the batch (cross-entropy of the layer label over the
 * admissible layers log2_g * d <= 24, plus lam x masked mean squared error of
 * the filter coordinates) into *d_loss, and its gradient with respect to
 * every parameter into d_grad[SKY_MLP_PARAMS]. Asynchronous. */
SKY_API sky_status sky_mlp_backward(const uint16_t* d_params_bf16, const float* d_feat, const int32_t* d_dims,
                                    const int32_t* d_labels, const float* d_targets, const float* d_masks,
                                    int32_t batch, float lam, float* d_grad, float* d_work, float* d_loss,
                                    void* stream);

/* One AdamW step (beta 0.9 / 0.999, eps 1e-8, decoupled decay wd) on the fp32
 * master parameters; refreshes the bfloat16 copy. `step` counts from 1. */
SKY_API sky_status sky_mlp_adamw(float* d_master, uint16_t* d_bf16, float* d_m, float* d_v, const float* d_grad,
                                 int32_t step, float lr, float wd, void* stream);

/* bfloat16 copy (round to nearest even) of `count` fp32 values. */
SKY_API sky_status sky_mlp_round(const float* d_master, uint16_t* d_bf16, int64_t count, void* stream);

/* Proposal for one point set: *h_log2g (host) and d_prop[16][d] (device)
 * filter points in data units, each moved up by `inflate` x the sample range
 * in every dimension. n_ref > 0 is the set size the weights were trained at:
 * the network's layer is then moved by the automatic policy's change from
 * n_ref to n rows (clamped to 1 .. max(1, 24 / d)); n_ref = 0 keeps it.
 * d_work: sky_propose_work_floats() floats, 8-byte aligned. Synchronises. */
SKY_API sky_status sky_propose(const float* d_pts, int64_t n, int32_t d, int64_t ld, const uint16_t* d_params_bf16,
                               float inflate, int64_t n_ref, float* d_prop, int32_t* h_log2g, float* d_work,
                               void* stream);
SKY_API size_t sky_propose_work_floats(void);
SKY_API const char* sky_mlp_last_error(void);

/*
 * Skyline of a point set that one sky_skyline call cannot take: up to 2^40
 * rows, in device memory or in host memory (streamed through the GPU).
 * Steps (a)-(c) run chunk by chunk against one occupancy bitmap of the whole
 * set [Eq. 1, Definition 3, Corollary 4]: a first pass marks every chunk's
 * cells, then (after the prefix-OR) a second pass appends the rows of
 * non-dominated cells, coordinates and 64-bit row ids, to a candidate
 * buffer; one in-core refinement of the candidates gives the skyline
 * [Definition 1]. The value map is decided once for all n rows (the rule of
 * sky_options.assume_unit over the whole set). Paper: Sec. 7 runs 3.2e9
 * points, more than one device holds at d >= 2 in the paper's hardware.
 *
 *   pts            n x d float32, row stride ld floats; device memory when
 *                  host_pts = 0, host memory when host_pts = 1 (pinned
 *                  memory streams fastest; each pass reads it once).
 *   opt            log2_g, assume_unit and survivors_only as for
 *                  sky_skyline; filter proposals are not accepted here.
 *   chunk_rows     rows per chunk, 1 .. 2^30; 0 = 2^28 (device input) or
 *                  2^26 (host input). Device workspace ~16 B per chunk row
 *                  (+ two staging chunks of 4d B per row for host input).
 *   max_candidates capacity of the candidate buffer (4d + 8 B each),
 *                  1 .. 2^31 - 1; 0 = min(n, 2^28). More candidates after
 *                  step (c) -> SKY_ERR_CAPACITY, message with the count.
 *   d_out_ids      device int64[capacity]: ascending row ids of the skyline
 *                  (of the candidates when survivors_only = 1); *h_count
 *                  gets their number, also when it exceeds capacity
 *                  (SKY_ERR_CAPACITY, nothing written).
 * Synchronises with `stream` before returning; the library's memory is
 * allocated and released inside the call.
 */
SKY_API sky_status sky_skyline_chunked(const float* pts, int32_t host_pts, int64_t n, int32_t d, int64_t ld,
                                       const sky_options* opt, int64_t chunk_rows, int64_t max_candidates,
                                       int64_t* d_out_ids, int64_t capacity, int64_t* h_count, void* stream);

/* Work counters of the last sky_skyline / sky_skyline_host call made on the
 * calling thread (for measurement; not part of the result). */
typedef struct sky_run_stats {
    int64_t n;
    int32_t d;
    int32_t log2_g;               /* layer used                                 */
    int64_t survivors;            /* points left after step (c)                 */
    int64_t skyline;              /* points in the result                       */
    int64_t pairs;                /* candidate pairs examined in step (d)       */
    int32_t n_filter_used;        /* proposals that snapped to a data point     */
    int32_t kernels;              /* kernels of this library the call launched  */
    int64_t tiles;                /* survivor tiles streamed by step (d)        */
    int64_t group_scans;          /* (warp, point-group) scans in step (d)      */
    int64_t code_hits;            /* pairs whose 7-bit codes allow q <= p       */
    int64_t exact_tests;          /* pairs that needed the float test           */
} sky_run_stats;

SKY_API sky_status sky_last_run_stats(sky_run_stats* out);

/* Device times of the last sky_skyline call on the calling thread, taken with
 * CUDA events recorded on the call's stream. Off until sky_set_phase_timing()
 * selects a mode on that thread:
 *   1  events between the phases; the kernels are launched one by one (no
 *      CUDA-graph replay), which adds host launch gaps; fills the *_ms phase
 *      fields, call_ms = 0;
 *   2  two events around the call's whole kernel sequence, graph replay kept;
 *      a bounded device-side delay (50 us) precedes the first event so that
 *      the host has enqueued everything before the device reaches it; fills
 *      call_ms only.
 * 0 turns recording off; other values return SKY_ERR_INVALID_ARGUMENT. */
typedef struct sky_phase_times {
    float normalize_ms;           /* min/max pass + map parameters             */
    float map_mark_ms;            /* steps (a)+(b)                             */
    float prune_ms;               /* step (c): proposal snap + prefix-OR       */
    float survivors_ms;           /* step (c): survivor compaction             */
    float sort_ms;                /* Morton sort of the survivors              */
    float gather_ms;              /* survivor layout + tile boxes              */
    float refine_ms;              /* step (d): dominance tests                 */
    float emit_ms;                /* step (d): index compaction                */
    float call_ms;                /* mode 2: the whole kernel sequence         */
} sky_phase_times;

SKY_API sky_status sky_set_phase_timing(int32_t enable);
SKY_API sky_status sky_last_phase_times(sky_phase_times* out);

/*
 * No-allocation variant of sky_skyline, for callers that cannot allocate
 * memory at the point of the call (for example a process whose device memory
 * is already owned by its own arena allocator, or a latency-critical loop
 * where an allocation's implicit synchronisation is not allowed). The paper
 * has no counterpart: it is a deployment addition.
 *
 * Same arguments and result as sky_skyline, but every piece of scratch memory
 * comes from one fixed array in device global memory that the library
 * reserves at load time (about 12 MiB per GPU that loads the library, held
 * until the process exits); the call performs no cudaMalloc, cudaFree or
 * other allocation. Limits: n <= SKY_NOALLOC_MAX_POINTS and a grid of at most
 * 2^20 cells (log2_g * d <= 20; the automatic choice is lowered to fit);
 * larger requests return SKY_ERR_TOO_LARGE. All calls share the array and it
 * keeps the last call's contents (what must start at zero is cleared by each
 * call): calls that overlap on the GPU race and must be serialised by the
 * caller. The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before starting any stream capture on the device. Synchronises `stream`
 * once, so it cannot be recorded in a CUDA graph: on a stream that is being
 * captured it returns SKY_ERR_INVALID_ARGUMENT and enqueues nothing. Errors
 * are described by sky_noalloc_last_error() (and by sky_last_error(), which
 * each call also sets).
 */
#define SKY_NOALLOC_MAX_POINTS 65536
SKY_API sky_status sky_skyline_noalloc(const float* d_pts, int64_t n, int32_t d, int64_t ld,
                                       const sky_options* opt, int32_t* d_out_idx, int64_t out_capacity,
                                       int64_t* h_out_count, void* stream);
SKY_API const char* sky_noalloc_last_error(void);

/* ------------------------------------------------------------------------ */
/* CPU baseline: the paper's sequential SkyCell (Alg. 1 driving the          */
/* sequential ShrinkKeyCells of Alg. 2, Sec. 4) on the host. It is the      */
/* comparison the GPU path is timed against, not part of the GPU path: no   */
/* GPU entry point calls it. Host pointers only; no CUDA call.              */
/*                                                                          */
/* Layers 0 .. log2_g are built from the points' Layer-log2_g cells (Eq. 1  */
/* on the unit cube with assume_unit = 1, otherwise after the min / max of  */
/* all rows). Layer by layer the cells are enumerated slice by slice        */
/* ([cl_{d-1} .. cl_1], dimension d-1 outermost) between a start bound       */
/* doubled from the previous layer (step (a) of Alg. 2) and an end bound     */
/* from the lower slices (MinGE); the first non-empty cell of a slice below  */
/* its end bound is a key cell (Def. 4). Points of cells that no non-empty   */
/* cell dominates (Def. 3) are refined by a sort-first skyline across cells. */
/* ------------------------------------------------------------------------ */

/* h_pts: n x d float32, row stride ld >= d (floats), finite values (else
 * SKY_ERR_NONFINITE); 1 <= d <= 16, 0 <= n < 2^31. log2_g: the layer rho
 * (-1: the GPU path's automatic rule); rho * d <= 24 (SKY_ERR_TOO_LARGE
 * otherwise). assume_unit: 1 = Eq. 1 on [0,1)^d, 0 = min / max scaling.
 * Writes the ascending skyline row ids to h_out (capacity entries; a larger
 * skyline returns SKY_ERR_CAPACITY with *h_count set), *h_count = |S|, and
 * *h_candidates (optional) = the points refined after the cell pruning. */
SKY_API sky_status sky_baseline_sequential(const float* h_pts, int64_t n, int32_t d, int64_t ld, int32_t log2_g,
                                           int32_t assume_unit, int32_t* h_out, int64_t capacity,
                                           int64_t* h_count, int64_t* h_candidates);

/* The key cells (Def. 4) of Layer log2_g (>= 0) found by the baseline's
 * enumeration, as cell keys sum_k c[k] 2^(log2_g k), ascending. Same input
 * conventions as sky_baseline_sequential. */
SKY_API sky_status sky_baseline_key_cells(const float* h_pts, int64_t n, int32_t d, int64_t ld, int32_t log2_g,
                                          int32_t assume_unit, int64_t* h_keys, int64_t capacity,
                                          int64_t* h_count);

/* Thread-local detail of the last error of the two baseline calls. */
SKY_API const char* sky_baseline_last_error(void);

/*
 * Test aid for the failure path: the poll limit of the bounded device-side
 * waits of the pipeline (mbarrier waits of the streaming stages, look-back
 * flags) on the current device, for the calls that start after this one
 * returns. 0 restores the default (2^22 polls with back-off, well over a
 * second). With a small limit (e.g. 1) the waits run out: the kernels record
 * SKY_ERR_TIMEOUT, let their own bulk copies in flight land (those waits keep
 * the default limit), and return; the call reports SKY_ERR_TIMEOUT and its
 * output is undefined. The device stays usable. Synchronises the device.
 */
SKY_API sky_status sky_set_wait_limit(uint32_t polls);

/* Static text for a status code. */
SKY_API const char* sky_status_string(sky_status status);

/* Thread-local detail of the last error raised on this thread ("" if none). */
SKY_API const char* sky_last_error(void);

/* Library version string. */
SKY_API const char* sky_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SKY_H_ */
