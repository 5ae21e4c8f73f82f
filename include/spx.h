/*
 * spx.h -- C ABI of libspx, an exact point-in-polygon join, selection and
 * count-aggregate over a large point table resident in GPU memory (GB300,
 * sm_103a), through a device-resident uniform-grid index.
 *
 * The operations follow SPADE's statement of the problem (Doraiswamy and
 * Freire, "SPADE: GPU-Powered Spatial Database Engine for Commodity
 * Hardware"):
 *   - selection of points by a polygonal constraint (§5.2, "Spatial Selection"),
 *   - the polygon-point join as a collection of selections (§5.2, "Spatial Joins"),
 *   - the count aggregation, with and without materialising the join
 *     (§5.2, "Spatial Aggregations"),
 *   - exact tests where the discretisation is ambiguous (§4.3, "Boundary Index"),
 *   - for points, intersection is containment (§7, "Containment Queries"),
 *   - the two-pass Map sizing of outputs (§5.1, "Map"): a call that runs out of
 *     output space returns SPX_ECAPACITY and the size that is needed.
 *
 * Coordinates are int32 fixed point: points in [0, 2^30)^2, polygon vertices in
 * [0, 2^30]^2.  A point p lies in polygon R iff the number of edges (a, b) of R
 * with (a.y > p.y) != (b.y > p.y) and orient(a, b, p) != 0 of the sign of
 * (b.y - a.y) is odd, orient(a, b, p) = (b.x-a.x)(p.y-a.y) - (b.y-a.y)(p.x-a.x)
 * evaluated exactly: p + (eps, eps^2) is in the even-odd interior of R.  Every
 * result is exact and deterministic (byte-identical across runs, grid sizes and
 * launch shapes).
 *
 * Conventions for every call:
 *   - Status codes only; nothing throws across the ABI.  On failure,
 *     spx_last_error(ctx) describes the cause (valid until the next call on
 *     that ctx from the same thread).
 *   - A ctx is bound to one device and is not thread-safe; use one per thread.
 *   - "Device" pointers are CUDA device memory of the ctx's device (e.g. the
 *     data_ptr() of a torch tensor on that device).  The caller owns every
 *     buffer it passes; handles are owned by the ctx and released by spx_free
 *     or spx_destroy.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *     calls are asynchronous on that stream, except where a host out-parameter
 *     is requested: then the call synchronises the stream before returning.
 */
#ifndef SPX_H
#define SPX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spx_ctx spx_ctx;
typedef uint64_t spx_points; /* handle: a point table in device memory */
typedef uint64_t spx_polys;  /* handle: a polygon set (host copy + device copy) */
typedef uint64_t spx_index;  /* handle: a built grid index over a polygon set */

typedef enum {
    SPX_OK = 0,
    SPX_EINVAL = -1,    /* bad argument: null pointer, bad handle, coordinate out of range */
    SPX_ENOMEM = -2,    /* host or device allocation failed */
    SPX_ECUDA = -3,     /* a CUDA runtime call failed (message has the CUDA error) */
    SPX_ECAPACITY = -4, /* output buffer too small; the required size was written */
    SPX_ETIMEOUT = -5,  /* a bounded device wait gave up (the kernel returned early) */
    SPX_EBUSY = -6,     /* result not ready yet (serving) */
    SPX_EKERNEL = -7    /* a kernel reported an internal error through its status word */
} spx_status;

/* Create a context on CUDA device `device`.  *out receives the context. */
spx_status spx_create(int device, spx_ctx **out);

/* Destroy a context and every handle it owns.  Safe on NULL. */
void spx_destroy(spx_ctx *ctx);

/* Text of the last error on this ctx (never NULL; "" after success). */
const char *spx_last_error(const spx_ctx *ctx);

/*
 * Load a point table (§5.2 "Spatial Selection": the point data set that every
 * selection scans).  xy holds n interleaved (x, y) int32 pairs, 8 bytes per
 * point, point id = row index (n < 2^32).  With xy_is_device = 0, xy is host
 * memory and is copied to a device buffer owned by the handle (coordinates are
 * validated: 0 <= x, y < 2^30, else SPX_EINVAL).  With xy_is_device = 1 the
 * handle borrows the caller's device buffer, which must stay alive and
 * unchanged while the handle is used; it is not validated (a point outside the
 * box lies in no polygon, as the exact definition says, and the kernels skip it).
 * Device buffers must be 16-byte aligned.
 */
spx_status spx_load_points(spx_ctx *ctx, const int32_t *xy, uint64_t n, int xy_is_device, spx_points *out);

/*
 * Cell-clustered copy of a point table (§5.3 "Grid-based index filtering":
 * SPADE stores its data as a clustered grid, each cell the block of data that
 * falls into it).  *out receives a new, owned table with the same n points
 * grouped by the cells of a 2^grid_log2 x 2^grid_log2 grid over the box
 * (row-major cell order, points outside the box last; the order within a cell
 * is unspecified).  Consecutive points then share index cells, so a pass over
 * the copy reads the index from cache.  The copy keeps its cell directory
 * (each cell's row range): spx_aggregate through an index whose coarse grid
 * is no finer than the clustering grid counts every cell that lies in a
 * coarse cell INSIDE one polygon from its range, without reading its points,
 * and reads only the points of cells in mixed coarse cells (§5.3: the blocks a
 * query needs).  Only spx_aggregate takes a clustered table -- per-polygon
 * counts do not depend on the order of the points; the join, the selection
 * and the server reject it with SPX_EINVAL (their outputs are keyed by row).
 * grid_log2 in [1, 13], 0 = 12.  Device memory: 8 B per point for the copy
 * and 8 B per cell for the directory.  Synchronises the ctx's stream.
 * Errors: SPX_EINVAL, SPX_ENOMEM, SPX_ECUDA.
 */
spx_status spx_cluster_points(spx_ctx *ctx, spx_points points, int grid_log2, spx_points *out);

/* Device address of a point table (valid while the handle lives), its number
 * of points, and its clustering grid (0: row order).  Any pointer may be NULL. */
spx_status spx_points_info(spx_ctx *ctx, spx_points points, const int32_t **xy_dev, uint64_t *n, int *cluster_log2);

/*
 * Load a polygon set from host memory (§4.2, polygons are the constraint
 * canvases of selections and joins).  Polygon q is the implicitly closed ring
 * xy[2*ring_off[q] .. 2*ring_off[q+1]) of int32 (x, y) vertices, 0 <= x, y <=
 * 2^30; ring_off has P + 1 non-decreasing entries with ring_off[0] = 0.  Rings
 * may be clockwise or counter-clockwise, concave, self-intersecting (even-odd)
 * or degenerate (then nothing is inside).  Polygons may overlap.  P < 2^30.
 * The data are copied.
 */
spx_status spx_load_polygons(spx_ctx *ctx, const int32_t *xy, const uint64_t *ring_off, uint32_t P, spx_polys *out);

/* Grid-index parameters (§4.3 canvas indexes; §5.3 grid cell size; §7 tuning). */
typedef struct {
    int grid_log2;   /* coarse grid of 2^grid_log2 cells per side, 1..13; 0 = choose automatically
                        (about 80 cells across the median polygon bounding box, clamped to 5..13) */
    int fp32_filter; /* 1: orientation in FP32 with exact int64 redo inside the error bound; 0: int64 only */
    int sub_log2;    /* a coarse cell cut by a polygon boundary is split into 2^sub_log2 x 2^sub_log2
                        fine cells, 1..3 (grid_log2 + sub_log2 <= 16); 0 = default (3) */
    int reserved[5]; /* must be zero */
} spx_index_params;

/*
 * Build the grid index of a polygon set (§4.2 canvas creation with conservative
 * rasterisation of the boundary; §4.3 boundary index).  Two levels: each cell
 * of a 2^g x 2^g coarse grid over the box is empty, wholly INSIDE exactly one
 * polygon, or mixed; a mixed cell is split into F x F fine cells (F =
 * 2^sub_log2), each of which is empty, INSIDE one polygon, or lists its
 * candidate polygons: INSIDE ones, and BOUNDARY ones with the polygon's edges
 * that can cross a rightward ray from a point of the fine cell (the exact test
 * runs on those).  A cell is INSIDE when no edge meets its open square and its
 * lower-left corner is inside.  params may be NULL (defaults: automatic grid,
 * FP32 filter on, sub_log2 3).  The index is built on the host (all cores) and
 * copied to the device; the polygon handle must stay alive while the index is
 * used.
 */
spx_status spx_build_index(spx_ctx *ctx, spx_polys polys, const spx_index_params *params, spx_index *out);

/*
 * The same index built on the device (§4.2 canvas creation; §6.1 builds the
 * index of query-time polygons on the fly, inside the query time): every
 * stage of the host build runs as kernels (per edge: conservative marks of
 * both levels and the corner thresholds of the rows it straddles; per row:
 * the parities that classify the cells no edge meets; per fine row: its edge
 * list sorted by right end; per cell: records, fine blocks and entries), and
 * the arrays are byte for byte those of spx_build_index with the same
 * parameters.  Same arguments, results and limits as spx_build_index.
 * Synchronous (the legacy default stream; the device is synchronised).
 * Temporary device memory is allocated and freed inside the call.  Errors:
 * SPX_EINVAL (bad handle or parameters, an index-format limit exceeded),
 * SPX_ENOMEM, SPX_ECUDA.
 */
spx_status spx_build_index_device(spx_ctx *ctx, spx_polys polys, const spx_index_params *params, spx_index *out);

/*
 * The arrays of a polygon index, copied to host memory (the layout of
 * spx_host_index_build, sentinels included): coarse words (sizes[0] uint32),
 * fine words (sizes[1] uint32), entries (sizes[2] x 4 uint32), edges
 * (sizes[3] x 4 int32).  Any output may be NULL (skipped); call with all NULL
 * to get the sizes.  Synchronous.  Errors: SPX_EINVAL (not a polygon index),
 * SPX_ECUDA.
 */
spx_status spx_index_arrays(spx_ctx *ctx, spx_index index, uint32_t *coarse, uint32_t *fine, uint32_t *entries,
                            int32_t *edges, uint64_t sizes[4]);

/*
 * Index of a set of disks for distance queries (§4.2 "Canvases for
 * Distance-Based Queries": a distance constraint around a point is a disk;
 * §5.2 "Distance-Based Queries": the pairs whose distance is <= r, one radius
 * per disk as in the paper's second distance join).  Disk q has centre
 * (cxy[2q], cxy[2q+1]) in [0, 2^30]^2 and radius r[q] in [0, 2^30); a point p
 * (in [0, 2^30)^2) is within it iff (px-cx)^2 + (py-cy)^2 <= r^2, decided
 * exactly.  The index is a 2^grid_log2 grid (0: about eight cells across the
 * median diameter); a cell wholly inside a disk needs no test.  The returned
 * index serves spx_join (pairs (point id, disk id) in that order, counts per
 * disk), spx_select (per-disk ascending point-id lists, at most 1024 disks)
 * and spx_aggregate; the other calls refuse it.  Host input, copied.
 * Errors: SPX_EINVAL (a centre or radius out of range, a grid too fine for the
 * number of entries), SPX_ENOMEM, SPX_ECUDA.
 */
spx_status spx_build_disk_index(spx_ctx *ctx, const int32_t *cxy, const int32_t *r, uint32_t Q, int grid_log2,
                                spx_index *out);

/*
 * The same index built on the GPU (the paper builds the indexes of
 * query-time constraints on the fly and counts that in query time, §6.1
 * "Database Setup and Tuning"; building it on the device keeps that cost small
 * for new query sets): every (cell, disk) pair of each disk's
 * bounding box is classified on the device, bucketed by cell, and the lists
 * laid out in cell order and sorted by disk, so the cell words, entries and
 * cover bitmap are byte for byte those of spx_build_disk_index (see
 * spx_disk_index_arrays).  Same arguments, checks, grid choice and errors;
 * the build synchronises the device.  It allocates temporaries of about
 * 20 B per cell of the 4^grid_log2 grid plus 8 B per (cell, disk) record.
 */
spx_status spx_build_disk_index_device(spx_ctx *ctx, const int32_t *cxy, const int32_t *r, uint32_t Q,
                                       int grid_log2, spx_index *out);

/*
 * Copies a disk index's arrays to host memory for inspection: sizes[0] = cell
 * words (4^grid_log2), sizes[1] = entry words, sizes[2] = grid_log2; cell and
 * entries (uint32, those sizes) may be NULL to query the sizes.  Layout as
 * described for spx_host_disk_index_build.  Synchronous.  Errors: SPX_EINVAL
 * (not a disk index), SPX_ECUDA.
 */
spx_status spx_disk_index_arrays(spx_ctx *ctx, spx_index index, uint32_t *cell, uint32_t *entries,
                                 uint64_t sizes[3]);

/* Sizes of a built index. */
typedef struct {
    int grid_log2;
    int sub_log2;
    uint32_t n_polys;
    uint32_t pad;
    uint64_t n_cells;        /* 4^grid_log2 coarse cells */
    uint64_t n_blocks;       /* mixed coarse cells (each holds 4^sub_log2 fine cells) */
    uint64_t n_entries;      /* list entries stored for fine cells */
    uint64_t n_inside;       /* (coarse cell, polygon) pairs wholly inside */
    uint64_t n_mixed;        /* (coarse cell, polygon) pairs split into fine cells */
    uint64_t n_boundary;     /* (fine cell, polygon) pairs that run the exact test */
    uint64_t n_edge_refs;    /* edges stored in per-fine-row edge lists */
    uint64_t device_bytes;   /* device memory held by the index */
    double build_ms;         /* host build + upload time */
    double sum_resolved;     /* fraction of the coarse level's block summary (2^min(g,8) blocks per side)
                                that is empty or INSIDE one polygon */
    int use_sum;             /* 1: join pass 1a reads the block summary from shared memory */
    int pad2;
    int edge_grid_log2;      /* buffered polygons: 2^edge_grid_log2 edge-grid cells per side; else 0 */
    int pad3;
    uint64_t n_edge_items;   /* buffered polygons: (cell, edge) entries of the edge grid; else 0 */
} spx_index_info;

spx_status spx_index_info_get(spx_ctx *ctx, spx_index index, spx_index_info *out);

/*
 * Index of a set of buffered polygons for distance queries (§4.2 "Canvases
 * for Distance-Based Queries": the constraint of distance r around a polygon
 * is the polygon together with a rounded rectangle of radius r around each of
 * its edges; §5.2 "Distance-Based Queries").  A point p (in [0, 2^30)^2)
 * meets polygon q of `polys` buffered by r[q] (in [0, 2^30)) iff p is inside
 * ring q (the crossing rule of spx_build_index) or within distance r[q] of one
 * of its edges taken as a closed segment (a ring of one vertex: a disk),
 * decided exactly (int64, and 128-bit products for the distance to an edge's
 * interior).  The index holds the polygons' own grid index (automatic grid,
 * fp32_filter as given) and an edge grid of 2^grid_log2 cells per side
 * (0: cells of about a quarter of the median radius, or of the median edge
 * length when the radii are 0, clamped to 5..12) that lists, per cell, the
 * edges whose r-neighbourhood may reach it, by polygon; a polygon whose
 * r-region holds the whole cell keeps one flagged item and its points need
 * no test, and a bitmap of the cells that list edges or meet a polygon lets
 * the other points leave after one lookup.
 * The returned index serves spx_join (pairs (point id, polygon id) in that
 * order, one per pair, counts per polygon), spx_select (at most 1024
 * polygons) and spx_aggregate; the other calls refuse it.  r: P host values,
 * copied.  The polygon handle must stay alive while the index is used.
 * Errors: SPX_EINVAL (bad handle, a radius out of range, grid_log2 outside
 * 0..12, an edge grid too large for 32-bit offsets), SPX_ENOMEM, SPX_ECUDA.
 */
spx_status spx_build_buffer_index(spx_ctx *ctx, spx_polys polys, const int32_t *r, int grid_log2, int fp32_filter,
                                  spx_index *out);

/* Autotuner settings.  Zero fields take the defaults. */
typedef struct {
    uint64_t sample_points; /* points of the sample; 0 = 1% of the table, but at least min(n, 2^22) */
    int grid_min;           /* smallest grid_log2 tried (default 6) */
    int grid_max;           /* largest grid_log2 tried (default 13) */
    int reps;               /* timed launches per candidate, the fastest kept (default 5) */
    int fp32_filter;        /* filter setting of every candidate and of the result: 1 (default) or 0 */
    uint64_t max_index_bytes; /* skip candidates whose index would exceed this (default 4 GiB) */
    int reserved[4];        /* must be zero */
} spx_tune_params;

/* One timed candidate. */
typedef struct {
    int grid_log2;
    int sub_log2;
    double ms;            /* fastest count-only launch over the sample */
    double build_ms;      /* host build + upload of the candidate's index */
    uint64_t device_bytes;
} spx_tune_trial;

/*
 * Choose the index resolution by timing (§6 "Database Setup and Tuning": the
 * paper fixes the cell size by a rule of thumb; §7 "Indexing Strategies and
 * Tuning" leaves automatic tuning open).  A deterministic sample (every
 * (n / m)-th point of `points`, m = the sample size) is copied once; then for
 * candidate (grid_log2, sub_log2) pairs the index of `polys` is built and the
 * count-only aggregate of the sample is timed (CUDA events on `stream`).
 * Search: grid_log2 rises from grid_min at the largest allowed sub_log2 and
 * stops after two candidates in a row that are not faster than the best; then
 * sub_log2 1..3 is tried at the best grid_log2.  The per-polygon counts of
 * every candidate are compared with the first: the resolution never changes a
 * result, and a mismatch fails the call with SPX_EKERNEL.
 *
 *   tp          settings (may be NULL: all defaults).
 *   best        receives the chosen grid_log2, sub_log2 and fp32_filter (reserved
 *               fields zero), ready for spx_build_index.
 *   trials      host array of max_trials records (may be NULL when max_trials
 *               is 0); *n_trials (may be NULL) receives the number of
 *               candidates timed, which can exceed max_trials (extra records
 *               are dropped).
 *   best_index  if not NULL, receives the chosen candidate's index (owned by
 *               the ctx; free it with spx_free); other candidates are freed.
 * Synchronises `stream`.  Needs device memory for the sample (8 B per point),
 * one index at a time and P counters.  Errors: SPX_EINVAL (bad handle, bad
 * settings, empty point table), SPX_ENOMEM, SPX_ECUDA, SPX_EKERNEL.
 */
spx_status spx_autotune(spx_ctx *ctx, spx_points points, spx_polys polys, const spx_tune_params *tp,
                        spx_index_params *best, spx_tune_trial *trials, uint32_t max_trials, uint32_t *n_trials,
                        spx_index *best_index, void *stream);

/*
 * Polygon-point join (§5.2 "Spatial Joins", Polygon x Point), one pass over the
 * points.  Output: every (point_id, polygon_id) with the point inside the
 * polygon, as uint32 pairs pairs_dev[2k] = point id, pairs_dev[2k+1] = polygon
 * id, sorted by point id then polygon id; counts_dev[q] (uint64, P entries,
 * may be NULL) = number of pairs with polygon q.  All device pointers.
 *   cap       capacity of pairs_dev in pairs; pairs past cap are not written.
 *   total_dev device uint64 that receives the total number of pairs (may be NULL).
 *   n_pairs   host uint64 (may be NULL).  If given, the call synchronises the
 *             stream, writes the total, and returns SPX_ECAPACITY if it
 *             exceeds cap (the first cap pairs are valid).
 * Without n_pairs the call is asynchronous and capture-safe once a first call
 * of at least this size has run on the ctx outside capture.
 */
spx_status spx_join(spx_ctx *ctx, spx_points points, spx_index index, uint32_t *pairs_dev, uint64_t cap,
                    uint64_t *counts_dev, uint64_t *total_dev, uint64_t *n_pairs, void *stream);

/*
 * Batched polygonal selection (§5.2 "Spatial Selection": the points inside a
 * polygonal constraint; here the P polygons of the index are P independent
 * query constraints answered in one pass over the points).  Output: for each
 * query q, the ascending ids of the points inside it, at
 * ids_dev[offsets_dev[q] .. offsets_dev[q+1]) (uint32 ids; offsets_dev holds
 * P + 1 uint64, offsets_dev[P] = total).  ids past cap are not written;
 * when the total exceeds cap, only offsets_dev[P] is meaningful.
 * n_ids (host, may be NULL): if given, the call synchronises, writes the total
 * and returns SPX_ECAPACITY if it exceeds cap.  At most 1024 query polygons
 * per index (SPX_EINVAL otherwise).
 * The first call with a given (points, index, ids_dev, cap, offsets_dev) runs
 * the passes directly and then captures them into a CUDA graph; later calls
 * with the same arguments replay that graph as one launch.  Graphs are
 * dropped when their points or index are freed or the ctx scratch grows.
 */
spx_status spx_select(spx_ctx *ctx, spx_points points, spx_index index, uint32_t *ids_dev, uint64_t cap,
                      uint64_t *offsets_dev, uint64_t *n_ids, void *stream);

/*
 * The same join through the plain comparison kernels: exact int64 orientation
 * only, one thread per point, a counting pass, a scan and a writing pass (the
 * two-pass Map of §5.1).  Same arguments and results as spx_join.
 */
spx_status spx_join_plain(spx_ctx *ctx, spx_points points, spx_index index, uint32_t *pairs_dev, uint64_t cap,
                          uint64_t *counts_dev, uint64_t *total_dev, uint64_t *n_pairs, void *stream);

/*
 * Allocation-free variant of spx_join_plain (the paper has no counterpart; it
 * exists for callers that cannot allocate device memory at call time: a
 * process whose device memory is held entirely by another allocator, such as
 * a framework's caching allocator, so cudaMalloc would fail; a latency-bound
 * request loop that cannot afford an allocator call, which may block and
 * synchronise the device; a deployment with a fixed device-memory budget
 * audited up front).  Same join, same results as spx_join_plain, with its
 * scratch in a fixed 512 KiB device array inside libspx instead of memory
 * from cudaMalloc; the call itself allocates nothing (the points, polygons
 * and index are loaded and built beforehand, and the caller passes the
 * outputs: pairs_dev, cap, counts_dev, total_dev as in spx_join_plain).
 *   - At most 16,777,216 points per call; a larger table is rejected with
 *     SPX_EINVAL and a message stating the limit.
 *   - Every GPU that loads libspx holds the 512 KiB array until the process
 *     exits.  All calls share it, and it keeps the last call's contents (the
 *     counting pass rewrites every value it later reads, so nothing needs
 *     clearing): calls whose kernels overlap on the GPU (different streams,
 *     different contexts in one process) race on it and corrupt each other's
 *     results; serialise them.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process: a device reset (cudaDeviceReset) between calls would leave it
 *     stale, so do not reset a device while libspx is in use on it.
 *   - Asynchronous on `stream`; no host out-parameter (read *total_dev).
 */
spx_status spx_join_plain_static(spx_ctx *ctx, spx_points points, spx_index index, uint32_t *pairs_dev,
                                 uint64_t cap, uint64_t *counts_dev, uint64_t *total_dev, void *stream);

/*
 * Count aggregation without materialising the join (§5.2 "Spatial
 * Aggregations", the plan for point data): counts_dev[q] (uint64, P entries,
 * device) = number of points inside polygon q.
 */
spx_status spx_aggregate(spx_ctx *ctx, spx_points points, spx_index index, uint64_t *counts_dev, void *stream);

/*
 * End-to-end join on host buffers: copies the n points at xy_host to the
 * device, joins them against the index, and returns pairs and counts in host
 * memory.  pairs_host holds cap pairs (2*cap uint32), counts_host P uint64 (may
 * be NULL); *n_pairs receives the total (SPX_ECAPACITY if above cap; the first
 * cap pairs are written).  The table is processed in slices of 2^23 points so
 * that the copy of a slice to the device, the join of the previous slice and
 * the copy of the pairs of the one before back to the host overlap (the copies
 * run on the copy engines).  Device staging buffers are owned by the ctx and
 * reused.  Pinned host memory makes the copies faster.  Synchronous.
 */
spx_status spx_join_host(spx_ctx *ctx, const int32_t *xy_host, uint64_t n, spx_index index, uint32_t *pairs_host,
                         uint64_t cap, uint64_t *counts_host, uint64_t *n_pairs);

/*
 * Count aggregation over a point table in host memory (§5.2 "Spatial
 * Aggregations" over a table that need not fit in device memory, §5.3
 * "Out-of-Core Queries"): the n points at xy_host stream through four device
 * slots of one slice each (the copy of a slice overlaps the counting of the
 * slices before it); counts_host receives P uint64.  Device memory does not
 * grow with n.  Synchronous.  Errors: SPX_EINVAL, SPX_ENOMEM, SPX_ECUDA.
 */
spx_status spx_aggregate_host(spx_ctx *ctx, const int32_t *xy_host, uint64_t n, spx_index index, uint64_t *counts_host);

/*
 * How spx_join_host moves a host table (§5.3 out-of-core queries; §7 names
 * pipelining as future work): mode 1 stages the whole table and the pairs in
 * device memory; mode 2 streams the table through four device slots and has
 * the kernels write the pairs straight into pairs_host (the device must be able
 * to write it: pinned memory, or pageable memory on a system whose GPU uses the
 * host page tables; else spx_join_host returns SPX_EINVAL), so device memory
 * does not grow with n; mode 0 (the default) stages when the table, its
 * results and the pairs fit in half the free device memory, else streams.
 * slice_log2: points per slice, 16..26 (0: 2^23 for the join, 2^25 for
 * spx_aggregate_host, which always streams).  Applies to later calls on this ctx.
 */
spx_status spx_set_host_streaming(spx_ctx *ctx, int mode, int slice_log2);

/*
 * Host-only build of the same grid index, for inspection (no device, no ctx):
 * the index build runs on the host, so its output can be checked without a
 * GPU.  spx_host_index_build builds it (grid_log2 0 = automatic, sub_log2 0 =
 * default) and reports the array sizes: sizes[0] = coarse words, sizes[1] =
 * fine words, sizes[2] = entries, sizes[3] = edges, sizes[4] = grid_log2,
 * sizes[5] = sub_log2.  spx_host_index_copy copies the arrays into caller
 * buffers of those sizes (words: uint32; entries: 4 uint32 each; edges: 4
 * int32 each); free the handle with spx_host_index_free.  Layout:
 *   coarse word c = (cy << g) | cx: bits 31..30 kind (0 none, 1 one INSIDE
 *     polygon = bits 29..0, 2 mixed: block b = bits 29..0);
 *   fine word of mixed block b, fine cell (fx, fy) = fine[b * F*F + (fy mod F)
 *     * F + (fx mod F)]: kind 0 none, 1 one INSIDE polygon, 2 list starting at
 *     entry bits 29..0;
 *   entry = (polygon id, first edge, edge count, flags: 1 BOUNDARY, 2 last);
 *   edge = (a.x, a.y, b.x, b.y); a BOUNDARY entry's edges are the polygon's
 *     non-horizontal edges meeting the fine cell's row strip with max x > the
 *     cell's left x, sorted by max x descending.
 */
typedef struct spx_host_index spx_host_index;
spx_status spx_host_index_build(const int32_t *xy, const uint64_t *ring_off, uint32_t P, int grid_log2,
                                int sub_log2, spx_host_index **out, uint64_t sizes[6]);
spx_status spx_host_index_copy(const spx_host_index *h, uint32_t *coarse, uint32_t *fine, uint32_t *entries,
                               int32_t *edges);
void spx_host_index_free(spx_host_index *h);

/*
 * Bounds check of a polygon index's arrays, as spx_host_index_build lays
 * them out (sizes in words / entries / edges, sentinels included): every
 * coarse word names a polygon below n_polys or a fine block that exists;
 * every fine word a polygon below n_polys or an entry list that ends with its
 * last entry before the four sentinel entries; every entry a polygon below
 * n_polys and an edge range inside the edge array (the sentinel edge
 * excluded).  spx_build_index applies it to every index before upload (a
 * failure there is SPX_EKERNEL); the kernels of a build with SPX_BOUNDS_CHECK
 * apply the same predicate to each offset they read.  SPX_OK, or SPX_EINVAL
 * with the first violation in msg (msg_len bytes, NUL-terminated; msg may be
 * NULL).  Host only; no device needed.
 */
spx_status spx_host_index_validate(const uint32_t *coarse, uint64_t n_coarse, const uint32_t *fine, uint64_t n_fine,
                                   const uint32_t *entries, uint64_t n_entries, const int32_t *edges,
                                   uint64_t n_edges, int grid_log2, int sub_log2, uint32_t n_polys, char *msg,
                                   uint64_t msg_len);

/*
 * Host-only build of the disk index of spx_build_disk_index (same arguments,
 * same checks), for inspection without a GPU.  sizes[0] = cell words (4^g),
 * sizes[1] = entry words, sizes[2] = grid_log2.  spx_host_disk_index_copy
 * copies the arrays into caller buffers of those sizes (uint32); free the
 * handle with spx_host_disk_index_free.  Layout: cell word c = (cy << g) | cx:
 * bits 31..30 kind (0 no disk reaches the cell; 1 the cell lies wholly inside
 * exactly one disk, id = bits 29..0, and no other disk reaches it; 2 list at
 * entry word bits 29..0); a list is n, then n words disk << 1 | boundary, in
 * disk order (boundary 0: the cell lies wholly inside that disk; 1: each point
 * takes the exact test).  Errors: SPX_EINVAL.
 */
typedef struct spx_host_disk_index spx_host_disk_index;
spx_status spx_host_disk_index_build(const int32_t *cxy, const int32_t *r, uint32_t Q, int grid_log2,
                                     spx_host_disk_index **out, uint64_t sizes[3]);
spx_status spx_host_disk_index_copy(const spx_host_disk_index *h, uint32_t *cell, uint32_t *entries);
void spx_host_disk_index_free(spx_host_disk_index *h);

/*
 * Host-only build of the edge grid of spx_build_buffer_index (P rings as for
 * spx_load_polygons, host radii r[P] in [0, 2^30), grid_log2 0..12 with 0
 * automatic), for inspection without a GPU.  sizes[0] = cell offsets
 * (4^g + 1), sizes[1] = items, sizes[2] = grid_log2.
 * spx_host_buffer_edges_copy copies the arrays into caller buffers: cell_off
 * (sizes[0] uint32; cell c = (cy << g) | cx holds items [cell_off[c],
 * cell_off[c + 1])), item_q (sizes[1] uint32: the polygon, ascending within a
 * cell; bit 31 set when the polygon's r-region holds every point of the cell,
 * the item then carrying no edge), item_seg (4 x sizes[1] int32: the edge's
 * ax, ay, bx, by; zero for a flagged item).  Free the handle with
 * spx_host_buffer_edges_free.  Errors: SPX_EINVAL.
 */
typedef struct spx_host_buffer_edges spx_host_buffer_edges;
spx_status spx_host_buffer_edges_build(const int32_t *xy, const uint64_t *ring_off, uint32_t P, const int32_t *r,
                                       int grid_log2, spx_host_buffer_edges **out, uint64_t sizes[3]);
spx_status spx_host_buffer_edges_copy(const spx_host_buffer_edges *h, uint32_t *cell_off, uint32_t *item_q,
                                      int32_t *item_seg);
void spx_host_buffer_edges_free(spx_host_buffer_edges *h);

/* Counters accumulated by the kernels of this ctx since the last reset, and
 * (with phase timing on) the device time of each pass, measured with CUDA
 * events on the caller's stream (the time breakdown of §6.2). */
typedef struct {
    uint64_t points_scanned;
    uint64_t edge_tests;       /* straddling-edge tests that needed an orientation */
    uint64_t fp32_escalations; /* of those, orientations redone in int64 because |d_f| <= E */
    uint64_t pairs_emitted;
    uint64_t timed_joins;      /* joins timed since the last reset */
    uint64_t timed_aggregates; /* aggregates timed since the last reset */
    double ms_resolve;         /* join pass 1 (distance join: all of it; polygon join: 1a, index lookups
                                  of every point, results and counts of points that need no exact test) */
    double ms_scan;            /* join pass 2: scan of per-tile pair totals */
    double ms_emit;            /* join pass 3: pairs written in point order */
    double ms_aggregate;       /* count-only aggregate */
    double ms_walk;            /* polygon join pass 1b: exact tests of the points whose cell lists edges */
    uint64_t points_from_directory; /* of points_scanned, those an aggregate over a clustered table counted
                                       from its cell directory without reading them */
} spx_stats_t;

/*
 * Checks the bounded-wait error path end to end (the join's pass 1a waits
 * for its bulk copies of points with at most a fixed number of polls): one
 * warp polls an mbarrier that nothing completes, `tries` times, then sets
 * the timeout bit of the ctx's error word, which the host reads and clears.
 * Returns SPX_ETIMEOUT (the expected result; the ctx stays usable) or
 * SPX_ECUDA.  Synchronises the stream.
 */
spx_status spx_check_bounded_wait(spx_ctx *ctx, uint32_t tries, void *stream);

/* Read (synchronising the device) and optionally reset the counters. */
spx_status spx_stats(spx_ctx *ctx, spx_stats_t *out, int reset);

/* Phase timing on (1) or off (0, the default).  While on, every join and
 * aggregate records CUDA events around its passes and synchronises the stream
 * after launching, to add the pass times to the counters. */
spx_status spx_set_phase_timing(spx_ctx *ctx, int on);

/* Release one handle (points, polygons or index).  An index must be freed
 * before the polygon set it was built from. */
spx_status spx_free(spx_ctx *ctx, uint64_t handle);

/* ------------------------------------------------------------------ serving
 *
 * A server answers a stream of selection and join requests against one
 * resident point table, on its own thread, with several requests in flight
 * (§7 "Improving I/O Performance" names pipelining as future work; the paper's
 * engine runs one query at a time).  Each batch goes through:
 *   1. a count pass over the points (§5.1 Map, first pass) that yields the exact
 *      size of every request's output,
 *   2. admission: the outputs are allocated once the server's output budget
 *      has room (device memory of results the caller still holds counts),
 *   3. the write pass, then (selections) the stable partition into per-query
 *      id lists.
 * Continuous batching: whenever a slot is free, the requests waiting at that
 * moment (up to max_batch, in arrival order) form one batch with one
 * admission.  By default each request's count and write passes are the join's
 * own kernels (spx_join's passes 1-3, its per-point results kept between the
 * passes in scratch the server takes from its pool per batch); with fused = 1,
 * every pass instead reads the point table once for the whole batch (§5.2's
 * one-pass batched selection, applied across requests), resolving each point
 * again in the write pass.  Requests that arrive later join the next free
 * slot; slots overlap on the device (one CUDA stream each).
 * Results are byte-identical to spx_join / spx_select on the same index,
 * whatever the batch composition.
 *
 * Thread safety: every spx_server_* call may come from any thread.  The ctx,
 * the point table and the listed indexes must stay alive and unchanged until
 * spx_server_destroy returns; the ctx may be used meanwhile (on its own
 * thread) for anything but freeing them.
 */
typedef struct spx_server spx_server;

typedef struct {
    int max_batch;          /* requests admitted together, 1..8 (0 = 8; 1 = no batching) */
    int slots;              /* batches in flight, 1..4 (0 = 2) */
    int plain;              /* 1: comparison mode: each request alone (max_batch = slots = 1) through the
                               plain kernels (int64 only, one thread per point, not persistent) */
    int fused;              /* 0: every request of a batch through the join's own passes (count pass of
                               each, one admission, write pass of each); 1: one fused pass over the
                               points for the whole batch (per-request lookups, no cached results) */
    uint64_t output_budget; /* device bytes of outputs and temporaries held at once; 0 = half of the free
                               device memory at creation.  A batch larger than the budget runs alone. */
    int reserved[4];        /* must be zero */
} spx_server_params;

enum { SPX_REQ_SELECT = 1, SPX_REQ_JOIN = 2 };

typedef struct {
    int kind;       /* SPX_REQ_SELECT: per-query ascending point-id lists (at most 1024 polygons);
                       SPX_REQ_JOIN: (point, polygon) pairs sorted by point then polygon, and counts */
    uint32_t index; /* position of the request's index in the list given to spx_server_create */
    uint64_t tag;   /* caller's value, returned in the result */
} spx_request;

typedef struct {
    int status;                  /* SPX_OK, or this request's error */
    int kind;
    uint64_t tag;
    uint64_t total;              /* pairs (join) or ids (selection) */
    uint32_t n_polys;            /* polygons of the request's index */
    uint32_t batch_size;         /* requests answered by the same passes */
    const uint32_t *pairs_dev;   /* join: 2 * total uint32 (point id, polygon) pairs; else NULL */
    const uint64_t *counts_dev;  /* join: n_polys counts; else NULL */
    const uint32_t *ids_dev;     /* selection: total point ids, query-major, ascending per query; else NULL */
    const uint64_t *offsets_dev; /* selection: n_polys + 1 list starts; else NULL */
    double t_submit_ms;          /* server clock (ms since creation): submission */
    double t_start_ms;           /* the batch's first launch */
    double t_done_ms;            /* results complete on the device (stream callback) */
    double t_counted_ms;         /* the batch's count pass complete on the device (stream callback) */
    double t_written_ms;         /* outputs admitted and the write pass launched */
} spx_result;

typedef struct {
    uint64_t submitted, completed, failed, batches;
    uint64_t batched_requests;   /* sum of batch sizes */
    uint64_t bytes_in_use;       /* outputs held (not yet released) plus temporaries */
    uint64_t peak_bytes_in_use;
    uint64_t admission_waits;    /* batches that waited for budget */
} spx_server_stats_t;

/*
 * Create a server on ctx's device over `points` and the n_indexes indexes
 * (requests name them by position).  params may be NULL (defaults).  Starts
 * the server thread.  Errors: SPX_EINVAL (bad handle or parameter), SPX_ENOMEM,
 * SPX_ECUDA.
 */
spx_status spx_server_create(spx_ctx *ctx, spx_points points, const spx_index *indexes, uint32_t n_indexes,
                             const spx_server_params *params, spx_server **out);

/* Queue one request; *req_id receives its id.  SPX_EINVAL for a bad kind or
 * index position, or a selection index of more than 1024 polygons. */
spx_status spx_server_submit(spx_server *srv, const spx_request *req, uint64_t *req_id);

/*
 * Queue one request that brings its own polygons (P rings as for
 * spx_load_polygons; host arrays, copied before the call returns) instead of
 * naming a prebuilt index.  Their grid index is built on the device when the
 * request's batch starts (one level coarser than the automatic grid of
 * spx_build_index, at least 5; sub_log2 3; FP32 filter on), so its
 * build time is part of the request's latency (§6.1 counts the index built
 * for query polygons in the query time; the build runs on the batch's own
 * stream, memory from the server's pool); its memory counts against the
 * output budget and goes back to the pool after the request's write pass.  The result is the
 * same as for a prebuilt index of those polygons.  SPX_EINVAL for a bad kind,
 * a selection of more than 1024 polygons, a vertex outside [0, 2^30]^2, bad
 * ring offsets or more than 2^32 - 1 vertices.
 */
spx_status spx_server_submit_polygons(spx_server *srv, int kind, const int32_t *xy, const uint64_t *ring_off,
                                      uint32_t P, uint64_t tag, uint64_t *req_id);

/* Result of a request: SPX_EBUSY while it is pending, SPX_EINVAL for an
 * unknown (or released) id; otherwise fills *out and returns SPX_OK (the
 * request's own status is out->status). */
spx_status spx_server_poll(spx_server *srv, uint64_t req_id, spx_result *out);

/* As spx_server_poll, waiting up to timeout_ms (< 0: without limit). */
spx_status spx_server_wait(spx_server *srv, uint64_t req_id, double timeout_ms, spx_result *out);

/* Give back a finished request's device buffers (its result pointers become
 * invalid).  SPX_EBUSY while it is pending, and while a spx_server_read of it
 * runs on another thread (the buffers are freed only once no read copies
 * them; call again after the read returns). */
spx_status spx_server_release(spx_server *srv, uint64_t req_id);

/* Copy a finished request's result to host memory (synchronous): a join's
 * pairs (8 * total bytes) to `a` and counts (8 * n_polys) to `b`; a selection's
 * ids (4 * total) to `a` and offsets (8 * (n_polys + 1)) to `b`.  a_bytes /
 * b_bytes are the buffers' sizes: SPX_ECAPACITY if one is too small, nothing
 * copied.  Either buffer may be NULL (skipped).  A release of the same
 * request on another thread while the copy runs returns SPX_EBUSY and frees
 * nothing.  SPX_EBUSY while pending. */
spx_status spx_server_read(spx_server *srv, uint64_t req_id, void *a, uint64_t a_bytes, void *b, uint64_t b_bytes);

spx_status spx_server_stats(spx_server *srv, spx_server_stats_t *out);

/* Text of the last error of a server call (never NULL). */
const char *spx_server_last_error(spx_server *srv);

/* Finish every queued and running request, stop the thread and free every
 * buffer, released or not.  Safe on NULL. */
void spx_server_destroy(spx_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* SPX_H */
