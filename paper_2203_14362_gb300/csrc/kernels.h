// Launch wrappers of libspx's kernels (internal; called from api.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace spx {

struct IndexView {
    const uint32_t *cell; // 4^g coarse words
    const uint32_t *fine; // blocks of 4^sub fine words
    const uint4 *ent;     // entries
    const int4 *edge;     // per-fine-row edge lists
    int sc;               // coarse shift: 30 - g
    int gc;               // g
    int sf;               // fine shift: 30 - g - sub
    int sb;               // sub
    uint32_t P;           // number of polygons
    const uint32_t *cover; // 4^cg bits: cover cell holds a non-empty coarse cell
    int scv;              // cover shift: 30 - cg
    int cg;               // cover grid log2: min(g, kCoverLog2)
    // Block summary of the coarse level: one 16-bit word per block of a
    // 2^sg x 2^sg grid (sg = min(g, kSumLog2)), row-major, 8 per uint4:
    // kSumEmpty (no coarse cell of the block can hold a polygon), kSumMixed
    // (look the coarse word up), or q < kSumEmpty (every coarse cell of the
    // block lies INSIDE polygon q and no other).  Read from shared memory by
    // join pass 1a when use_sum is set.
    const uint4 *sum;
    int ssh;              // summary shift: 30 - sg
    int sg;               // summary grid log2
    int use_sum;          // the summary resolves enough of the box to be worth its shared memory
    // array sizes (sentinels included) and the error word, for the bounds
    // checks of a build with SPX_BOUNDS_CHECK
    uint64_t n_fine, n_ent, n_edge;
    unsigned *err;
};
constexpr int kCoverLog2 = 8;
constexpr int kSumLog2 = 8;
constexpr uint32_t kSumMixed = 0xffffu;
constexpr uint32_t kSumEmpty = 0xfffeu;

// A grid index of disks (distance queries): cell words as the coarse level of
// IndexView; lists in ent (n, then n words disk << 1 | boundary); disks as
// (cx, cy, r, 0); the cover bitmap as in IndexView (4^cg bits, at least one
// word).
struct DiskView {
    const uint32_t *cell;
    const uint32_t *ent;
    const int4 *disk;
    const uint32_t *cover;
    int sc; // 30 - g
    int g;
    uint32_t Q;
    int scv; // 30 - cg
    int cg;  // min(g, kCoverLog2)
};

struct DiskLaunch {
    DiskView dv;
    const int2 *pts;
    uint64_t n;
    uint2 *pairs; // may be null when cap == 0
    uint64_t cap;
    unsigned long long *counts; // Q entries or null; zeroed by the launchers
    unsigned long long *total;  // device total or null
    unsigned long long *stats;
};

// Distance join: pairs (point, disk) with distance <= r, in (point, disk)
// order, counts, total.  scratch: disk_scratch_bytes(n).  ev (or null): four
// events recorded before pass 1, before the scan, before pass 3 and after it.
size_t disk_scratch_bytes(uint64_t n);
cudaError_t launch_disk_join(const DiskLaunch &a, void *scratch, cudaStream_t s, cudaEvent_t *ev);
// Counts only.
cudaError_t launch_disk_aggregate(const DiskLaunch &a, cudaStream_t s);
// Per-disk ascending point-id lists (the selection); scratch:
// disk_select_scratch_bytes(n, Q, cap).
size_t disk_select_scratch_bytes(uint64_t n, uint32_t Q, uint64_t cap);
cudaError_t launch_disk_select(const DiskLaunch &a, uint32_t *ids, uint64_t cap, unsigned long long *offsets,
                               void *scratch, cudaStream_t s);

// Buffered polygons (SPADE §4.2 distance canvases: a polygon plus a rounded
// rectangle of radius r around each edge): the polygon index answers
// containment, an edge grid the distance part.
struct BufferView {
    const uint32_t *cell_off; // 4^g + 1 item offsets per edge-grid cell
    const uint32_t *item_q;   // polygon of each item, ascending within a cell
    const int4 *item_seg;     // the item's edge (ax, ay, bx, by)
    const int32_t *rad;       // P radii, each in [0, 2^30)
    const uint32_t *mask;     // a bit per cell: it lists edges or meets a non-empty cell of the polygon index
    int g, sc;                // 2^g cells per side of 2^sc units
    uint32_t P;
    uint64_t n_items;
};

struct BufferLaunch {
    IndexView ix; // the polygons' own index (containment)
    BufferView bv;
    const int2 *pts;
    uint64_t n;
    uint2 *pairs; // may be null when cap == 0
    uint64_t cap;
    unsigned long long *counts; // P entries or null; zeroed by the launchers
    unsigned long long *total;  // device total or null
    unsigned long long *stats;
    int fp32;
};

// Buffered-polygon join: pairs (point, polygon) of the points inside the
// polygon or within its radius of one of its edges, in (point, polygon)
// order, counts, total; scratch: buffer_scratch_bytes(n).
size_t buffer_scratch_bytes(uint64_t n);
cudaError_t launch_buffer_join(const BufferLaunch &a, void *scratch, cudaStream_t s);
// Counts only.
cudaError_t launch_buffer_aggregate(const BufferLaunch &a, cudaStream_t s);
// Per-polygon ascending point-id lists; scratch: buffer_select_scratch_bytes(n, P, cap).
size_t buffer_select_scratch_bytes(uint64_t n, uint32_t P, uint64_t cap);
// ORs into mask (a bit per cell of a 2^g grid) every cell that meets a
// non-empty coarse cell of polygon index ix.
cudaError_t launch_buffer_mask(const IndexView &ix, uint32_t *mask, int g, cudaStream_t s);
cudaError_t launch_buffer_select(const BufferLaunch &a, uint32_t *ids, uint64_t cap, unsigned long long *offsets,
                                 void *scratch, cudaStream_t s);

// Device build of the disk index of Q disks (host array of (cx, cy, r, 0),
// already checked) on a 2^g grid: the same cell words and entries as the host
// build (build_disk_index) and the same cover bitmap, in one new device
// allocation laid out as the host path lays it out (cells | entries | disks |
// cover, each part 256-byte aligned); the caller owns out.mem.  Runs on the
// legacy default stream and synchronises the device.  Returns 0, 1 when the
// entries would not fit 30-bit offsets (use a coarser grid), or 2 on a CUDA
// error (in cerr).
struct DiskIndexDev {
    void *mem;
    size_t bytes;
    uint32_t *cell, *ent, *cover;
    int4 *disk;
    uint64_t n_ent, n_inside, n_boundary;
};
int build_disk_index_device(const int4 *disks_host, uint32_t Q, int g, DiskIndexDev &out, cudaError_t &cerr);

// Device status word bits (ORed into the ctx's persistent error word).
constexpr unsigned kErrTimeout = 1u;   // a bounded wait (for a bulk copy) gave up
constexpr unsigned kErrInternal = 2u;  // a bounds check of an index walk failed (SPX_BOUNDS_CHECK builds)

// Per-ctx device counters, in this order.
enum { kStatPoints = 0, kStatTests = 1, kStatEscalations = 2, kStatPairs = 3, kStatDirPoints = 4, kStatCount = 5 };

struct JoinLaunch {
    IndexView ix;
    const int2 *pts;
    uint64_t n;
    uint2 *pairs;                 // may be null when cap == 0
    uint64_t cap;
    unsigned long long *counts;   // P entries or null; zeroed by the launcher
    unsigned long long *total;    // device total or null
    uint32_t *res;                // join pass 1 -> 3: per-point result (scratch)
    unsigned long long *tile_tot; // join: per-chunk pair totals, then offsets (scratch)
    unsigned *err;                // persistent error word
    unsigned long long *stats;    // kStatCount counters
    int fp32;
    // chunked joins (a slice of a larger table): point ids are pid0 + row;
    // pair offsets start at *pair_base (device, null: 0); keep_counts: counts
    // are not zeroed (they accumulate over the slices)
    uint32_t pid0;
    int keep_counts;
    const unsigned long long *pair_base;
    int clustered;  // the points are grouped by cell: lanes of a warp mostly share a polygon
    // count aggregate over a cell-clustered table with its directory (cell k's
    // points are rows [k ? cell_end[k - 1] : 0, cell_end[k]) of a 2^cluster_log2
    // grid, then one bin of points outside the box); used when cluster_log2 >= g
    const unsigned long long *cell_end;
    int cluster_log2;
    // set by launch_join: the per-point results of passes 1 -> 3 are 16-bit
    // words (the index has at most kRes16MaxP polygons)
    int narrow;
    // with narrow results, or null: a word per point where pass 1b packs the
    // polygons (four 16-bit ids, ascending) of a point in two to four of
    // them, so that pass 3 writes its pairs without walking its list again
    uint64_t *aux;
};

// Largest polygon count whose join keeps 16-bit per-point results.
constexpr uint32_t kRes16MaxP = 0xfffeu;

// Scratch bytes the join needs for n points (per-point results, tile totals, counter).
size_t join_scratch_bytes(uint64_t n);
size_t plain_scratch_bytes(uint64_t n);

// scratch: device memory of join_scratch_bytes(n) bytes.  ev (may be null):
// five events recorded before pass 1, after pass 1a (resolve), after pass 1b
// (walk), after pass 2 (scan) and after pass 3 (emit).
cudaError_t launch_join(const JoinLaunch &a, void *scratch, cudaStream_t s, cudaEvent_t *ev = nullptr);
// launch_join in two halves over the same scratch, for callers that size the
// output between them: passes 1 and 2 (counts, per-point results, offsets,
// *a.total; ev as for launch_join, first three events), then pass 3 (pairs).
cudaError_t launch_join_count(const JoinLaunch &a, void *scratch, cudaStream_t s, cudaEvent_t *ev = nullptr);
cudaError_t launch_join_write(const JoinLaunch &a, void *scratch, cudaStream_t s);
cudaError_t launch_join_plain(const JoinLaunch &a, void *scratch, cudaStream_t s);
// scratch: aggregate_scratch_bytes(a) bytes (the chunk bitmap of the directory
// path; unused otherwise).  a.keep_counts: add to the counts instead of
// zeroing them first.
size_t aggregate_scratch_bytes(const JoinLaunch &a);
cudaError_t launch_aggregate(const JoinLaunch &a, void *scratch, cudaStream_t s, cudaEvent_t *ev = nullptr);

// Batched selection: per-query ascending point-id lists in ids (cap entries),
// offsets[q] / offsets[P] (device, P + 1 values; offsets[P] = total).  At most
// 1024 queries per index.  scratch: select_scratch_bytes(n, P, cap).
size_t select_scratch_bytes(uint64_t n, uint32_t P, uint64_t cap);
cudaError_t launch_select(const JoinLaunch &a, uint32_t *ids, uint64_t cap, unsigned long long *offsets,
                          void *scratch, cudaStream_t s);
constexpr uint32_t kSelectMaxQueries = 1024;

// Stable partition of (point, query) pairs (point order) by query: ids[] gets
// the point ids of query 0, then of query 1, ..., offsets[] (P + 1 values) the
// list starts.  Reads min(*total, cap) pairs.  scratch: partition_scratch_bytes.
size_t partition_scratch_bytes(uint64_t cap, uint32_t P);
cudaError_t launch_partition(const uint2 *pairs, const unsigned long long *total, uint64_t cap, uint32_t P,
                             uint32_t *ids, unsigned long long *offsets, void *scratch, cudaStream_t s);

// Several requests, each with its own index, answered in one pass over the
// points (serving).  At most kMaxBatch requests; their polygons together are
// counted in shared memory when qbase[K] <= kMultiHistMax, else with global
// atomics.
constexpr int kMaxBatch = 8;
constexpr uint32_t kMultiHistMax = 11776;

struct MultiLaunch {
    IndexView ix[kMaxBatch];
    uint32_t qbase[kMaxBatch + 1];           // prefix sums of the requests' polygon counts
    unsigned long long *counts[kMaxBatch];   // per request: P counters (or null); zeroed by the count launcher
    uint2 *pairs[kMaxBatch];                 // per request: (point, polygon) pairs, point order (emit pass)
    uint64_t cap[kMaxBatch];                 // capacity of pairs[r]
    unsigned long long *totals;              // K device totals, written by the count launcher
    const int2 *pts;
    uint64_t n;
    int K;
    int fp32;
    unsigned *err;
    unsigned long long *stats;
};

// scratch of one batch (per-request tile totals / offsets and scan partials),
// shared by the count and emit launches of that batch.
size_t multi_scratch_bytes(uint64_t n, int K);
// Pass 1 + scans: per-polygon counts and the K totals (m.totals).
cudaError_t launch_multi_count(const MultiLaunch &m, void *scratch, cudaStream_t s);
// Pass 2: every request's pairs in (point, polygon) order.
cudaError_t launch_multi_emit(const MultiLaunch &m, void *scratch, cudaStream_t s);

// The plain join (int64 only, one thread per point, not persistent) in two
// halves: count + device-wide scan (a.total), then write.  Same scratch.
size_t plain_split_scratch_bytes(uint64_t n);
cudaError_t launch_plain_count(const JoinLaunch &a, void *scratch, cudaStream_t s);
cudaError_t launch_plain_write(const JoinLaunch &a, void *scratch, cudaStream_t s);

// The join's passes as separate launches, for callers that pipeline slices of
// a table: a.res (4 B per point) and a.tile_tot (one u64 per
// join_chunk_points() points) are given by the caller.  resolve = pass 1 (1a
// and 1b) and the scan (*a.total = the slice's pair total; part:
// join_part_words(n) u64, for the row bitmap of pass 1 and the scan); emit =
// pass 3.
uint32_t join_chunk_points();
uint64_t join_part_words(uint64_t n);
cudaError_t launch_join_resolve(const JoinLaunch &a, unsigned long long *part, cudaStream_t s);
// pend: the row bitmap of pass 1 as pass 1b left it (needed when a.narrow).
cudaError_t launch_join_emit(const JoinLaunch &a, cudaStream_t s, const uint32_t *pend = nullptr);

// *dst = *x + *y (one thread; sliced joins chain their pair offsets).
cudaError_t launch_sum_u64(unsigned long long *dst, const unsigned long long *x, const unsigned long long *y,
                           cudaStream_t s);

// Copy of n points grouped by the cells of a 2^c x 2^c grid (row-major cells,
// points outside the box last; order within a cell unspecified), c in 1..13.
// scratch: cluster_scratch_bytes(c).
size_t cluster_scratch_bytes(int c);
cudaError_t launch_cluster(const int2 *pts, uint64_t n, int c, void *scratch, int2 *out, cudaStream_t s);

// dst[i] = src[i * (n / m)] for i < m (m <= n): the tuner's deterministic sample.
cudaError_t launch_gather_stride(const int2 *src, uint64_t n, int2 *dst, uint64_t m, cudaStream_t s);

int device_sm_count();

// One warp waits, at most `tries` polls, on an mbarrier that nothing completes,
// as pass 1a waits for its bulk copies, and sets kErrTimeout in *err.
cudaError_t launch_wait_check(unsigned *err, uint32_t tries, cudaStream_t s);

// Exclusive scan of n u64 values in place on stream s; *total (device, or
// null) gets their sum.  part: scan_part_words(n) u64 of scratch.
uint64_t scan_part_words(uint64_t n);
cudaError_t launch_exclusive_scan(unsigned long long *v, uint64_t n, unsigned long long *total,
                                  unsigned long long *part, cudaStream_t s);

// Device build of the polygon grid index: the same arrays as the host build
// (build_grid_index: coarse words, fine blocks, entries with their sentinels,
// edges with their sentinel), and the cover bitmap and block summary the
// host path computes from the coarse words, in one new device allocation laid
// out as the host path lays it out (cells | fine | entries | edges | cover |
// summary, each part 256-byte aligned); the caller owns out.mem.  xy (2 V
// int32) and ring_off (P + 1) are host arrays, already checked.  Runs on the
// legacy default stream and synchronises the device.  Returns 0; 1 when a
// limit of the index format is exceeded (err says which); 2 on a CUDA error
// (in cerr).
struct GridIndexDev {
    void *mem;
    size_t bytes;
    uint32_t *cell, *fine, *ent;
    int4 *edge;
    uint32_t *cover;
    uint16_t *sum;
    uint64_t n_cell, n_fine, n_ent, n_edge, n_blocks; // n_ent, n_edge with their sentinels
    uint64_t n_inside, n_mixed, n_boundary;
    double sum_resolved; // fraction of summary blocks that are empty or INSIDE one polygon
};
// s (or null: the legacy default stream, cudaMalloc, device-wide waits):
// every copy, kernel and allocation on stream s, memory from `pool` (or the
// device's default pool) with stream-ordered frees; out.mem must then be
// freed with cudaFreeAsync.
int build_grid_index_device(const int32_t *xy, const uint64_t *ring_off, uint32_t P, int g, int sb,
                            GridIndexDev &out, const char *&err, cudaError_t &cerr, cudaStream_t s = nullptr,
                            cudaMemPool_t pool = nullptr);

} // namespace spx
