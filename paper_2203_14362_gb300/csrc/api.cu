// C ABI of libspx (declared in include/spx.h): contexts, handles, argument
// checks, device memory of the index and the scratch, and dispatch to the
// kernels.  Every step of the join runs in kernels.cu; this file only moves
// bytes and checks arguments.
#include "kernels.h"
#include "server_internal.h"
#include "spx.h"
#include "spx_internal.h"

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <string>
#include <thread>
#include <vector>

using namespace spx;

#ifndef SPX_HOST_SLICE_LOG2
#define SPX_HOST_SLICE_LOG2 23 // points per slice of spx_join_host (a multiple of the join's chunk)
#endif

namespace {

enum : uint64_t { kTagPoints = 1, kTagPolys = 2, kTagIndex = 3 };
constexpr int kTagShift = 56;
// Least fraction of the block summary's blocks that must be resolved (empty or
// INSIDE one polygon) for join pass 1a to read it.
#ifndef SPX_SUM_MIN_RESOLVED
#define SPX_SUM_MIN_RESOLVED 0.33
#endif
constexpr double kSumMinResolved = SPX_SUM_MIN_RESOLVED;

struct PointsObj {
    int32_t *dev = nullptr;
    uint64_t n = 0;
    bool owned = false;
    int cluster_log2 = 0; // > 0: a cell-clustered copy (point order is not row order)
    unsigned long long *cell_end = nullptr; // its directory: end row of every cell, then of the outside bin
};

struct PolysObj {
    std::vector<int32_t> xy;
    std::vector<uint64_t> off;
    uint32_t P = 0;
    int n_index = 0; // live indexes built from it
};

struct IndexObj {
    uint64_t polys = 0;
    int kind = 0;        // 0: polygons (view), 1: disks (dview), 2: buffered polygons (view and bview)
    DiskView dview{};
    BufferView bview{};
    void *mem2 = nullptr; // buffered polygons: edge grid (cell offsets | polygons | segments | radii)
    IndexView view{};
    int fp32 = 1;
    void *mem = nullptr; // one allocation: cells | fine | entries | edges | cover | summary
    uint64_t n_fine = 0, n_ent = 0, n_edge = 0; // words / entries / edges of a polygon index, sentinels included
    spx_index_info info{};
};

// Persistent per-ctx device words.
struct Aux {
    unsigned err;                       // kernel error bits, cleared when reported
    unsigned pad;
    unsigned long long stats[kStatCount];
    unsigned long long total;           // internal total when the caller passes none
};

} // namespace

struct spx_ctx {
    int device = 0;
    std::string err;
    uint64_t next_id = 1;
    std::map<uint64_t, std::unique_ptr<PointsObj>> points;
    std::map<uint64_t, std::unique_ptr<PolysObj>> polys;
    std::map<uint64_t, std::unique_ptr<IndexObj>> indexes;
    Aux *aux = nullptr;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    // staging buffers of spx_join_host
    void *st_pts = nullptr, *st_pairs = nullptr, *st_counts = nullptr;
    size_t st_pts_b = 0, st_pairs_b = 0, st_counts_b = 0;
    cudaStream_t stream = nullptr;
    // spx_join_host: copy-in, emit and copy-out streams, three events per
    // slice, pinned (base, total) words per slice
    cudaStream_t in_stream = nullptr, emit_stream = nullptr, out_stream = nullptr;
    std::vector<cudaEvent_t> slice_ev;
    unsigned long long *slice_words = nullptr;
    size_t slice_words_n = 0;
    int host_mode = 0;                          // 0 automatic, 1 staged, 2 streamed
    int host_slice_log2 = SPX_HOST_SLICE_LOG2;  // points per slice
    bool host_slice_set = false;                // set by the caller (else the aggregate takes 2^25)
    // batched selection: captured launch sequences, keyed by their arguments
    std::map<std::tuple<uint64_t, uint64_t, uintptr_t, uint64_t, uintptr_t>, cudaGraphExec_t> select_graphs;
    cudaStream_t capture_stream = nullptr;
    // phase timing
    bool timing = false;
    cudaEvent_t ev[5] = {};
    uint64_t timed_joins = 0, timed_aggs = 0;
    double ms_resolve = 0, ms_walk = 0, ms_scan = 0, ms_emit = 0, ms_agg = 0;
};

namespace {

spx_status fail(spx_ctx *c, spx_status s, const std::string &msg)
{
    if (c)
        c->err = msg;
    return s;
}

spx_status cuda_fail(spx_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, SPX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SPX_CUDA(call, what)                                                                                           \
    do {                                                                                                               \
        cudaError_t e_ = (call);                                                                                       \
        if (e_ != cudaSuccess)                                                                                         \
            return cuda_fail(ctx, e_, what);                                                                           \
    } while (0)

uint64_t make_handle(spx_ctx *c, uint64_t tag) { return (tag << kTagShift) | (c->next_id++); }

template <class T>
T *lookup(std::map<uint64_t, std::unique_ptr<T>> &m, uint64_t h)
{
    auto it = m.find(h);
    return it == m.end() ? nullptr : it->second.get();
}

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess)
        return false;
    return st != cudaStreamCaptureStatusNone;
}

// Grow a device buffer (never while the stream is being captured).
spx_status ensure(spx_ctx *ctx, void **buf, size_t *have, size_t need, cudaStream_t s, const char *what)
{
    if (*have >= need)
        return SPX_OK;
    if (capturing(s))
        return fail(ctx, SPX_EINVAL,
                    std::string(what) + ": scratch must be sized by a first call outside stream capture");
    if (*buf) {
        cudaStreamSynchronize(s);
        cudaFree(*buf);
        *buf = nullptr;
        *have = 0;
    }
    size_t sz = need < 256 ? 256 : need;
    if (buf == &ctx->scratch) {
        // captured selections point at the old scratch
        for (auto &kv : ctx->select_graphs)
            cudaGraphExecDestroy(kv.second);
        ctx->select_graphs.clear();
    }
    cudaError_t e = cudaMalloc(buf, sz);
    if (e != cudaSuccess)
        return fail(ctx, SPX_ENOMEM, std::string(what) + ": cudaMalloc failed: " + cudaGetErrorString(e));
    *have = sz;
    return SPX_OK;
}

// Read and clear the kernel error word (synchronises the stream).
spx_status check_kernel_err(spx_ctx *ctx, cudaStream_t s)
{
    SPX_CUDA(cudaStreamSynchronize(s), "stream synchronize");
    unsigned w = 0;
    SPX_CUDA(cudaMemcpy(&w, &ctx->aux->err, sizeof(w), cudaMemcpyDeviceToHost), "read error word");
    if (w) {
        SPX_CUDA(cudaMemset(&ctx->aux->err, 0, sizeof(unsigned)), "clear error word");
        if (w & kErrTimeout)
            return fail(ctx, SPX_ETIMEOUT, "a bounded device wait gave up; results of that call are invalid");
        return fail(ctx, SPX_EKERNEL, "kernel reported an internal error");
    }
    return SPX_OK;
}

// Cover bitmap of a 2^g x 2^g grid of cell words: one bit per block of
// cells of a 2^cg x 2^cg grid (cg = min(g, kCoverLog2)), set when any cell of
// the block is not empty.
std::vector<uint32_t> cover_bitmap(const uint32_t *cell, int g)
{
    const int cg = std::min(g, kCoverLog2);
    std::vector<uint32_t> cover(std::max<size_t>((size_t(1) << (2 * cg)) / 32, 1), 0u);
    for (uint32_t cy = 0; cy < (1u << g); ++cy)
        for (uint32_t cx = 0; cx < (1u << g); ++cx)
            if ((cell[(size_t(cy) << g) | cx] >> 30) != kCellEmpty) {
                const uint32_t b = ((cy >> (g - cg)) << cg) | (cx >> (g - cg));
                cover[b >> 5] |= 1u << (b & 31);
            }
    return cover;
}

// Block summary of a 2^g x 2^g grid of coarse words on a 2^sg x 2^sg grid
// (sg = min(g, kSumLog2)): per block kSumEmpty when every cell is empty, q
// when every cell is INSIDE exactly polygon q (q < kSumEmpty), else
// kSumMixed.  *resolved: the fraction of blocks that are not mixed.
std::vector<uint16_t> block_summary(const uint32_t *cell, int g, double *resolved)
{
    const int sg = std::min(g, kSumLog2), sh = g - sg;
    const uint32_t nb = 1u << sg;
    std::vector<uint16_t> sum(size_t(nb) * nb);
    uint64_t n_res = 0;
    for (uint32_t by = 0; by < nb; ++by)
        for (uint32_t bx = 0; bx < nb; ++bx) {
            const uint32_t w0 = cell[(size_t(by << sh) << g) | (bx << sh)];
            bool same = (w0 >> 30) == kCellEmpty || ((w0 >> 30) == kCellInsideOne && (w0 & kPayloadMask) < kSumEmpty);
            for (uint32_t cy = by << sh; same && cy < ((by + 1) << sh); ++cy)
                for (uint32_t cx = bx << sh; same && cx < ((bx + 1) << sh); ++cx)
                    same = cell[(size_t(cy) << g) | cx] == w0;
            const uint16_t v = !same ? uint16_t(kSumMixed)
                                     : (w0 >> 30) == kCellEmpty ? uint16_t(kSumEmpty) : uint16_t(w0 & kPayloadMask);
            sum[size_t(by) * nb + bx] = v;
            n_res += same ? 1 : 0;
        }
    *resolved = double(n_res) / double(sum.size());
    return sum;
}

// Adds the phases of the join just launched to the totals: a polygon join
// recorded five events (pass 1a, pass 1b, scan, emit), a distance join four
// (pass 1, scan, emit).
spx_status add_phase_times(spx_ctx *ctx, bool polygons)
{
    const int last = polygons ? 4 : 3;
    SPX_CUDA(cudaEventSynchronize(ctx->ev[last]), "join timing");
    float t[4] = {0, 0, 0, 0};
    for (int k = 0; k < last; ++k)
        cudaEventElapsedTime(&t[k], ctx->ev[k], ctx->ev[k + 1]);
    ctx->ms_resolve += t[0];
    if (polygons)
        ctx->ms_walk += t[1];
    ctx->ms_scan += t[last - 2];
    ctx->ms_emit += t[last - 1];
    ctx->timed_joins++;
    return SPX_OK;
}

// The distance join (a disk index): same contract as the polygon join.
spx_status disk_join_common(spx_ctx *ctx, PointsObj *pts, IndexObj *ix, uint32_t *pairs_dev, uint64_t cap,
                            uint64_t *counts_dev, uint64_t *total_dev, uint64_t *n_pairs, void *stream)
{
    if (cap && !pairs_dev)
        return fail(ctx, SPX_EINVAL, "join: pairs_dev is NULL with cap > 0");
    if ((reinterpret_cast<uintptr_t>(pairs_dev) & 7) || (reinterpret_cast<uintptr_t>(counts_dev) & 7) ||
        (reinterpret_cast<uintptr_t>(total_dev) & 7))
        return fail(ctx, SPX_EINVAL, "join: output pointers must be 8-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    spx_status st = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, disk_scratch_bytes(pts->n), s, "join");
    if (st != SPX_OK)
        return st;
    DiskLaunch a{};
    a.dv = ix->dview;
    a.pts = reinterpret_cast<const int2 *>(pts->dev);
    a.n = pts->n;
    a.pairs = reinterpret_cast<uint2 *>(pairs_dev);
    a.cap = pairs_dev ? cap : 0;
    a.counts = reinterpret_cast<unsigned long long *>(counts_dev);
    a.total = total_dev ? reinterpret_cast<unsigned long long *>(total_dev) : (n_pairs ? &ctx->aux->total : nullptr);
    a.stats = ctx->aux->stats;
    const bool timed = ctx->timing;
    cudaError_t e = launch_disk_join(a, ctx->scratch, s, timed ? ctx->ev : nullptr);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "join launch");
    if (timed && pts->n && (st = add_phase_times(ctx, false)) != SPX_OK)
        return st;
    if (n_pairs) {
        if ((st = check_kernel_err(ctx, s)) != SPX_OK)
            return st;
        unsigned long long t = 0;
        SPX_CUDA(cudaMemcpy(&t, a.total, sizeof(t), cudaMemcpyDeviceToHost), "read total");
        *n_pairs = t;
        if (t > cap)
            return fail(ctx, SPX_ECAPACITY, "join: " + std::to_string(t) + " pairs exceed capacity " +
                                                std::to_string(cap));
    }
    return SPX_OK;
}

BufferLaunch buffer_launch(spx_ctx *ctx, PointsObj *pts, IndexObj *ix)
{
    BufferLaunch a{};
    a.ix = ix->view;
    a.bv = ix->bview;
    a.pts = reinterpret_cast<const int2 *>(pts->dev);
    a.n = pts->n;
    a.stats = ctx->aux->stats;
    a.fp32 = ix->fp32;
    return a;
}

// The buffered-polygon join: same contract as the polygon join.
spx_status buffer_join_common(spx_ctx *ctx, PointsObj *pts, IndexObj *ix, uint32_t *pairs_dev, uint64_t cap,
                              uint64_t *counts_dev, uint64_t *total_dev, uint64_t *n_pairs, void *stream)
{
    if (cap && !pairs_dev)
        return fail(ctx, SPX_EINVAL, "join: pairs_dev is NULL with cap > 0");
    if ((reinterpret_cast<uintptr_t>(pairs_dev) & 7) || (reinterpret_cast<uintptr_t>(counts_dev) & 7) ||
        (reinterpret_cast<uintptr_t>(total_dev) & 7))
        return fail(ctx, SPX_EINVAL, "join: output pointers must be 8-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    spx_status st = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, buffer_scratch_bytes(pts->n), s, "join");
    if (st != SPX_OK)
        return st;
    BufferLaunch a = buffer_launch(ctx, pts, ix);
    a.pairs = reinterpret_cast<uint2 *>(pairs_dev);
    a.cap = pairs_dev ? cap : 0;
    a.counts = reinterpret_cast<unsigned long long *>(counts_dev);
    a.total = total_dev ? reinterpret_cast<unsigned long long *>(total_dev) : (n_pairs ? &ctx->aux->total : nullptr);
    cudaError_t e = launch_buffer_join(a, ctx->scratch, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "join launch");
    if (n_pairs) {
        if ((st = check_kernel_err(ctx, s)) != SPX_OK)
            return st;
        unsigned long long t = 0;
        SPX_CUDA(cudaMemcpy(&t, a.total, sizeof(t), cudaMemcpyDeviceToHost), "read total");
        *n_pairs = t;
        if (t > cap)
            return fail(ctx, SPX_ECAPACITY, "join: " + std::to_string(t) + " pairs exceed capacity " +
                                                std::to_string(cap));
    }
    return SPX_OK;
}

spx_status join_common(spx_ctx *ctx, spx_points points, spx_index index, uint32_t *pairs_dev, uint64_t cap,
                       uint64_t *counts_dev, uint64_t *total_dev, uint64_t *n_pairs, void *stream, bool plain)
{
    if (!ctx)
        return SPX_EINVAL;
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    PointsObj *pts = lookup(ctx->points, points);
    IndexObj *ix = lookup(ctx->indexes, index);
    if (!pts || !ix)
        return fail(ctx, SPX_EINVAL, "join: bad points or index handle");
    if (pts->cluster_log2)
        return fail(ctx, SPX_EINVAL, "join: a cell-clustered point table has no row order; use spx_aggregate");
    if (ix->kind == 1)
        return disk_join_common(ctx, pts, ix, pairs_dev, cap, counts_dev, total_dev, n_pairs, stream);
    if (ix->kind == 2)
        return buffer_join_common(ctx, pts, ix, pairs_dev, cap, counts_dev, total_dev, n_pairs, stream);
    if (cap && !pairs_dev)
        return fail(ctx, SPX_EINVAL, "join: pairs_dev is NULL with cap > 0");
    if ((reinterpret_cast<uintptr_t>(pairs_dev) & 7) || (reinterpret_cast<uintptr_t>(counts_dev) & 7) ||
        (reinterpret_cast<uintptr_t>(total_dev) & 7))
        return fail(ctx, SPX_EINVAL, "join: output pointers must be 8-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t need = plain ? plain_scratch_bytes(pts->n) : join_scratch_bytes(pts->n);
    spx_status st = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, need, s, "join");
    if (st != SPX_OK)
        return st;
    JoinLaunch a{};
    a.ix = ix->view;
    a.pts = reinterpret_cast<const int2 *>(pts->dev);
    a.n = pts->n;
    a.pairs = reinterpret_cast<uint2 *>(pairs_dev);
    a.cap = pairs_dev ? cap : 0;
    a.counts = reinterpret_cast<unsigned long long *>(counts_dev);
    a.total = total_dev ? reinterpret_cast<unsigned long long *>(total_dev) : (n_pairs ? &ctx->aux->total : nullptr);
    a.err = &ctx->aux->err;
    a.stats = ctx->aux->stats;
    a.fp32 = ix->fp32;
    const bool timed = ctx->timing && !plain;
    cudaError_t e = plain ? launch_join_plain(a, ctx->scratch, s) : launch_join(a, ctx->scratch, s, timed ? ctx->ev : nullptr);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "join launch");
    if (timed && pts->n && (st = add_phase_times(ctx, true)) != SPX_OK)
        return st;
    if (n_pairs) {
        st = check_kernel_err(ctx, s);
        if (st != SPX_OK)
            return st;
        unsigned long long t = 0;
        SPX_CUDA(cudaMemcpy(&t, a.total, sizeof(t), cudaMemcpyDeviceToHost), "read total");
        *n_pairs = t;
        if (t > cap)
            return fail(ctx, SPX_ECAPACITY, "join: " + std::to_string(t) + " pairs exceed capacity " +
                                                std::to_string(cap));
    }
    return SPX_OK;
}

// Scratch of the allocation-free plain join (spx_join_plain_static): one
// uint64 block total per 256-point block of the counting pass, 512 KiB in all.
// It is a file-scope device array, so every GPU that loads this library holds
// it until the process exits; every call shares it.
constexpr uint64_t kStaticJoinMaxPoints = uint64_t(1) << 24;
constexpr uint64_t kStaticJoinBlocks = kStaticJoinMaxPoints / 256;
static __device__ __align__(256) unsigned long long g_static_join_scratch[kStaticJoinBlocks + 2];

// Device address of g_static_join_scratch, resolved once per device (host
// code cannot use the array's name as a device address).
void *static_join_scratch(int device, cudaError_t &err)
{
    static std::mutex mu;
    static void *addr[64] = {};
    err = cudaSuccess;
    if (device < 0 || device >= 64) {
        err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        err = cudaGetSymbolAddress(&p, g_static_join_scratch);
        if (err != cudaSuccess)
            return nullptr;
        addr[device] = p;
    }
    return addr[device];
}

// The parts of a polygon index's device allocation (cells | fine | entries |
// edges | cover | summary) and its statistics, for register_grid_index.
struct GridParts {
    char *cell, *fine, *ent, *edge, *cover, *sum;
    uint64_t n_cell, n_fine, n_ent, n_edge, n_blocks, n_inside, n_mixed, n_boundary;
    double sum_resolved;
};

// Views and info of a polygon index whose allocation ix->mem holds `gp`;
// takes the index into the ctx and returns its handle.
// The kernels' view of a polygon index whose arrays are `gp`.
static IndexView grid_view(const GridParts &gp, int g, int sb, uint32_t P)
{
    IndexView v{};
    const int cg = std::min(g, kCoverLog2);
    v.cell = reinterpret_cast<const uint32_t *>(gp.cell);
    v.fine = reinterpret_cast<const uint32_t *>(gp.fine);
    v.ent = reinterpret_cast<const uint4 *>(gp.ent);
    v.edge = reinterpret_cast<const int4 *>(gp.edge);
    v.sc = kBoxLog2 - g;
    v.gc = g;
    v.sf = kBoxLog2 - g - sb;
    v.sb = sb;
    v.P = P;
    v.cover = reinterpret_cast<const uint32_t *>(gp.cover);
    v.scv = kBoxLog2 - cg;
    v.cg = cg;
    v.sum = reinterpret_cast<const uint4 *>(gp.sum);
    v.sg = std::min(g, kSumLog2);
    v.ssh = kBoxLog2 - v.sg;
    // the summary costs pass 1a three quarters of its warps per SM (one CTA
    // holds it); worth it when it answers a third of the box or more
    v.use_sum = gp.sum_resolved >= kSumMinResolved ? 1 : 0;
    v.n_fine = gp.n_fine;
    v.n_ent = gp.n_ent;
    v.n_edge = gp.n_edge;
    return v;
}

static GridParts device_parts(const GridIndexDev &d)
{
    char *base = static_cast<char *>(d.mem);
    auto at = [&](const void *p) { return base + (static_cast<const char *>(p) - base); };
    return GridParts{at(d.cell), at(d.fine), at(d.ent), at(d.edge), at(d.cover), at(d.sum), d.n_cell, d.n_fine,
                     d.n_ent, d.n_edge, d.n_blocks, d.n_inside, d.n_mixed, d.n_boundary, d.sum_resolved};
}

spx_status register_grid_index(spx_ctx *ctx, spx_polys polys, std::unique_ptr<IndexObj> ix, size_t total, int g, int sb,
                               int fp32, const GridParts &gp, std::chrono::steady_clock::time_point t0, spx_index *out)
{
    PolysObj *pg = lookup(ctx->polys, polys);
    ix->polys = polys;
    ix->fp32 = fp32 ? 1 : 0;
    ix->view = grid_view(gp, g, sb, pg->P);
    ix->n_fine = gp.n_fine;
    ix->n_ent = gp.n_ent;
    ix->n_edge = gp.n_edge;
    ix->view.err = &ctx->aux->err;
    spx_index_info &inf = ix->info;
    inf.grid_log2 = g;
    inf.sub_log2 = sb;
    inf.n_polys = pg->P;
    inf.n_cells = gp.n_cell;
    inf.n_blocks = gp.n_blocks;
    inf.n_entries = gp.n_ent;
    inf.n_inside = gp.n_inside;
    inf.n_mixed = gp.n_mixed;
    inf.n_boundary = gp.n_boundary;
    inf.n_edge_refs = gp.n_edge;
    inf.device_bytes = total;
    inf.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    inf.sum_resolved = gp.sum_resolved;
    inf.use_sum = ix->view.use_sum;
    pg->n_index++;
    const uint64_t h = make_handle(ctx, kTagIndex);
    ctx->indexes[h] = std::move(ix);
    *out = h;
    return SPX_OK;
}

// Build the index of polygon set `polys` with the checked parameters prm.  An
// index of more than max_bytes device bytes is not uploaded: *out is then 0.
spx_status build_index_impl(spx_ctx *ctx, spx_polys polys, const spx_index_params &prm, spx_index *out,
                            size_t max_bytes = SIZE_MAX)
{
    PolysObj *pg = lookup(ctx->polys, polys);
    if (!pg)
        return fail(ctx, SPX_EINVAL, "build_index: bad polygon handle");
    const auto t0 = std::chrono::steady_clock::now();
    const int g = prm.grid_log2 ? prm.grid_log2 : default_grid_log2(pg->xy.data(), pg->off.data(), pg->P);
    const int sb = prm.sub_log2 ? prm.sub_log2 : kMaxSubLog2;
    if (g < 1 || g > kMaxGridLog2 || sb < 1 || sb > kMaxSubLog2 || g + sb > kMaxFineLog2)
        return fail(ctx, SPX_EINVAL, "build_index: grid_log2 must be in [1, 13] (0 = automatic), sub_log2 in "
                                     "[1, 3] (0 = default), grid_log2 + sub_log2 <= 16");
    HostIndex hi;
    std::string err;
    const int threads = std::max(1u, std::thread::hardware_concurrency());
    if (!build_grid_index(pg->xy.data(), pg->off.data(), pg->P, g, sb, threads, hi, err))
        return fail(ctx, SPX_EINVAL, "build_index: " + err);
    // the arrays the kernels will walk: every offset and id in bounds
    if (!validate_grid_index(hi.cell.data(), hi.cell.size(), hi.fine.data(), hi.fine.size(), hi.entries.data(),
                             hi.entries.size() / 4, hi.edges.data(), hi.edges.size() / 4, g, sb, pg->P, err))
        return fail(ctx, SPX_EKERNEL, "build_index: internal consistency check of the index failed: " + err);
    const std::vector<uint32_t> cover = cover_bitmap(hi.cell.data(), g);
    double sum_resolved = 0;
    const std::vector<uint16_t> sum = block_summary(hi.cell.data(), g, &sum_resolved);
    const size_t b_cell = hi.cell.size() * 4, b_fine = hi.fine.size() * 4, b_ent = hi.entries.size() * 4,
                 b_edge = hi.edges.size() * 4, b_cover = cover.size() * 4, b_sum = std::max<size_t>(sum.size() * 2, 16);
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t total = up(b_cell) + up(b_fine) + up(b_ent) + up(b_edge) + up(b_cover) + up(b_sum) + 256;
    if (total > max_bytes) {
        *out = 0;
        return SPX_OK;
    }
    auto ix = std::make_unique<IndexObj>();
    if (cudaMalloc(&ix->mem, total) != cudaSuccess)
        return fail(ctx, SPX_ENOMEM, "build_index: cudaMalloc of " + std::to_string(total) + " bytes failed");
    char *m = static_cast<char *>(ix->mem);
    char *p_cell = m, *p_fine = p_cell + up(b_cell), *p_ent = p_fine + up(b_fine), *p_edge = p_ent + up(b_ent),
         *p_cover = p_edge + up(b_edge), *p_sum = p_cover + up(b_cover);
    cudaError_t e = cudaMemcpy(p_cell, hi.cell.data(), b_cell, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p_cover, cover.data(), b_cover, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p_sum, sum.data(), sum.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && b_fine)
        e = cudaMemcpy(p_fine, hi.fine.data(), b_fine, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && b_ent)
        e = cudaMemcpy(p_ent, hi.entries.data(), b_ent, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && b_edge)
        e = cudaMemcpy(p_edge, hi.edges.data(), b_edge, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(ix->mem);
        return cuda_fail(ctx, e, "build_index upload");
    }
    GridParts gp{p_cell, p_fine, p_ent, p_edge, p_cover, p_sum, hi.cell.size(), hi.fine.size(), hi.entries.size() / 4,
                 hi.edges.size() / 4, hi.n_blocks, hi.n_inside, hi.n_mixed, hi.n_boundary, sum_resolved};
    return register_grid_index(ctx, polys, std::move(ix), total, g, sb, prm.fp32_filter, gp, t0, out);
}

} // namespace

namespace spx {

std::string check_rings(const int32_t *xy, const uint64_t *ring_off, uint32_t P)
{
    if (P >= (1u << 30))
        return "too many polygons (limit 2^30 - 1)";
    if (ring_off[0] != 0)
        return "ring_off[0] must be 0";
    for (uint32_t q = 0; q < P; ++q)
        if (ring_off[q + 1] < ring_off[q])
            return "ring_off must be non-decreasing";
    if (P && ring_off[P] >= (uint64_t(1) << 32))
        return "more than 2^32 - 1 vertices";
    for (uint64_t i = 0; i < (P ? ring_off[P] : 0); ++i)
        if (xy[2 * i] < 0 || xy[2 * i] > int32_t(kBox) || xy[2 * i + 1] < 0 || xy[2 * i + 1] > int32_t(kBox))
            return "vertex " + std::to_string(i) + " outside [0, 2^30]^2";
    return {};
}

int device_grid_index(const int32_t *xy, const uint64_t *ring_off, uint32_t P, IndexView &view, void *&mem,
                      size_t &bytes, std::string &err, cudaStream_t s, cudaMemPool_t pool)
{
    // built inside a request's latency: one level coarser than the automatic
    // grid (the build scans every coarse cell, four times fewer of them)
    const int g = std::max(5, default_grid_log2(xy, ring_off, P) - 1), sb = kMaxSubLog2;
    GridIndexDev d{};
    const char *why = nullptr;
    cudaError_t e = cudaSuccess;
    const int st = build_grid_index_device(xy, ring_off, P, g, sb, d, why, e, s, pool);
    if (st != 0) {
        err = st == 1 ? std::string(why) : std::string(cudaGetErrorString(e));
        return st;
    }
    view = grid_view(device_parts(d), g, sb, P);
    mem = d.mem;
    bytes = d.bytes;
    return 0;
}

spx_status served_data(spx_ctx *ctx, spx_points points, const spx_index *indexes, uint32_t n, ServedData &out)
{
    PointsObj *pts = lookup(ctx->points, points);
    if (!pts)
        return fail(ctx, SPX_EINVAL, "server: bad points handle");
    if (pts->cluster_log2)
        return fail(ctx, SPX_EINVAL, "server: a cell-clustered point table has no row order");
    out.device = ctx->device;
    out.pts = reinterpret_cast<const int2 *>(pts->dev);
    out.n = pts->n;
    out.ix.clear();
    out.fp32.clear();
    for (uint32_t i = 0; i < n; ++i) {
        IndexObj *ix = lookup(ctx->indexes, indexes[i]);
        if (!ix || ix->kind != 0)
            return fail(ctx, SPX_EINVAL, "server: bad index handle at position " + std::to_string(i) +
                                             " (polygon indexes only)");
        out.ix.push_back(ix->view);
        out.fp32.push_back(ix->fp32);
    }
    return SPX_OK;
}

spx_status ctx_error(spx_ctx *ctx, spx_status st, const std::string &msg) { return fail(ctx, st, msg); }

} // namespace spx

extern "C" {

spx_status spx_join_plain_static(spx_ctx *ctx, spx_points points, spx_index index, uint32_t *pairs_dev, uint64_t cap,
                                 uint64_t *counts_dev, uint64_t *total_dev, void *stream)
{
    if (!ctx)
        return SPX_EINVAL;
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    PointsObj *pts = lookup(ctx->points, points);
    IndexObj *ix = lookup(ctx->indexes, index);
    if (!pts || !ix)
        return fail(ctx, SPX_EINVAL, "join_plain_static: bad points or index handle");
    if (pts->cluster_log2)
        return fail(ctx, SPX_EINVAL, "join_plain_static: a cell-clustered point table has no row order");
    if (ix->kind != 0)
        return fail(ctx, SPX_EINVAL, "join_plain_static: needs a polygon index");
    if (pts->n > kStaticJoinMaxPoints)
        return fail(ctx, SPX_EINVAL, "join_plain_static: the point table has " + std::to_string(pts->n) +
                                         " points; the allocation-free join takes at most " +
                                         std::to_string(kStaticJoinMaxPoints));
    if (cap && !pairs_dev)
        return fail(ctx, SPX_EINVAL, "join_plain_static: pairs_dev is NULL with cap > 0");
    if ((reinterpret_cast<uintptr_t>(pairs_dev) & 7) || (reinterpret_cast<uintptr_t>(counts_dev) & 7) ||
        (reinterpret_cast<uintptr_t>(total_dev) & 7))
        return fail(ctx, SPX_EINVAL, "join_plain_static: output pointers must be 8-byte aligned");
    cudaError_t e = cudaSuccess;
    void *scratch = static_join_scratch(ctx->device, e);
    if (!scratch)
        return cuda_fail(ctx, e, "join_plain_static: cudaGetSymbolAddress of the static scratch");
    JoinLaunch a{};
    a.ix = ix->view;
    a.pts = reinterpret_cast<const int2 *>(pts->dev);
    a.n = pts->n;
    a.pairs = reinterpret_cast<uint2 *>(pairs_dev);
    a.cap = pairs_dev ? cap : 0;
    a.counts = reinterpret_cast<unsigned long long *>(counts_dev);
    a.total = reinterpret_cast<unsigned long long *>(total_dev);
    a.err = &ctx->aux->err;
    a.stats = ctx->aux->stats;
    a.fp32 = 0;
    // every block total is written by the counting pass before it is read: no clearing needed
    e = launch_join_plain(a, scratch, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "join_plain_static launch");
    return SPX_OK;
}

spx_status spx_create(int device, spx_ctx **out)
{
    if (!out)
        return SPX_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return SPX_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess)
        return SPX_ECUDA;
    std::unique_ptr<spx_ctx> c(new spx_ctx());
    c->device = device;
    if (cudaMalloc(reinterpret_cast<void **>(&c->aux), sizeof(Aux)) != cudaSuccess)
        return SPX_ENOMEM;
    if (cudaMemset(c->aux, 0, sizeof(Aux)) != cudaSuccess)
        return SPX_ECUDA;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
        return SPX_ECUDA;
    *out = c.release();
    return SPX_OK;
}

void spx_destroy(spx_ctx *ctx)
{
    if (!ctx)
        return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &kv : ctx->indexes)
        cudaFree(kv.second->mem);
    for (auto &kv : ctx->points) {
        if (kv.second->owned)
            cudaFree(kv.second->dev);
        cudaFree(kv.second->cell_end);
    }
    cudaFree(ctx->aux);
    cudaFree(ctx->scratch);
    cudaFree(ctx->st_pts);
    cudaFree(ctx->st_pairs);
    cudaFree(ctx->st_counts);
    for (auto &kv : ctx->select_graphs)
        cudaGraphExecDestroy(kv.second);
    if (ctx->capture_stream)
        cudaStreamDestroy(ctx->capture_stream);
    if (ctx->in_stream)
        cudaStreamDestroy(ctx->in_stream);
    if (ctx->emit_stream)
        cudaStreamDestroy(ctx->emit_stream);
    if (ctx->out_stream)
        cudaStreamDestroy(ctx->out_stream);
    cudaFreeHost(ctx->slice_words);
    for (auto e : ctx->slice_ev)
        cudaEventDestroy(e);
    if (ctx->stream)
        cudaStreamDestroy(ctx->stream);
    for (auto &e : ctx->ev)
        if (e)
            cudaEventDestroy(e);
    delete ctx;
}

const char *spx_last_error(const spx_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

spx_status spx_load_points(spx_ctx *ctx, const int32_t *xy, uint64_t n, int xy_is_device, spx_points *out)
{
    if (!ctx || !out || (!xy && n))
        return fail(ctx, SPX_EINVAL, "load_points: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    if (n >= (1ull << 32))
        return fail(ctx, SPX_EINVAL, "load_points: n must be < 2^32 (point ids are uint32)");
    auto p = std::make_unique<PointsObj>();
    p->n = n;
    if (xy_is_device) {
        if (reinterpret_cast<uintptr_t>(xy) & 15)
            return fail(ctx, SPX_EINVAL, "load_points: device buffer must be 16-byte aligned");
        p->dev = const_cast<int32_t *>(xy);
        p->owned = false;
    } else {
        for (uint64_t i = 0; i < 2 * n; ++i)
            if (xy[i] < 0 || xy[i] >= int32_t(kBox))
                return fail(ctx, SPX_EINVAL, "load_points: coordinate " + std::to_string(xy[i]) + " at point " +
                                                 std::to_string(i / 2) + " outside [0, 2^30)");
        void *d = nullptr;
        if (cudaMalloc(&d, n ? n * 8 : 16) != cudaSuccess)
            return fail(ctx, SPX_ENOMEM, "load_points: cudaMalloc failed");
        const cudaError_t e = n ? cudaMemcpy(d, xy, n * 8, cudaMemcpyHostToDevice) : cudaSuccess;
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(ctx, e, "load_points copy");
        }
        p->dev = static_cast<int32_t *>(d);
        p->owned = true;
    }
    const uint64_t h = make_handle(ctx, kTagPoints);
    ctx->points[h] = std::move(p);
    *out = h;
    return SPX_OK;
}

spx_status spx_cluster_points(spx_ctx *ctx, spx_points points, int grid_log2, spx_points *out)
{
    if (!ctx || !out)
        return fail(ctx, SPX_EINVAL, "cluster_points: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    PointsObj *src = lookup(ctx->points, points);
    if (!src)
        return fail(ctx, SPX_EINVAL, "cluster_points: bad points handle");
    const int c = grid_log2 ? grid_log2 : 12;
    if (c < 1 || c > 13)
        return fail(ctx, SPX_EINVAL, "cluster_points: grid_log2 must be in [1, 13] (0 = 12)");
    auto p = std::make_unique<PointsObj>();
    p->n = src->n;
    p->owned = true;
    p->cluster_log2 = c;
    void *d = nullptr, *scratch = nullptr;
    if (cudaMalloc(&d, src->n ? src->n * 8 : 16) != cudaSuccess)
        return fail(ctx, SPX_ENOMEM, "cluster_points: cudaMalloc of the copy failed");
    if (cudaMalloc(&scratch, cluster_scratch_bytes(c)) != cudaSuccess) {
        cudaFree(d);
        return fail(ctx, SPX_ENOMEM, "cluster_points: cudaMalloc of the cell counters failed");
    }
    const size_t bins = (size_t(1) << (2 * c)) + 1;
    if (cudaMalloc(reinterpret_cast<void **>(&p->cell_end), bins * 8) != cudaSuccess) {
        cudaFree(d);
        cudaFree(scratch);
        return fail(ctx, SPX_ENOMEM, "cluster_points: cudaMalloc of the cell directory failed");
    }
    cudaStream_t s = ctx->stream;
    cudaError_t e = src->n ? cudaSuccess : cudaMemsetAsync(scratch, 0, bins * 8, s);
    if (e == cudaSuccess)
        e = launch_cluster(reinterpret_cast<const int2 *>(src->dev), src->n, c, scratch, static_cast<int2 *>(d), s);
    // after the scatter the counting sort's cursors are the cells' end rows: the directory
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->cell_end, scratch, bins * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (e != cudaSuccess) {
        cudaFree(d);
        cudaFree(p->cell_end);
        return cuda_fail(ctx, e, "cluster_points");
    }
    p->dev = static_cast<int32_t *>(d);
    const uint64_t h = make_handle(ctx, kTagPoints);
    ctx->points[h] = std::move(p);
    *out = h;
    return SPX_OK;
}

spx_status spx_points_info(spx_ctx *ctx, spx_points points, const int32_t **xy_dev, uint64_t *n, int *cluster_log2)
{
    if (!ctx)
        return SPX_EINVAL;
    PointsObj *p = lookup(ctx->points, points);
    if (!p)
        return fail(ctx, SPX_EINVAL, "points_info: bad points handle");
    if (xy_dev)
        *xy_dev = p->dev;
    if (n)
        *n = p->n;
    if (cluster_log2)
        *cluster_log2 = p->cluster_log2;
    return SPX_OK;
}

spx_status spx_load_polygons(spx_ctx *ctx, const int32_t *xy, const uint64_t *ring_off, uint32_t P, spx_polys *out)
{
    if (!ctx || !out || !ring_off)
        return fail(ctx, SPX_EINVAL, "load_polygons: null argument");
    ctx->err.clear();
    if (P >= (1u << 30))
        return fail(ctx, SPX_EINVAL, "load_polygons: P must be < 2^30");
    if (ring_off[0] != 0)
        return fail(ctx, SPX_EINVAL, "load_polygons: ring_off[0] must be 0");
    for (uint32_t q = 0; q < P; ++q)
        if (ring_off[q + 1] < ring_off[q])
            return fail(ctx, SPX_EINVAL, "load_polygons: ring_off must be non-decreasing");
    const uint64_t V = ring_off[P];
    if (V && !xy)
        return fail(ctx, SPX_EINVAL, "load_polygons: xy is NULL");
    for (uint64_t i = 0; i < 2 * V; ++i)
        if (xy[i] < 0 || xy[i] > int32_t(kBox))
            return fail(ctx, SPX_EINVAL, "load_polygons: vertex coordinate " + std::to_string(xy[i]) +
                                             " outside [0, 2^30]");
    auto p = std::make_unique<PolysObj>();
    p->xy.assign(xy, xy + 2 * V);
    p->off.assign(ring_off, ring_off + P + 1);
    p->P = P;
    const uint64_t h = make_handle(ctx, kTagPolys);
    ctx->polys[h] = std::move(p);
    *out = h;
    return SPX_OK;
}

spx_status spx_build_index_device(spx_ctx *ctx, spx_polys polys, const spx_index_params *params, spx_index *out)
{
    if (!ctx || !out)
        return fail(ctx, SPX_EINVAL, "build_index_device: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    spx_index_params prm{};
    prm.fp32_filter = 1;
    if (params) {
        prm = *params;
        for (int r : prm.reserved)
            if (r)
                return fail(ctx, SPX_EINVAL, "build_index_device: reserved fields must be zero");
    }
    PolysObj *pg = lookup(ctx->polys, polys);
    if (!pg)
        return fail(ctx, SPX_EINVAL, "build_index_device: bad polygon handle");
    const auto t0 = std::chrono::steady_clock::now();
    const int g = prm.grid_log2 ? prm.grid_log2 : default_grid_log2(pg->xy.data(), pg->off.data(), pg->P);
    const int sb = prm.sub_log2 ? prm.sub_log2 : kMaxSubLog2;
    if (g < 1 || g > kMaxGridLog2 || sb < 1 || sb > kMaxSubLog2 || g + sb > kMaxFineLog2)
        return fail(ctx, SPX_EINVAL, "build_index_device: grid_log2 must be in [1, 13] (0 = automatic), sub_log2 "
                                     "in [1, 3] (0 = default), grid_log2 + sub_log2 <= 16");
    if (pg->P >= (1u << 30))
        return fail(ctx, SPX_EINVAL, "build_index_device: too many polygons (limit 2^30 - 1)");
    if (pg->P && pg->off[pg->P] >= (uint64_t(1) << 32))
        return fail(ctx, SPX_EINVAL, "build_index_device: more than 2^32 - 1 vertices");
    GridIndexDev d{};
    const char *why = nullptr;
    cudaError_t e = cudaSuccess;
    const int st = build_grid_index_device(pg->xy.data(), pg->off.data(), pg->P, g, sb, d, why, e);
    if (st == 1)
        return fail(ctx, SPX_EINVAL, std::string("build_index_device: ") + why);
    if (st != 0)
        return e == cudaErrorMemoryAllocation ? fail(ctx, SPX_ENOMEM, "build_index_device: out of device memory")
                                              : cuda_fail(ctx, e, "build_index_device");
    auto ix = std::make_unique<IndexObj>();
    ix->mem = d.mem;
    return register_grid_index(ctx, polys, std::move(ix), d.bytes, g, sb, prm.fp32_filter, device_parts(d), t0, out);
}

spx_status spx_index_arrays(spx_ctx *ctx, spx_index index, uint32_t *coarse, uint32_t *fine, uint32_t *entries,
                            int32_t *edges, uint64_t sizes[4])
{
    if (!ctx || !sizes)
        return fail(ctx, SPX_EINVAL, "index_arrays: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    IndexObj *ix = lookup(ctx->indexes, index);
    if (!ix || ix->kind != 0)
        return fail(ctx, SPX_EINVAL, "index_arrays: not a polygon index");
    sizes[0] = ix->info.n_cells;
    sizes[1] = ix->n_fine;
    sizes[2] = ix->n_ent;
    sizes[3] = ix->n_edge;
    if (coarse)
        SPX_CUDA(cudaMemcpy(coarse, ix->view.cell, sizes[0] * 4, cudaMemcpyDeviceToHost), "index_arrays coarse");
    if (fine)
        SPX_CUDA(cudaMemcpy(fine, ix->view.fine, sizes[1] * 4, cudaMemcpyDeviceToHost), "index_arrays fine");
    if (entries)
        SPX_CUDA(cudaMemcpy(entries, ix->view.ent, sizes[2] * 16, cudaMemcpyDeviceToHost), "index_arrays entries");
    if (edges)
        SPX_CUDA(cudaMemcpy(edges, ix->view.edge, sizes[3] * 16, cudaMemcpyDeviceToHost), "index_arrays edges");
    return SPX_OK;
}

spx_status spx_build_index(spx_ctx *ctx, spx_polys polys, const spx_index_params *params, spx_index *out)
{
    if (!ctx || !out)
        return fail(ctx, SPX_EINVAL, "build_index: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    spx_index_params prm{};
    prm.fp32_filter = 1;
    if (params) {
        prm = *params;
        for (int r : prm.reserved)
            if (r)
                return fail(ctx, SPX_EINVAL, "build_index: reserved fields must be zero");
    }
    return build_index_impl(ctx, polys, prm, out);
}

spx_status spx_autotune(spx_ctx *ctx, spx_points points, spx_polys polys, const spx_tune_params *tp,
                        spx_index_params *best, spx_tune_trial *trials, uint32_t max_trials, uint32_t *n_trials,
                        spx_index *best_index, void *stream)
{
    if (!ctx || !best || (max_trials && !trials))
        return fail(ctx, SPX_EINVAL, "autotune: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    PointsObj *pts = lookup(ctx->points, points);
    PolysObj *pg = lookup(ctx->polys, polys);
    if (!pts || !pg)
        return fail(ctx, SPX_EINVAL, "autotune: bad points or polygon handle");
    if (pts->n == 0)
        return fail(ctx, SPX_EINVAL, "autotune: the point table is empty");
    spx_tune_params q{};
    if (tp) {
        q = *tp;
        for (int r : q.reserved)
            if (r)
                return fail(ctx, SPX_EINVAL, "autotune: reserved fields must be zero");
    } else {
        q.fp32_filter = 1;
    }
    const int gmin = q.grid_min ? q.grid_min : 6, gmax = q.grid_max ? q.grid_max : kMaxGridLog2;
    const int reps = q.reps ? q.reps : 5;
    const uint64_t max_bytes = q.max_index_bytes ? q.max_index_bytes : (uint64_t(4) << 30);
    if (gmin < 1 || gmax > kMaxGridLog2 || gmin > gmax || reps < 1 || reps > 1000 ||
        (q.fp32_filter != 0 && q.fp32_filter != 1))
        return fail(ctx, SPX_EINVAL, "autotune: need 1 <= grid_min <= grid_max <= 13, 1 <= reps <= 1000, "
                                     "fp32_filter 0 or 1");
    uint64_t m = q.sample_points ? q.sample_points : std::max(pts->n / 100, std::min<uint64_t>(pts->n, 1u << 22));
    if (m > pts->n)
        m = pts->n;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint32_t P = pg->P;

    // device memory of the tuner: sample | reference counts | candidate counts | counter words
    const size_t b_sample = (m * 8 + 255) & ~size_t(255), b_counts = ((size_t(P) + 1) * 8 + 255) & ~size_t(255);
    void *mem = nullptr;
    if (cudaMalloc(&mem, b_sample + 2 * b_counts + 256) != cudaSuccess)
        return fail(ctx, SPX_ENOMEM, "autotune: cudaMalloc of the sample failed");
    std::unique_ptr<void, decltype(&cudaFree)> mem_guard(mem, &cudaFree);
    int2 *sample = static_cast<int2 *>(mem);
    auto *ref = reinterpret_cast<unsigned long long *>(static_cast<char *>(mem) + b_sample);
    auto *cur = reinterpret_cast<unsigned long long *>(static_cast<char *>(mem) + b_sample + b_counts);
    void *words = static_cast<char *>(mem) + b_sample + 2 * b_counts;
    SPX_CUDA(launch_gather_stride(reinterpret_cast<const int2 *>(pts->dev), pts->n, sample, m, s), "autotune sample");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SPX_CUDA(cudaEventCreate(&e0), "event create");
    SPX_CUDA(cudaEventCreate(&e1), "event create");
    std::unique_ptr<CUevent_st, decltype(&cudaEventDestroy)> g0(e0, &cudaEventDestroy), g1(e1, &cudaEventDestroy);

    std::vector<spx_tune_trial> done;
    std::vector<unsigned long long> h_ref(P ? P : 1), h_cur(P ? P : 1);
    spx_index best_h = 0;
    double best_ms = 0;
    spx_index_params best_p{};
    // time one candidate: 1 = timed, 0 = skipped (index too large or not allowed)
    auto run = [&](int g, int sb, int &outcome) -> spx_status {
        outcome = 0;
        if (g < 1 || g > kMaxGridLog2 || sb < 1 || sb > kMaxSubLog2 || g + sb > kMaxFineLog2)
            return SPX_OK;
        for (const auto &t : done)
            if (t.grid_log2 == g && t.sub_log2 == sb)
                return SPX_OK;
        spx_index_params prm{};
        prm.grid_log2 = g;
        prm.sub_log2 = sb;
        prm.fp32_filter = q.fp32_filter;
        spx_index h = 0;
        spx_status st = build_index_impl(ctx, polys, prm, &h, max_bytes);
        if (st != SPX_OK)
            return st;
        if (!h)
            return SPX_OK;
        IndexObj *ix = lookup(ctx->indexes, h);
        JoinLaunch a{};
        a.ix = ix->view;
        a.pts = sample;
        a.n = m;
        a.counts = done.empty() ? ref : cur;
        a.err = &ctx->aux->err;
        a.stats = ctx->aux->stats;
        a.fp32 = ix->fp32;
        a.clustered = pts->cluster_log2 ? 1 : 0; // the strided sample keeps the table's order
        float best_t = 0;
        cudaError_t e = cudaSuccess;
        for (int r = 0; r <= reps && e == cudaSuccess; ++r) { // launch 0 warms the index into L2
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess)
                e = launch_aggregate(a, words, s);
            if (e == cudaSuccess)
                e = cudaEventRecord(e1, s);
            if (e == cudaSuccess)
                e = cudaEventSynchronize(e1);
            float t = 0;
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&t, e0, e1);
            if (r == 1 || (r > 1 && t < best_t))
                best_t = t;
        }
        if (e != cudaSuccess) {
            spx_free(ctx, h);
            return cuda_fail(ctx, e, "autotune launch");
        }
        st = check_kernel_err(ctx, s);
        if (st == SPX_OK && !done.empty()) {
            cudaError_t e2 = cudaMemcpy(h_cur.data(), cur, sizeof(unsigned long long) * P, cudaMemcpyDeviceToHost);
            if (e2 != cudaSuccess)
                st = cuda_fail(ctx, e2, "autotune counts");
            else if (h_cur != h_ref)
                st = fail(ctx, SPX_EKERNEL, "autotune: counts at grid_log2 " + std::to_string(g) + ", sub_log2 " +
                                                std::to_string(sb) + " differ from the first candidate's");
        } else if (st == SPX_OK) {
            cudaError_t e2 = cudaMemcpy(h_ref.data(), ref, sizeof(unsigned long long) * P, cudaMemcpyDeviceToHost);
            if (e2 != cudaSuccess)
                st = cuda_fail(ctx, e2, "autotune counts");
        }
        if (st != SPX_OK) {
            const std::string msg = ctx->err;
            spx_free(ctx, h);
            ctx->err = msg;
            return st;
        }
        done.push_back({g, sb, double(best_t), ix->info.build_ms, ix->info.device_bytes});
        outcome = 1;
        if (!best_h || best_t < best_ms) {
            if (best_h)
                spx_free(ctx, best_h);
            best_h = h;
            best_ms = best_t;
            best_p = prm;
        } else {
            spx_free(ctx, h);
        }
        return SPX_OK;
    };
    auto cleanup_fail = [&](spx_status st) {
        const std::string msg = ctx->err;
        if (best_h)
            spx_free(ctx, best_h);
        ctx->err = msg;
        return st;
    };
    // 1. grid_log2 upwards at the largest sub_log2 allowed
    int misses = 0;
    for (int g = gmin; g <= gmax && misses < 2; ++g) {
        const double before = best_h ? best_ms : 0;
        const bool had = best_h != 0;
        int outcome = 0;
        spx_status st = run(g, std::min(kMaxSubLog2, kMaxFineLog2 - g), outcome);
        if (st != SPX_OK)
            return cleanup_fail(st);
        if (!outcome)
            continue;
        misses = (had && !(best_ms < before)) ? misses + 1 : 0;
    }
    if (!best_h)
        return fail(ctx, SPX_EINVAL, "autotune: every candidate's index exceeds max_index_bytes");
    // 2. sub_log2 at the best grid_log2
    const int gb = best_p.grid_log2;
    for (int sb = 1; sb <= kMaxSubLog2; ++sb) {
        int outcome = 0;
        spx_status st = run(gb, sb, outcome);
        if (st != SPX_OK)
            return cleanup_fail(st);
    }
    *best = best_p;
    if (n_trials)
        *n_trials = uint32_t(done.size());
    for (uint32_t i = 0; i < max_trials && i < done.size(); ++i)
        trials[i] = done[i];
    if (best_index)
        *best_index = best_h;
    else
        spx_free(ctx, best_h);
    return SPX_OK;
}

// Why a disk set cannot be indexed (empty: it can).
static std::string check_disks(const int32_t *cxy, const int32_t *r, uint32_t Q)
{
    if (Q >= (1u << 30))
        return "Q must be < 2^30";
    for (uint32_t q = 0; q < Q; ++q) {
        if (cxy[2 * q] < 0 || cxy[2 * q] > int32_t(kBox) || cxy[2 * q + 1] < 0 || cxy[2 * q + 1] > int32_t(kBox))
            return "centre " + std::to_string(q) + " outside [0, 2^30]^2";
        if (r[q] < 0 || r[q] >= int32_t(kBox))
            return "radius " + std::to_string(q) + " outside [0, 2^30)";
    }
    return {};
}

// Registers a disk index whose arrays are in one device allocation.
static spx_status register_disk_index(spx_ctx *ctx, void *mem, size_t total, const uint32_t *cell, const uint32_t *ent,
                                      const int4 *disk, const uint32_t *cover, int g, uint32_t Q, uint64_t n_entries,
                                      uint64_t n_inside, uint64_t n_boundary,
                                      std::chrono::steady_clock::time_point t0, spx_index *out)
{
    auto ix = std::make_unique<IndexObj>();
    ix->mem = mem;
    ix->kind = 1;
    ix->dview.cell = cell;
    ix->dview.ent = ent;
    ix->dview.disk = disk;
    ix->dview.cover = cover;
    ix->dview.sc = kBoxLog2 - g;
    ix->dview.g = g;
    ix->dview.cg = std::min(g, kCoverLog2);
    ix->dview.scv = kBoxLog2 - ix->dview.cg;
    ix->dview.Q = Q;
    spx_index_info &inf = ix->info;
    inf.grid_log2 = g;
    inf.n_polys = Q;
    inf.n_cells = uint64_t(1) << (2 * g);
    inf.n_entries = n_entries;
    inf.n_inside = n_inside;
    inf.n_boundary = n_boundary;
    inf.device_bytes = total;
    inf.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    const uint64_t h = make_handle(ctx, kTagIndex);
    ctx->indexes[h] = std::move(ix);
    *out = h;
    return SPX_OK;
}

static std::vector<int4> disk_array(const int32_t *cxy, const int32_t *r, uint32_t Q)
{
    std::vector<int4> disks(std::max<uint32_t>(Q, 1));
    for (uint32_t q = 0; q < Q; ++q)
        disks[q] = make_int4(cxy[2 * q], cxy[2 * q + 1], r[q], 0);
    return disks;
}

spx_status spx_build_disk_index(spx_ctx *ctx, const int32_t *cxy, const int32_t *r, uint32_t Q, int grid_log2,
                                spx_index *out)
{
    if (!ctx || !out || (Q && (!cxy || !r)))
        return fail(ctx, SPX_EINVAL, "build_disk_index: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    {
        const std::string bad = check_disks(cxy, r, Q);
        if (!bad.empty())
            return fail(ctx, SPX_EINVAL, "build_disk_index: " + bad);
    }
    const auto t0 = std::chrono::steady_clock::now();
    const int g = grid_log2 ? grid_log2 : default_disk_grid_log2(r, Q);
    HostDiskIndex hd;
    std::string err;
    if (!build_disk_index(cxy, r, Q, g, hd, err))
        return fail(ctx, SPX_EINVAL, "build_disk_index: " + err);
    const std::vector<int4> disks = disk_array(cxy, r, Q);
    const std::vector<uint32_t> cover = cover_bitmap(hd.cell.data(), g);
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t b_cell = hd.cell.size() * 4, b_ent = hd.entries.size() * 4, b_disk = disks.size() * sizeof(int4),
                 b_cover = cover.size() * 4;
    const size_t total = up(b_cell) + up(b_ent) + up(b_disk) + up(b_cover);
    void *mem = nullptr;
    if (cudaMalloc(&mem, total) != cudaSuccess)
        return fail(ctx, SPX_ENOMEM, "build_disk_index: cudaMalloc failed");
    char *m = static_cast<char *>(mem), *p_ent = m + up(b_cell), *p_disk = p_ent + up(b_ent),
         *p_cover = p_disk + up(b_disk);
    cudaError_t e = cudaMemcpy(m, hd.cell.data(), b_cell, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p_ent, hd.entries.data(), b_ent, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p_disk, disks.data(), b_disk, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p_cover, cover.data(), b_cover, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(mem);
        return cuda_fail(ctx, e, "build_disk_index upload");
    }
    return register_disk_index(ctx, mem, total, reinterpret_cast<const uint32_t *>(m),
                               reinterpret_cast<const uint32_t *>(p_ent), reinterpret_cast<const int4 *>(p_disk),
                               reinterpret_cast<const uint32_t *>(p_cover), g, Q, hd.entries.size(), hd.n_inside,
                               hd.n_boundary, t0, out);
}

spx_status spx_build_disk_index_device(spx_ctx *ctx, const int32_t *cxy, const int32_t *r, uint32_t Q, int grid_log2,
                                       spx_index *out)
{
    if (!ctx || !out || (Q && (!cxy || !r)))
        return fail(ctx, SPX_EINVAL, "build_disk_index_device: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    {
        const std::string bad = check_disks(cxy, r, Q);
        if (!bad.empty())
            return fail(ctx, SPX_EINVAL, "build_disk_index_device: " + bad);
    }
    const auto t0 = std::chrono::steady_clock::now();
    const int g = grid_log2 ? grid_log2 : default_disk_grid_log2(r, Q);
    if (g < 1 || g > kMaxGridLog2)
        return fail(ctx, SPX_EINVAL, "build_disk_index_device: grid_log2 must be in [1, 13]");
    const std::vector<int4> disks = disk_array(cxy, r, Q);
    DiskIndexDev d{};
    cudaError_t e = cudaSuccess;
    const int st = build_disk_index_device(disks.data(), Q, g, d, e);
    if (st == 1)
        return fail(ctx, SPX_EINVAL, "build_disk_index_device: too many disk entries for one index; use a smaller grid");
    if (st != 0)
        return e == cudaErrorMemoryAllocation ? fail(ctx, SPX_ENOMEM, "build_disk_index_device: out of device memory")
                                              : cuda_fail(ctx, e, "build_disk_index_device");
    return register_disk_index(ctx, d.mem, d.bytes, d.cell, d.ent, d.disk, d.cover, g, Q, d.n_ent, d.n_inside,
                               d.n_boundary, t0, out);
}

spx_status spx_disk_index_arrays(spx_ctx *ctx, spx_index index, uint32_t *cell, uint32_t *entries, uint64_t sizes[3])
{
    if (!ctx || !sizes)
        return fail(ctx, SPX_EINVAL, "disk_index_arrays: null argument");
    ctx->err.clear();
    IndexObj *ix = lookup(ctx->indexes, index);
    if (!ix || ix->kind != 1)
        return fail(ctx, SPX_EINVAL, "disk_index_arrays: not a disk index handle");
    cudaSetDevice(ctx->device);
    sizes[0] = ix->info.n_cells;
    sizes[1] = ix->info.n_entries;
    sizes[2] = uint64_t(ix->info.grid_log2);
    if (cell)
        SPX_CUDA(cudaMemcpy(cell, ix->dview.cell, sizes[0] * 4, cudaMemcpyDeviceToHost), "disk_index_arrays copy");
    if (entries)
        SPX_CUDA(cudaMemcpy(entries, ix->dview.ent, sizes[1] * 4, cudaMemcpyDeviceToHost), "disk_index_arrays copy");
    return SPX_OK;
}

spx_status spx_build_buffer_index(spx_ctx *ctx, spx_polys polys, const int32_t *r, int grid_log2, int fp32_filter,
                                  spx_index *out)
{
    if (!ctx || !out)
        return fail(ctx, SPX_EINVAL, "build_buffer_index: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    PolysObj *pg = lookup(ctx->polys, polys);
    if (!pg)
        return fail(ctx, SPX_EINVAL, "build_buffer_index: bad polygon handle");
    if (pg->P && !r)
        return fail(ctx, SPX_EINVAL, "build_buffer_index: null radii");
    if (pg->P >= kBufferFull)
        return fail(ctx, SPX_EINVAL, "build_buffer_index: more than 2^31 - 1 polygons");
    for (uint32_t q = 0; q < pg->P; ++q)
        if (r[q] < 0 || r[q] >= int32_t(kBox))
            return fail(ctx, SPX_EINVAL, "build_buffer_index: radius " + std::to_string(q) + " outside [0, 2^30)");
    if (grid_log2 < 0 || grid_log2 > 12)
        return fail(ctx, SPX_EINVAL, "build_buffer_index: grid_log2 must be in [1, 12] (0 = automatic)");
    const auto t0 = std::chrono::steady_clock::now();
    const int g = grid_log2 ? grid_log2 : default_buffer_grid_log2(pg->xy.data(), pg->off.data(), pg->P, r);
    HostBufferEdges he;
    std::string err;
    if (!build_buffer_edges(pg->xy.data(), pg->off.data(), pg->P, r, g, he, err))
        return fail(ctx, SPX_EINVAL, "build_buffer_index: " + err);
    // the polygons' own index answers containment; it becomes part of this one
    spx_index_params prm{};
    prm.fp32_filter = fp32_filter ? 1 : 0;
    prm.sub_log2 = kMaxSubLog2;
    spx_index h = 0;
    spx_status st = build_index_impl(ctx, polys, prm, &h);
    if (st != SPX_OK)
        return st;
    auto it = ctx->indexes.find(h);
    std::unique_ptr<IndexObj> ix = std::move(it->second);
    ctx->indexes.erase(it);
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    const uint32_t P = pg->P;
    const size_t n_items = he.item_q.size();
    const size_t b_off = he.cell_off.size() * 4, b_q = std::max<size_t>(n_items, 1) * 4,
                 b_seg = std::max<size_t>(n_items, 1) * 16, b_r = std::max<size_t>(P, 1) * 4;
    // the screen: cells with edges here, cells meeting a polygon by launch_buffer_mask
    const uint64_t ncell = uint64_t(1) << (2 * g);
    std::vector<uint32_t> mask(std::max<uint64_t>(ncell / 32, 1), 0u);
    for (uint64_t c = 0; c < ncell; ++c)
        if (he.cell_off[c + 1] > he.cell_off[c])
            mask[c >> 5] |= 1u << (c & 31);
    const size_t b_mask = mask.size() * 4;
    const size_t total = up(b_off) + up(b_q) + up(b_seg) + up(b_r) + up(b_mask);
    void *mem2 = nullptr;
    if (cudaMalloc(&mem2, total) != cudaSuccess) {
        cudaFree(ix->mem);
        pg->n_index--;
        return fail(ctx, SPX_ENOMEM, "build_buffer_index: cudaMalloc failed");
    }
    char *m = static_cast<char *>(mem2), *p_q = m + up(b_off), *p_seg = p_q + up(b_q), *p_r = p_seg + up(b_seg),
         *p_mask = p_r + up(b_r);
    cudaError_t e = cudaMemcpy(m, he.cell_off.data(), b_off, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_items)
        e = cudaMemcpy(p_q, he.item_q.data(), n_items * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_items)
        e = cudaMemcpy(p_seg, he.item_seg.data(), n_items * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && P)
        e = cudaMemcpy(p_r, r, size_t(P) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p_mask, mask.data(), b_mask, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_buffer_mask(ix->view, reinterpret_cast<uint32_t *>(p_mask), g, nullptr);
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(mem2);
        cudaFree(ix->mem);
        pg->n_index--;
        return cuda_fail(ctx, e, "build_buffer_index upload");
    }
    ix->kind = 2;
    ix->mem2 = mem2;
    ix->bview.cell_off = reinterpret_cast<const uint32_t *>(m);
    ix->bview.item_q = reinterpret_cast<const uint32_t *>(p_q);
    ix->bview.item_seg = reinterpret_cast<const int4 *>(p_seg);
    ix->bview.rad = reinterpret_cast<const int32_t *>(p_r);
    ix->bview.mask = reinterpret_cast<const uint32_t *>(p_mask);
    ix->bview.g = g;
    ix->bview.sc = kBoxLog2 - g;
    ix->bview.P = P;
    ix->bview.n_items = n_items;
    ix->info.edge_grid_log2 = g;
    ix->info.n_edge_items = n_items;
    ix->info.device_bytes += total;
    ix->info.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    const uint64_t hb = make_handle(ctx, kTagIndex);
    ctx->indexes[hb] = std::move(ix);
    *out = hb;
    return SPX_OK;
}

spx_status spx_index_info_get(spx_ctx *ctx, spx_index index, spx_index_info *out)
{
    if (!ctx || !out)
        return fail(ctx, SPX_EINVAL, "index_info: null argument");
    IndexObj *ix = lookup(ctx->indexes, index);
    if (!ix)
        return fail(ctx, SPX_EINVAL, "index_info: bad index handle");
    *out = ix->info;
    return SPX_OK;
}

spx_status spx_join(spx_ctx *ctx, spx_points points, spx_index index, uint32_t *pairs_dev, uint64_t cap,
                    uint64_t *counts_dev, uint64_t *total_dev, uint64_t *n_pairs, void *stream)
{
    return join_common(ctx, points, index, pairs_dev, cap, counts_dev, total_dev, n_pairs, stream, false);
}

spx_status spx_join_plain(spx_ctx *ctx, spx_points points, spx_index index, uint32_t *pairs_dev, uint64_t cap,
                          uint64_t *counts_dev, uint64_t *total_dev, uint64_t *n_pairs, void *stream)
{
    return join_common(ctx, points, index, pairs_dev, cap, counts_dev, total_dev, n_pairs, stream, true);
}

spx_status spx_select(spx_ctx *ctx, spx_points points, spx_index index, uint32_t *ids_dev, uint64_t cap,
                      uint64_t *offsets_dev, uint64_t *n_ids, void *stream)
{
    if (!ctx)
        return SPX_EINVAL;
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    PointsObj *pts = lookup(ctx->points, points);
    IndexObj *ix = lookup(ctx->indexes, index);
    if (!pts || !ix)
        return fail(ctx, SPX_EINVAL, "select: bad points or index handle");
    if (pts->cluster_log2)
        return fail(ctx, SPX_EINVAL, "select: a cell-clustered point table has no row order; use spx_aggregate");
    if (!offsets_dev || (cap && !ids_dev))
        return fail(ctx, SPX_EINVAL, "select: offsets_dev is NULL, or ids_dev is NULL with cap > 0");
    if ((reinterpret_cast<uintptr_t>(offsets_dev) & 7) || (reinterpret_cast<uintptr_t>(ids_dev) & 3))
        return fail(ctx, SPX_EINVAL, "select: misaligned output pointer");
    const uint32_t PQ = ix->kind == 1 ? ix->dview.Q : ix->kind == 2 ? ix->bview.P : ix->view.P;
    if (PQ > kSelectMaxQueries)
        return fail(ctx, SPX_EINVAL, "select: an index of " + std::to_string(PQ) +
                                         " queries; batched selection takes at most " +
                                         std::to_string(kSelectMaxQueries));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (ix->kind == 2) {
        // buffered polygons: points inside or within r of each polygon, ascending per polygon
        spx_status st = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, buffer_select_scratch_bytes(pts->n, PQ, cap),
                               s, "select");
        if (st != SPX_OK)
            return st;
        unsigned long long *offs = reinterpret_cast<unsigned long long *>(offsets_dev);
        cudaError_t e = launch_buffer_select(buffer_launch(ctx, pts, ix), ids_dev, cap, offs, ctx->scratch, s);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "select launch");
        if (n_ids) {
            if ((st = check_kernel_err(ctx, s)) != SPX_OK)
                return st;
            unsigned long long t = 0;
            SPX_CUDA(cudaMemcpy(&t, offs + PQ, sizeof(t), cudaMemcpyDeviceToHost), "select total");
            *n_ids = t;
            if (t > cap)
                return fail(ctx, SPX_ECAPACITY, "select: " + std::to_string(t) + " ids exceed capacity " +
                                                    std::to_string(cap));
        }
        return SPX_OK;
    }
    if (ix->kind == 1) {
        // distance selection: points within r of each centre, ascending per disk
        spx_status st = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, disk_select_scratch_bytes(pts->n, PQ, cap), s,
                               "select");
        if (st != SPX_OK)
            return st;
        DiskLaunch a{};
        a.dv = ix->dview;
        a.pts = reinterpret_cast<const int2 *>(pts->dev);
        a.n = pts->n;
        a.stats = ctx->aux->stats;
        unsigned long long *offs = reinterpret_cast<unsigned long long *>(offsets_dev);
        cudaError_t e = launch_disk_select(a, ids_dev, cap, offs, ctx->scratch, s);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "select launch");
        if (n_ids) {
            if ((st = check_kernel_err(ctx, s)) != SPX_OK)
                return st;
            unsigned long long t = 0;
            SPX_CUDA(cudaMemcpy(&t, offs + PQ, sizeof(t), cudaMemcpyDeviceToHost), "select total");
            *n_ids = t;
            if (t > cap)
                return fail(ctx, SPX_ECAPACITY, "select: " + std::to_string(t) + " ids exceed capacity " +
                                                    std::to_string(cap));
        }
        return SPX_OK;
    }
    spx_status st = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, select_scratch_bytes(pts->n, ix->view.P, cap), s,
                           "select");
    if (st != SPX_OK)
        return st;
    JoinLaunch a{};
    a.ix = ix->view;
    a.pts = reinterpret_cast<const int2 *>(pts->dev);
    a.n = pts->n;
    a.err = &ctx->aux->err;
    a.stats = ctx->aux->stats;
    a.fp32 = ix->fp32;
    unsigned long long *offs = reinterpret_cast<unsigned long long *>(offsets_dev);
    const auto key = std::make_tuple(points, index, reinterpret_cast<uintptr_t>(ids_dev), cap,
                                     reinterpret_cast<uintptr_t>(offsets_dev));
    auto it = ctx->select_graphs.find(key);
    if (it == ctx->select_graphs.end()) {
        // first call with these arguments: run once directly (sets kernel attributes),
        // then capture the whole sequence into a graph for the next calls
        cudaError_t e = launch_select(a, ids_dev, cap, offs, ctx->scratch, s);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "select launch");
        if (!ctx->capture_stream)
            SPX_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking), "capture stream");
        SPX_CUDA(cudaStreamSynchronize(s), "select synchronize");
        SPX_CUDA(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeRelaxed), "select capture");
        e = launch_select(a, ids_dev, cap, offs, ctx->scratch, ctx->capture_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g)
                cudaGraphDestroy(g);
            return cuda_fail(ctx, e != cudaSuccess ? e : e2, "select capture");
        }
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "select graph instantiate");
        ctx->select_graphs[key] = ge;
    } else {
        SPX_CUDA(cudaGraphLaunch(it->second, s), "select graph launch");
    }
    if (n_ids) {
        st = check_kernel_err(ctx, s);
        if (st != SPX_OK)
            return st;
        unsigned long long t = 0;
        SPX_CUDA(cudaMemcpy(&t, offs + ix->view.P, sizeof(t), cudaMemcpyDeviceToHost), "select total");
        *n_ids = t;
        if (t > cap)
            return fail(ctx, SPX_ECAPACITY, "select: " + std::to_string(t) + " ids exceed capacity " +
                                                std::to_string(cap));
    }
    return SPX_OK;
}

spx_status spx_aggregate(spx_ctx *ctx, spx_points points, spx_index index, uint64_t *counts_dev, void *stream)
{
    if (!ctx || !counts_dev)
        return fail(ctx, SPX_EINVAL, "aggregate: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    PointsObj *pts = lookup(ctx->points, points);
    IndexObj *ix = lookup(ctx->indexes, index);
    if (!pts || !ix)
        return fail(ctx, SPX_EINVAL, "aggregate: bad points or index handle");
    if (reinterpret_cast<uintptr_t>(counts_dev) & 7)
        return fail(ctx, SPX_EINVAL, "aggregate: counts_dev must be 8-byte aligned");
    if (ix->kind == 1) {
        DiskLaunch d{};
        d.dv = ix->dview;
        d.pts = reinterpret_cast<const int2 *>(pts->dev);
        d.n = pts->n;
        d.counts = reinterpret_cast<unsigned long long *>(counts_dev);
        d.stats = ctx->aux->stats;
        cudaError_t e = launch_disk_aggregate(d, reinterpret_cast<cudaStream_t>(stream));
        return e == cudaSuccess ? SPX_OK : cuda_fail(ctx, e, "aggregate launch");
    }
    if (ix->kind == 2) { // counts do not depend on the point order: clustered tables too
        BufferLaunch b = buffer_launch(ctx, pts, ix);
        b.counts = reinterpret_cast<unsigned long long *>(counts_dev);
        cudaError_t e = launch_buffer_aggregate(b, reinterpret_cast<cudaStream_t>(stream));
        return e == cudaSuccess ? SPX_OK : cuda_fail(ctx, e, "aggregate launch");
    }
    JoinLaunch a{};
    a.ix = ix->view;
    a.pts = reinterpret_cast<const int2 *>(pts->dev);
    a.n = pts->n;
    a.counts = reinterpret_cast<unsigned long long *>(counts_dev);
    a.err = &ctx->aux->err;
    a.stats = ctx->aux->stats;
    a.fp32 = ix->fp32;
    a.clustered = pts->cluster_log2 ? 1 : 0;
    a.cell_end = pts->cell_end;
    a.cluster_log2 = pts->cluster_log2;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    spx_status st = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, aggregate_scratch_bytes(a), s, "aggregate");
    if (st != SPX_OK)
        return st;
    cudaError_t e = launch_aggregate(a, ctx->scratch, s, ctx->timing ? ctx->ev : nullptr);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "aggregate launch");
    if (ctx->timing && pts->n) {
        SPX_CUDA(cudaEventSynchronize(ctx->ev[1]), "aggregate timing");
        float t = 0;
        cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[1]);
        ctx->ms_agg += t;
        ctx->timed_aggs++;
    }
    return SPX_OK;
}

static spx_status join_host_staged(spx_ctx *ctx, IndexObj *ix, const int32_t *xy_host, uint64_t n, uint32_t *pairs_host,
                                   uint64_t cap, uint64_t *counts_host, uint64_t *n_pairs, uint64_t kSlice)
{
    cudaStream_t s = ctx->stream;
    // Slices of kSlice points flow through four streams: copy-in of slice
    // k + 1 (in_stream), resolve of slice k (stream), emit of slice k - 1 into
    // device staging (emit_stream) and copy-out of the slice before
    // (out_stream).  Slice k's pairs start at base[k] = base[k - 1] +
    // total[k - 1], computed on the device; the host reads (base[k], total[k])
    // to size the slice's copy-out.  Both copy directions run on the copy
    // engines, beside the kernels.
    const uint64_t n_slices = (n + kSlice - 1) / kSlice;
    const uint64_t cpts = join_chunk_points(), nchunks = (n + cpts - 1) / cpts;
    const size_t b_res = ((n * 4 + 15) & ~uint64_t(15)), words = nchunks + join_part_words(kSlice) + 2 * n_slices + 2;
    spx_status st;
    if ((st = ensure(ctx, &ctx->st_pts, &ctx->st_pts_b, n * 8 + 16, s, "join_host")) != SPX_OK ||
        (st = ensure(ctx, &ctx->st_pairs, &ctx->st_pairs_b, cap * 8 + 16, s, "join_host")) != SPX_OK ||
        (st = ensure(ctx, &ctx->st_counts, &ctx->st_counts_b, size_t(ix->view.P) * 8 + 16, s, "join_host")) != SPX_OK ||
        (st = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, b_res + words * 8, s, "join_host")) != SPX_OK)
        return st;
    while (ctx->slice_ev.size() < 3 * n_slices + 1) {
        cudaEvent_t e = nullptr;
        SPX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "join_host event");
        ctx->slice_ev.push_back(e);
    }
    if (ctx->slice_words_n < 2 * n_slices + 2) {
        cudaFreeHost(ctx->slice_words);
        ctx->slice_words = nullptr;
        ctx->slice_words_n = 0;
        SPX_CUDA(cudaMallocHost(reinterpret_cast<void **>(&ctx->slice_words), (2 * n_slices + 2) * 8),
                 "join_host pinned words");
        ctx->slice_words_n = 2 * n_slices + 2;
    }
    cudaEvent_t *ev_in = ctx->slice_ev.data(), *ev_res = ev_in + n_slices, *ev_emit = ev_res + n_slices;
    uint32_t *res = static_cast<uint32_t *>(ctx->scratch);
    unsigned long long *chunk_tot = reinterpret_cast<unsigned long long *>(static_cast<char *>(ctx->scratch) + b_res);
    unsigned long long *part = chunk_tot + nchunks;
    unsigned long long *bt = part + join_part_words(kSlice); // (base[k], total[k]) pairs, then base[n_slices]
    SPX_CUDA(cudaMemsetAsync(bt, 0, 8, s), "join_host base");
    if (ix->view.P)
        SPX_CUDA(cudaMemsetAsync(ctx->st_counts, 0, size_t(ix->view.P) * 8, s), "join_host counts");
    for (uint64_t k = 0; k < n_slices; ++k) {
        const uint64_t lo = k * kSlice, m = n - lo < kSlice ? n - lo : kSlice;
        SPX_CUDA(cudaMemcpyAsync(static_cast<char *>(ctx->st_pts) + lo * 8, xy_host + 2 * lo, m * 8,
                                 cudaMemcpyHostToDevice, ctx->in_stream),
                 "join_host H2D");
        SPX_CUDA(cudaEventRecord(ev_in[k], ctx->in_stream), "join_host event");
    }
    for (uint64_t k = 0; k < n_slices; ++k) {
        const uint64_t lo = k * kSlice, m = n - lo < kSlice ? n - lo : kSlice;
        JoinLaunch a{};
        a.ix = ix->view;
        a.pts = reinterpret_cast<const int2 *>(static_cast<char *>(ctx->st_pts) + lo * 8);
        a.n = m;
        a.pairs = reinterpret_cast<uint2 *>(ctx->st_pairs);
        a.cap = cap;
        a.counts = reinterpret_cast<unsigned long long *>(ctx->st_counts);
        a.res = res + lo;
        a.tile_tot = chunk_tot + lo / cpts;
        a.total = bt + 2 * k + 1;
        a.err = &ctx->aux->err;
        a.stats = ctx->aux->stats;
        a.fp32 = ix->fp32;
        a.pid0 = uint32_t(lo);
        a.keep_counts = 1;
        a.pair_base = bt + 2 * k;
        // resolve slice k once its points are in; base[k + 1]; (base, total) to the host
        cudaError_t e = cudaStreamWaitEvent(s, ev_in[k], 0);
        if (e == cudaSuccess)
            e = launch_join_resolve(a, part, s);
        if (e == cudaSuccess)
            e = launch_sum_u64(bt + 2 * k + 2, bt + 2 * k, bt + 2 * k + 1, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->slice_words + 2 * k, bt + 2 * k, 16, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaEventRecord(ev_res[k], s);
        // emit slice k into the device staging buffer
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(ctx->emit_stream, ev_res[k], 0);
        if (e == cudaSuccess)
            e = launch_join_emit(a, ctx->emit_stream);
        if (e == cudaSuccess)
            e = cudaEventRecord(ev_emit[k], ctx->emit_stream);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "join_host launch");
    }
    // copy-out, slice by slice, as soon as each slice's size is known
    uint64_t t = 0;
    for (uint64_t k = 0; k < n_slices; ++k) {
        SPX_CUDA(cudaEventSynchronize(ev_res[k]), "join_host slice size");
        const uint64_t b0 = ctx->slice_words[2 * k], tk = ctx->slice_words[2 * k + 1];
        t = b0 + tk;
        const uint64_t hi = t < cap ? t : cap;
        SPX_CUDA(cudaStreamWaitEvent(ctx->out_stream, ev_emit[k], 0), "join_host wait");
        if (b0 < hi)
            SPX_CUDA(cudaMemcpyAsync(pairs_host + 2 * b0, static_cast<char *>(ctx->st_pairs) + b0 * 8, (hi - b0) * 8,
                                     cudaMemcpyDeviceToHost, ctx->out_stream),
                     "join_host D2H");
    }
    cudaEvent_t ev_done = ctx->slice_ev[3 * n_slices];
    SPX_CUDA(cudaEventRecord(ev_done, ctx->out_stream), "join_host event");
    SPX_CUDA(cudaStreamWaitEvent(s, ev_done, 0), "join_host wait");
    if (counts_host && ix->view.P)
        SPX_CUDA(cudaMemcpyAsync(counts_host, ctx->st_counts, size_t(ix->view.P) * 8, cudaMemcpyDeviceToHost, s),
                 "join_host counts D2H");
    if ((st = check_kernel_err(ctx, s)) != SPX_OK)
        return st;
    *n_pairs = t;
    if (t > cap)
        return fail(ctx, SPX_ECAPACITY, "join_host: " + std::to_string(t) + " pairs exceed capacity");
    return SPX_OK;
}

// Can kernels of this device write host memory at p directly (pinned and
// mapped at the same address, managed, or pageable memory that the device
// reaches through the host page tables)?
static bool device_reaches_host(int device, const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) == cudaSuccess) {
        if ((at.type == cudaMemoryTypeHost && at.devicePointer == p) || at.type == cudaMemoryTypeManaged)
            return true;
    } else {
        cudaGetLastError();
    }
    int pageable = 0;
    cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device);
    return pageable == 1;
}

constexpr uint64_t kRing = 4; // device slots of a streamed host table

// Tables larger than device memory (§5.3 "Out-of-Core Queries"): the points
// cycle through kRing device slots of kSlice points (the copy of slice k + 4
// waits until slice k is emitted), and the pairs go straight into pairs_host,
// which the device writes through the host link.  Device memory does not grow
// with n.
static spx_status join_host_streamed(spx_ctx *ctx, IndexObj *ix, const int32_t *xy_host, uint64_t n,
                                     uint32_t *pairs_host, uint64_t cap, uint64_t *counts_host, uint64_t *n_pairs,
                                     uint64_t kSlice)
{
    cudaStream_t s = ctx->stream;
    const uint64_t n_slices = (n + kSlice - 1) / kSlice;
    const uint64_t cpts = join_chunk_points(), slice_chunks = (kSlice + cpts - 1) / cpts;
    const size_t b_pts = kSlice * 8, b_res = kSlice * 4, b_tot = slice_chunks * 8;
    const size_t words = join_part_words(kSlice) + 2 * n_slices + 2;
    spx_status st;
    if ((st = ensure(ctx, &ctx->st_counts, &ctx->st_counts_b, size_t(ix->view.P) * 8 + 16, s, "join_host")) != SPX_OK ||
        (st = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, kRing * (b_pts + b_res + b_tot) + words * 8 + 256, s,
                     "join_host")) != SPX_OK)
        return st;
    while (ctx->slice_ev.size() < 3 * n_slices + 1) {
        cudaEvent_t e = nullptr;
        SPX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "join_host event");
        ctx->slice_ev.push_back(e);
    }
    cudaEvent_t *ev_in = ctx->slice_ev.data(), *ev_res = ev_in + n_slices, *ev_emit = ev_res + n_slices;
    char *m0 = static_cast<char *>(ctx->scratch);
    char *ring_pts = m0, *ring_res = m0 + kRing * b_pts, *ring_tot = ring_res + kRing * b_res;
    unsigned long long *part = reinterpret_cast<unsigned long long *>(ring_tot + kRing * b_tot);
    unsigned long long *bt = part + join_part_words(kSlice); // (base[k], total[k]) pairs, then base[n_slices]
    SPX_CUDA(cudaMemsetAsync(bt, 0, 8, s), "join_host base");
    if (ix->view.P)
        SPX_CUDA(cudaMemsetAsync(ctx->st_counts, 0, size_t(ix->view.P) * 8, s), "join_host counts");
    // the first copy waits for the zeroing above (the ring may hold a previous call's data)
    cudaEvent_t ev_start = ctx->slice_ev[3 * n_slices];
    SPX_CUDA(cudaEventRecord(ev_start, s), "join_host event");
    SPX_CUDA(cudaStreamWaitEvent(ctx->in_stream, ev_start, 0), "join_host wait");
    for (uint64_t k = 0; k < n_slices; ++k) {
        const uint64_t slot = k % kRing, lo = k * kSlice, m = n - lo < kSlice ? n - lo : kSlice;
        cudaError_t e = cudaSuccess;
        if (k >= kRing)
            e = cudaStreamWaitEvent(ctx->in_stream, ev_emit[k - kRing], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ring_pts + slot * b_pts, xy_host + 2 * lo, m * 8, cudaMemcpyHostToDevice,
                                ctx->in_stream);
        if (e == cudaSuccess)
            e = cudaEventRecord(ev_in[k], ctx->in_stream);
        JoinLaunch a{};
        a.ix = ix->view;
        a.pts = reinterpret_cast<const int2 *>(ring_pts + slot * b_pts);
        a.n = m;
        a.pairs = reinterpret_cast<uint2 *>(pairs_host);
        a.cap = cap;
        a.counts = reinterpret_cast<unsigned long long *>(ctx->st_counts);
        a.res = reinterpret_cast<uint32_t *>(ring_res + slot * b_res);
        a.tile_tot = reinterpret_cast<unsigned long long *>(ring_tot + slot * b_tot);
        a.total = bt + 2 * k + 1;
        a.err = &ctx->aux->err;
        a.stats = ctx->aux->stats;
        a.fp32 = ix->fp32;
        a.pid0 = uint32_t(lo);
        a.keep_counts = 1;
        a.pair_base = bt + 2 * k;
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(s, ev_in[k], 0);
        if (e == cudaSuccess)
            e = launch_join_resolve(a, part, s);
        if (e == cudaSuccess)
            e = launch_sum_u64(bt + 2 * k + 2, bt + 2 * k, bt + 2 * k + 1, s);
        if (e == cudaSuccess)
            e = cudaEventRecord(ev_res[k], s);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(ctx->emit_stream, ev_res[k], 0);
        if (e == cudaSuccess)
            e = launch_join_emit(a, ctx->emit_stream);
        if (e == cudaSuccess)
            e = cudaEventRecord(ev_emit[k], ctx->emit_stream);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "join_host launch");
    }
    cudaEvent_t ev_done = ctx->slice_ev[3 * n_slices];
    SPX_CUDA(cudaEventRecord(ev_done, ctx->emit_stream), "join_host event");
    SPX_CUDA(cudaStreamWaitEvent(s, ev_done, 0), "join_host wait");
    unsigned long long t = 0;
    SPX_CUDA(cudaMemcpyAsync(&t, bt + 2 * n_slices, sizeof(t), cudaMemcpyDeviceToHost, s), "join_host total");
    if (counts_host && ix->view.P)
        SPX_CUDA(cudaMemcpyAsync(counts_host, ctx->st_counts, size_t(ix->view.P) * 8, cudaMemcpyDeviceToHost, s),
                 "join_host counts D2H");
    if ((st = check_kernel_err(ctx, s)) != SPX_OK)
        return st;
    *n_pairs = t;
    if (t > cap)
        return fail(ctx, SPX_ECAPACITY, "join_host: " + std::to_string(t) + " pairs exceed capacity");
    return SPX_OK;
}

spx_status spx_join_host(spx_ctx *ctx, const int32_t *xy_host, uint64_t n, spx_index index, uint32_t *pairs_host,
                         uint64_t cap, uint64_t *counts_host, uint64_t *n_pairs)
{
    if (!ctx || (!xy_host && n) || (!pairs_host && cap) || !n_pairs)
        return fail(ctx, SPX_EINVAL, "join_host: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    IndexObj *ix = lookup(ctx->indexes, index);
    if (!ix || ix->kind != 0)
        return fail(ctx, SPX_EINVAL, "join_host: bad index handle (a polygon index is needed)");
    if (n >= (1ull << 32))
        return fail(ctx, SPX_EINVAL, "join_host: n must be < 2^32");
    for (cudaStream_t *p : {&ctx->in_stream, &ctx->emit_stream, &ctx->out_stream})
        if (!*p)
            SPX_CUDA(cudaStreamCreateWithFlags(p, cudaStreamNonBlocking), "join_host stream");
    const uint64_t slice = uint64_t(1) << ctx->host_slice_log2;
    const bool reach = cap == 0 || device_reaches_host(ctx->device, pairs_host);
    int mode = ctx->host_mode;
    if (mode == 0) {
        // staged when the table, its results and the pairs fit in half the free device memory
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        const uint64_t staged = n * 8 + n * 4 + cap * 8 + (uint64_t(1) << 26);
        mode = (staged <= fr / 2 || !reach) ? 1 : 2;
    }
    if (mode == 2 && !reach)
        return fail(ctx, SPX_EINVAL, "join_host: streaming needs pairs_host that the device can write "
                                     "(pinned memory, or a system whose GPU uses the host page tables)");
    return mode == 1 ? join_host_staged(ctx, ix, xy_host, n, pairs_host, cap, counts_host, n_pairs, slice)
                     : join_host_streamed(ctx, ix, xy_host, n, pairs_host, cap, counts_host, n_pairs, slice);
}

spx_status spx_aggregate_host(spx_ctx *ctx, const int32_t *xy_host, uint64_t n, spx_index index, uint64_t *counts_host)
{
    if (!ctx || (!xy_host && n) || !counts_host)
        return fail(ctx, SPX_EINVAL, "aggregate_host: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    IndexObj *ix = lookup(ctx->indexes, index);
    if (!ix || ix->kind != 0)
        return fail(ctx, SPX_EINVAL, "aggregate_host: bad index handle (a polygon index is needed)");
    cudaStream_t s = ctx->stream;
    if (!ctx->in_stream)
        SPX_CUDA(cudaStreamCreateWithFlags(&ctx->in_stream, cudaStreamNonBlocking), "aggregate_host stream");
    // the points cycle through kRing device slots; counts accumulate on the
    // device.  Without a slice size from the caller, 2^25 points: the count
    // pass has no output to overlap, so larger slices cut the per-slice cost.
    const uint64_t kSlice = uint64_t(1) << (ctx->host_slice_set ? ctx->host_slice_log2 : 25);
    const uint64_t n_slices = (n + kSlice - 1) / kSlice;
    const size_t b_pts = kSlice * 8;
    spx_status st;
    if ((st = ensure(ctx, &ctx->st_counts, &ctx->st_counts_b, size_t(ix->view.P) * 8 + 16, s, "aggregate_host")) !=
            SPX_OK ||
        (st = ensure(ctx, &ctx->scratch, &ctx->scratch_bytes, kRing * b_pts + 256, s, "aggregate_host")) != SPX_OK)
        return st;
    while (ctx->slice_ev.size() < 2 * n_slices + 1) {
        cudaEvent_t e = nullptr;
        SPX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "aggregate_host event");
        ctx->slice_ev.push_back(e);
    }
    cudaEvent_t *ev_in = ctx->slice_ev.data(), *ev_agg = ev_in + n_slices;
    char *ring = static_cast<char *>(ctx->scratch);
    unsigned long long *counts = reinterpret_cast<unsigned long long *>(ctx->st_counts);
    if (ix->view.P)
        SPX_CUDA(cudaMemsetAsync(counts, 0, size_t(ix->view.P) * 8, s), "aggregate_host counts");
    cudaEvent_t ev_start = ctx->slice_ev[2 * n_slices];
    SPX_CUDA(cudaEventRecord(ev_start, s), "aggregate_host event");
    SPX_CUDA(cudaStreamWaitEvent(ctx->in_stream, ev_start, 0), "aggregate_host wait");
    for (uint64_t k = 0; k < n_slices; ++k) {
        const uint64_t slot = k % kRing, lo = k * kSlice, m = n - lo < kSlice ? n - lo : kSlice;
        cudaError_t e = cudaSuccess;
        if (k >= kRing)
            e = cudaStreamWaitEvent(ctx->in_stream, ev_agg[k - kRing], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ring + slot * b_pts, xy_host + 2 * lo, m * 8, cudaMemcpyHostToDevice, ctx->in_stream);
        if (e == cudaSuccess)
            e = cudaEventRecord(ev_in[k], ctx->in_stream);
        JoinLaunch a{};
        a.ix = ix->view;
        a.pts = reinterpret_cast<const int2 *>(ring + slot * b_pts);
        a.n = m;
        a.counts = counts;
        a.err = &ctx->aux->err;
        a.stats = ctx->aux->stats;
        a.fp32 = ix->fp32;
        a.keep_counts = 1;
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(s, ev_in[k], 0);
        if (e == cudaSuccess)
            e = launch_aggregate(a, nullptr, s);
        if (e == cudaSuccess)
            e = cudaEventRecord(ev_agg[k], s);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "aggregate_host launch");
    }
    if (ix->view.P)
        SPX_CUDA(cudaMemcpyAsync(counts_host, counts, size_t(ix->view.P) * 8, cudaMemcpyDeviceToHost, s),
                 "aggregate_host counts D2H");
    return check_kernel_err(ctx, s);
}

spx_status spx_set_host_streaming(spx_ctx *ctx, int mode, int slice_log2)
{
    if (!ctx)
        return SPX_EINVAL;
    if (mode < 0 || mode > 2 || (slice_log2 && (slice_log2 < 16 || slice_log2 > 26)))
        return fail(ctx, SPX_EINVAL, "set_host_streaming: mode 0..2, slice_log2 0 or 16..26");
    ctx->host_mode = mode;
    ctx->host_slice_log2 = slice_log2 ? slice_log2 : SPX_HOST_SLICE_LOG2;
    ctx->host_slice_set = slice_log2 != 0;
    return SPX_OK;
}

struct spx_host_index {
    HostIndex hi;
};

spx_status spx_host_index_build(const int32_t *xy, const uint64_t *ring_off, uint32_t P, int grid_log2,
                                int sub_log2, spx_host_index **out, uint64_t sizes[6])
{
    if (!out || !ring_off || !sizes || (!xy && ring_off[P]))
        return SPX_EINVAL;
    *out = nullptr;
    const int g = grid_log2 ? grid_log2 : default_grid_log2(xy, ring_off, P);
    const int sb = sub_log2 ? sub_log2 : kMaxSubLog2;
    auto h = std::make_unique<spx_host_index>();
    std::string err;
    const int threads = std::max(1u, std::thread::hardware_concurrency());
    if (!build_grid_index(xy, ring_off, P, g, sb, threads, h->hi, err))
        return SPX_EINVAL;
    sizes[0] = h->hi.cell.size();
    sizes[1] = h->hi.fine.size();
    sizes[2] = h->hi.entries.size() / 4;
    sizes[3] = h->hi.edges.size() / 4;
    sizes[4] = uint64_t(g);
    sizes[5] = uint64_t(sb);
    *out = h.release();
    return SPX_OK;
}

spx_status spx_host_index_copy(const spx_host_index *h, uint32_t *coarse, uint32_t *fine, uint32_t *entries,
                               int32_t *edges)
{
    if (!h)
        return SPX_EINVAL;
    if (coarse)
        std::memcpy(coarse, h->hi.cell.data(), h->hi.cell.size() * 4);
    if (fine)
        std::memcpy(fine, h->hi.fine.data(), h->hi.fine.size() * 4);
    if (entries)
        std::memcpy(entries, h->hi.entries.data(), h->hi.entries.size() * 4);
    if (edges)
        std::memcpy(edges, h->hi.edges.data(), h->hi.edges.size() * 4);
    return SPX_OK;
}

void spx_host_index_free(spx_host_index *h) { delete h; }

spx_status spx_host_index_validate(const uint32_t *coarse, uint64_t n_coarse, const uint32_t *fine, uint64_t n_fine,
                                   const uint32_t *entries, uint64_t n_entries, const int32_t *edges,
                                   uint64_t n_edges, int grid_log2, int sub_log2, uint32_t n_polys, char *msg,
                                   uint64_t msg_len)
{
    if (!coarse || !fine || !entries || !edges)
        return SPX_EINVAL;
    std::string err;
    const bool ok = validate_grid_index(coarse, n_coarse, fine, n_fine, entries, n_entries, edges, n_edges, grid_log2,
                                        sub_log2, n_polys, err);
    if (msg && msg_len) {
        const size_t m = std::min<size_t>(err.size(), size_t(msg_len - 1));
        std::memcpy(msg, err.data(), m);
        msg[m] = 0;
    }
    return ok ? SPX_OK : SPX_EINVAL;
}

struct spx_host_disk_index {
    HostDiskIndex hd;
};

spx_status spx_host_disk_index_build(const int32_t *cxy, const int32_t *r, uint32_t Q, int grid_log2,
                                     spx_host_disk_index **out, uint64_t sizes[3])
{
    if (!out || !sizes || (Q && (!cxy || !r)))
        return SPX_EINVAL;
    *out = nullptr;
    if (!check_disks(cxy, r, Q).empty())
        return SPX_EINVAL;
    const int g = grid_log2 ? grid_log2 : default_disk_grid_log2(r, Q);
    auto h = std::make_unique<spx_host_disk_index>();
    std::string err;
    if (!build_disk_index(cxy, r, Q, g, h->hd, err))
        return SPX_EINVAL;
    sizes[0] = h->hd.cell.size();
    sizes[1] = h->hd.entries.size();
    sizes[2] = uint64_t(g);
    *out = h.release();
    return SPX_OK;
}

spx_status spx_host_disk_index_copy(const spx_host_disk_index *h, uint32_t *cell, uint32_t *entries)
{
    if (!h)
        return SPX_EINVAL;
    if (cell)
        std::memcpy(cell, h->hd.cell.data(), h->hd.cell.size() * 4);
    if (entries)
        std::memcpy(entries, h->hd.entries.data(), h->hd.entries.size() * 4);
    return SPX_OK;
}

void spx_host_disk_index_free(spx_host_disk_index *h) { delete h; }

struct spx_host_buffer_edges {
    HostBufferEdges he;
};

spx_status spx_host_buffer_edges_build(const int32_t *xy, const uint64_t *ring_off, uint32_t P, const int32_t *r,
                                       int grid_log2, spx_host_buffer_edges **out, uint64_t sizes[3])
{
    if (!out || !sizes || !ring_off || (P && (!xy || !r)))
        return SPX_EINVAL;
    *out = nullptr;
    if (!check_rings(xy, ring_off, P).empty() || P >= kBufferFull || grid_log2 < 0 || grid_log2 > 12)
        return SPX_EINVAL;
    for (uint32_t q = 0; q < P; ++q)
        if (r[q] < 0 || r[q] >= int32_t(kBox))
            return SPX_EINVAL;
    const int g = grid_log2 ? grid_log2 : default_buffer_grid_log2(xy, ring_off, P, r);
    auto h = std::make_unique<spx_host_buffer_edges>();
    std::string err;
    if (!build_buffer_edges(xy, ring_off, P, r, g, h->he, err))
        return SPX_EINVAL;
    sizes[0] = h->he.cell_off.size();
    sizes[1] = h->he.item_q.size();
    sizes[2] = uint64_t(g);
    *out = h.release();
    return SPX_OK;
}

spx_status spx_host_buffer_edges_copy(const spx_host_buffer_edges *h, uint32_t *cell_off, uint32_t *item_q,
                                      int32_t *item_seg)
{
    if (!h)
        return SPX_EINVAL;
    if (cell_off)
        std::memcpy(cell_off, h->he.cell_off.data(), h->he.cell_off.size() * 4);
    if (item_q && !h->he.item_q.empty())
        std::memcpy(item_q, h->he.item_q.data(), h->he.item_q.size() * 4);
    if (item_seg && !h->he.item_seg.empty())
        std::memcpy(item_seg, h->he.item_seg.data(), h->he.item_seg.size() * 4);
    return SPX_OK;
}

void spx_host_buffer_edges_free(spx_host_buffer_edges *h) { delete h; }

spx_status spx_stats(spx_ctx *ctx, spx_stats_t *out, int reset)
{
    if (!ctx || !out)
        return fail(ctx, SPX_EINVAL, "stats: null argument");
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    SPX_CUDA(cudaDeviceSynchronize(), "stats synchronize");
    unsigned long long v[kStatCount];
    SPX_CUDA(cudaMemcpy(v, ctx->aux->stats, sizeof(v), cudaMemcpyDeviceToHost), "stats read");
    out->points_scanned = v[kStatPoints];
    out->edge_tests = v[kStatTests];
    out->fp32_escalations = v[kStatEscalations];
    out->pairs_emitted = v[kStatPairs];
    out->timed_joins = ctx->timed_joins;
    out->timed_aggregates = ctx->timed_aggs;
    out->ms_resolve = ctx->ms_resolve;
    out->ms_scan = ctx->ms_scan;
    out->ms_emit = ctx->ms_emit;
    out->ms_aggregate = ctx->ms_agg;
    out->ms_walk = ctx->ms_walk;
    out->points_from_directory = v[kStatDirPoints];
    if (reset) {
        SPX_CUDA(cudaMemset(ctx->aux->stats, 0, sizeof(v)), "stats reset");
        ctx->timed_joins = ctx->timed_aggs = 0;
        ctx->ms_resolve = ctx->ms_walk = ctx->ms_scan = ctx->ms_emit = ctx->ms_agg = 0;
    }
    return check_kernel_err(ctx, nullptr);
}

spx_status spx_check_bounded_wait(spx_ctx *ctx, uint32_t tries, void *stream)
{
    if (!ctx)
        return SPX_EINVAL;
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    SPX_CUDA(launch_wait_check(&ctx->aux->err, tries, s), "bounded wait launch");
    return check_kernel_err(ctx, s);
}

spx_status spx_set_phase_timing(spx_ctx *ctx, int on)
{
    if (!ctx)
        return SPX_EINVAL;
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    if (on && !ctx->ev[0])
        for (auto &e : ctx->ev)
            SPX_CUDA(cudaEventCreate(&e), "event create");
    ctx->timing = on != 0;
    return SPX_OK;
}

spx_status spx_free(spx_ctx *ctx, uint64_t handle)
{
    if (!ctx)
        return SPX_EINVAL;
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    const uint64_t tag = handle >> kTagShift;
    if (tag == kTagIndex) {
        IndexObj *ix = lookup(ctx->indexes, handle);
        if (!ix)
            return fail(ctx, SPX_EINVAL, "free: bad index handle");
        cudaDeviceSynchronize();
        for (auto it = ctx->select_graphs.begin(); it != ctx->select_graphs.end();)
            if (std::get<1>(it->first) == handle) {
                cudaGraphExecDestroy(it->second);
                it = ctx->select_graphs.erase(it);
            } else {
                ++it;
            }
        cudaFree(ix->mem);
        cudaFree(ix->mem2);
        PolysObj *pg = lookup(ctx->polys, ix->polys);
        if (pg)
            pg->n_index--;
        ctx->indexes.erase(handle);
        return SPX_OK;
    }
    if (tag == kTagPolys) {
        PolysObj *pg = lookup(ctx->polys, handle);
        if (!pg)
            return fail(ctx, SPX_EINVAL, "free: bad polygon handle");
        if (pg->n_index)
            return fail(ctx, SPX_EINVAL, "free: an index built from this polygon set is still alive");
        ctx->polys.erase(handle);
        return SPX_OK;
    }
    if (tag == kTagPoints) {
        PointsObj *p = lookup(ctx->points, handle);
        if (!p)
            return fail(ctx, SPX_EINVAL, "free: bad points handle");
        cudaDeviceSynchronize();
        for (auto it = ctx->select_graphs.begin(); it != ctx->select_graphs.end();)
            if (std::get<0>(it->first) == handle) {
                cudaGraphExecDestroy(it->second);
                it = ctx->select_graphs.erase(it);
            } else {
                ++it;
            }
        if (p->owned)
            cudaFree(p->dev);
        cudaFree(p->cell_end);
        ctx->points.erase(handle);
        return SPX_OK;
    }
    return fail(ctx, SPX_EINVAL, "free: unknown handle");
}

} // extern "C"
