// sm_103a kernels of libspx: the point-in-polygon join, count aggregate and
// the plain comparison join (SPADE §5.2 selection / join / aggregation: the
// per-point work of the paper's fragment shader -- mask with exact boundary
// tests, additive blend for counts, Map with scan compaction, §5.1).
//
// Per point:
//   coarse word  (y >> sc) << g | (x >> sc)      -- geometric transform to a cell
//   mixed cell   -> fine word of the cell's F x F block
//   resolved word: none / one INSIDE polygon / entry list
//   entry INSIDE -> the point is in the polygon       -- mask, inside pixel
//         BOUNDARY -> crossing parity over the fine row's edges  -- boundary pixel
// The crossing rule is exact: an edge a->b counts iff it straddles y
// ((a.y > y) != (b.y > y)) and the orientation d = (b.x-a.x)(y-a.y) -
// (b.y-a.y)(x-a.x) is nonzero with the sign of b.y - a.y.  The sign of d comes
// from FP32 when |d_f| > 2^-21 (|t1| + |t2|) (forward error bound of the FP32
// evaluation with a factor-2 margin), else from an exact int64 recomputation.
//
// The fused kernel is persistent: each CTA claims 2048-point tiles in order,
// and TMA bulk-copies the NEXT tile's points into shared memory (mbarrier
// completion) while it works on the current one.  Within a tile every thread
// resolves 8 points with independent loads; the few points whose fine cell
// holds an entry list are compacted into a shared-memory queue and walked by
// all threads together, so the edge loops run converged.  The join then scans
// the per-point match counts, gets the tile's output offset by decoupled
// look-back and writes the pairs in point order.
#include "kernels.h"
#include "spx_internal.h"

#include <climits>
#include <cuda_runtime.h>

namespace spx {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;                   // points per thread per tile
constexpr int kTile = kThreads * kItems;    // 2048 points per tile
constexpr uint32_t kTileBytes = kTile * 8;  // 16 KB of points
constexpr int kQueue = 1024;                // list points compacted per tile (more are walked in place)
constexpr int kBufs = 3;                    // tile buffers: working, arriving, staged
constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kPending = 0xffffffffu;
constexpr int kHistMax = 11776;             // polygons counted in shared memory (46 KB)
constexpr size_t kSmemFixed = kBufs * kTileBytes + kQueue * sizeof(uint2);

constexpr unsigned long long kFlagAgg = 1ull << 62;   // tile total published
constexpr unsigned long long kFlagPre = 2ull << 62;   // inclusive prefix published
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr unsigned kSpinLimit = 1u << 22;             // ~ seconds with the back-off below

// ------------------------------------------------------------------- PTX helpers
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// L2 eviction policies: the index stays resident (evict_last) while the
// streamed points pass through (evict_first).
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint32_t ld_idx(const uint32_t *p, uint64_t pol)
{
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint4 ld_idx(const uint4 *p, uint64_t pol)
{
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int4 ld_idx(const int4 *p, uint64_t pol)
{
    int4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
// 1-D bulk copy global -> shared (TMA), completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// ------------------------------------------------------------- the predicate
// sign of d = (bx-ax)(py-ay) - (by-ay)(px-ax)
template <bool FP32>
__device__ __forceinline__ int orient_sign(int ax, int ay, int bx, int by, int px, int py, uint32_t &esc)
{
    const int dx1 = bx - ax, dy1 = py - ay, dy2 = by - ay, dx2 = px - ax;
    if (FP32) {
        const float t1 = __fmul_rn(__int2float_rn(dx1), __int2float_rn(dy1));
        const float t2 = __fmul_rn(__int2float_rn(dy2), __int2float_rn(dx2));
        const float df = __fsub_rn(t1, t2);
        const float E = __fmul_rn(__fadd_rn(fabsf(t1), fabsf(t2)), 4.76837158203125e-07f); // 2^-21
        if (fabsf(df) > E)
            return df > 0.f ? 1 : -1;
        ++esc;
    }
    const long long d = (long long)dx1 * dy1 - (long long)dy2 * dx2;
    return (d > 0) - (d < 0);
}

// Parity of the crossings of the rightward ray from (px, py) with a fine-row
// edge list sorted by max x descending.  Edges are loaded four at a time so
// a list costs one L2 round trip per four edges.
template <bool FP32>
__device__ __forceinline__ uint32_t row_parity(const int4 *__restrict__ e, uint32_t n, int px, int py,
                                               uint32_t &tests, uint32_t &esc, uint64_t pol)
{
    uint32_t par = 0;
    for (uint32_t k = 0; k < n; k += 4) {
        int4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            v[j] = (k + j < n) ? ld_idx(e + k + j, pol) : make_int4(INT_MIN, 0, INT_MIN, 0);
        bool stop = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (stop || max(v[j].x, v[j].z) <= px) {
                stop = true; // this and every later edge ends left of p: no crossing right of p
                continue;
            }
            if ((v[j].y > py) == (v[j].w > py))
                continue; // does not straddle
            if (min(v[j].x, v[j].z) > px) {
                par ^= 1u; // the crossing lies right of p
                continue;
            }
            ++tests;
            const int s = orient_sign<FP32>(v[j].x, v[j].y, v[j].z, v[j].w, px, py, esc);
            par ^= uint32_t((s != 0) & ((s > 0) == (v[j].w > v[j].y)));
        }
        if (stop)
            break;
    }
    return par;
}

__device__ __forceinline__ uint32_t coarse_word(const IndexView &ix, uint32_t px, uint32_t py, uint64_t pol)
{
    return ld_idx(ix.cell + (((py >> ix.sc) << ix.gc) | (px >> ix.sc)), pol);
}
__device__ __forceinline__ uint32_t fine_word(const IndexView &ix, uint32_t w, uint32_t px, uint32_t py,
                                              uint64_t pol)
{
    const uint32_t fm = (1u << ix.sb) - 1;
    return ld_idx(ix.fine + (((w & kPayloadMask) << (2 * ix.sb)) | (((py >> ix.sf) & fm) << ix.sb) |
                             ((px >> ix.sf) & fm)),
                  pol);
}
// Resolved word of an in-box point: kind 0 none, 1 one INSIDE polygon, 2 list.
__device__ __forceinline__ uint32_t resolve(const IndexView &ix, uint32_t px, uint32_t py, uint64_t pol)
{
    const uint32_t w = coarse_word(ix, px, py, pol);
    return (w >> 30) == kCellSub ? fine_word(ix, w, px, py, pol) : w;
}

// One edge's contribution to the crossing parity of (px, py).
template <bool FP32>
__device__ __forceinline__ uint32_t edge_cross(const int4 &v, int px, int py, uint32_t &tests, uint32_t &esc)
{
    if ((v.y > py) == (v.w > py))
        return 0u; // does not straddle
    if (min(v.x, v.z) > px)
        return 1u; // the crossing lies right of p
    if (max(v.x, v.z) <= px)
        return 0u; // the crossing lies at or left of p
    ++tests;
    const int s = orient_sign<FP32>(v.x, v.y, v.z, v.w, px, py, esc);
    return uint32_t((s != 0) & ((s > 0) == (v.w > v.y)));
}

// Membership of (px, py) in one entry's polygon, given the entry's first four
// edges (already loaded; missing ones never straddle).  Longer lists continue
// in row order.
template <bool FP32>
__device__ __forceinline__ uint32_t entry_in(const IndexView &ix, const uint4 &en, const int4 (&v)[4], int px, int py,
                                             uint32_t &tests, uint32_t &esc, uint64_t pol)
{
    if (!(en.w & kEntBoundary))
        return 1u;
    uint32_t par = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        par ^= edge_cross<FP32>(v[j], px, py, tests, esc);
    if (en.z > 4 && max(v[3].x, v[3].z) > px)
        par ^= row_parity<FP32>(ix.edge + en.y + 4, en.z - 4, px, py, tests, esc, pol);
    return par;
}

// Walk an entry list: number of polygons containing (px, py), smallest id.
// The common case (at most two entries of at most four edges each) takes two
// dependent round trips with every load issued up front and no data-dependent
// branch around a load; longer lists continue one entry at a time.  The entry
// array ends with a sentinel, so reading two entries is always in bounds.
template <bool FP32>
__device__ __forceinline__ uint32_t walk_list(const IndexView &ix, uint32_t e0, int px, int py, uint32_t &first,
                                              uint32_t &tests, uint32_t &esc, uint64_t pol)
{
    const uint4 *e = ix.ent + e0;
    const uint4 en0 = ld_idx(e, pol), en1 = ld_idx(e + 1, pol);
    const bool two = !(en0.w & kEntLast);
    const uint32_t n0 = (en0.w & kEntBoundary) ? en0.z : 0u;
    const uint32_t n1 = (two && (en1.w & kEntBoundary)) ? en1.z : 0u;
    int4 v0[4], v1[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v0[j] = (uint32_t)j < n0 ? ld_idx(ix.edge + en0.y + j, pol) : make_int4(0, 0, 0, 0);
        v1[j] = (uint32_t)j < n1 ? ld_idx(ix.edge + en1.y + j, pol) : make_int4(0, 0, 0, 0);
    }
    uint32_t c = 0;
    if (entry_in<FP32>(ix, en0, v0, px, py, tests, esc, pol)) {
        first = en0.x;
        c = 1;
    }
    if (two) {
        if (entry_in<FP32>(ix, en1, v1, px, py, tests, esc, pol)) {
            if (!c)
                first = en1.x;
            ++c;
        }
        if (!(en1.w & kEntLast)) {
            for (const uint4 *p = e + 2;; ++p) {
                const uint4 en = ld_idx(p, pol);
                if (!(en.w & kEntBoundary) || row_parity<FP32>(ix.edge + en.y, en.z, px, py, tests, esc, pol)) {
                    if (!c)
                        first = en.x;
                    ++c;
                }
                if (en.w & kEntLast)
                    break;
            }
        }
    }
    return c;
}

// Shared-memory histogram update, aggregated over the lanes that add to the
// same polygon (clustered points put many lanes on one counter).
__device__ __forceinline__ void hist_add(uint32_t *h, uint32_t q)
{
    const uint32_t peers = __match_any_sync(__activemask(), q);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1)
        atomicAdd(h + q, (uint32_t)__popc(peers));
}

// Whole predicate for one point (plain kernels, overflow path).
template <bool FP32>
__device__ __forceinline__ uint32_t point_count(const IndexView &ix, int px, int py, uint32_t &first,
                                                uint32_t &tests, uint32_t &esc, uint64_t pol)
{
    if ((unsigned)px >= kBox || (unsigned)py >= kBox)
        return 0;
    const uint32_t w = resolve(ix, (uint32_t)px, (uint32_t)py, pol);
    const uint32_t kind = w >> 30;
    if (kind == kCellEmpty)
        return 0;
    if (kind == kCellInsideOne) {
        first = w & kPayloadMask;
        return 1;
    }
    return walk_list<FP32>(ix, w & kPayloadMask, px, py, first, tests, esc, pol);
}

// Calls f(polygon) for every polygon containing the in-box point (px, py),
// ascending (only called for points with more than one match: their word is a list).
template <bool FP32, class F>
__device__ __forceinline__ void point_emit(const IndexView &ix, int px, int py, uint64_t pol, F f)
{
    uint32_t t = 0, s = 0;
    const uint32_t w = resolve(ix, (uint32_t)px, (uint32_t)py, pol);
    if ((w >> 30) != kCellList)
        return;
    const uint4 *e = ix.ent + (w & kPayloadMask);
    for (;;) {
        const uint4 en = ld_idx(e++, pol);
        if (!(en.w & kEntBoundary) || row_parity<FP32>(ix.edge + en.y, en.z, px, py, t, s, pol))
            f(en.x);
        if (en.w & kEntLast)
            break;
    }
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ void add_stats(unsigned long long *stats, uint32_t pts, uint32_t tests, uint32_t esc,
                                          uint32_t pairs)
{
    const unsigned long long a = warp_sum64(pts), b = warp_sum64(tests), c = warp_sum64(esc), d = warp_sum64(pairs);
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(stats + kStatPoints, a);
        if (b) atomicAdd(stats + kStatTests, b);
        if (c) atomicAdd(stats + kStatEscalations, c);
        if (d) atomicAdd(stats + kStatPairs, d);
    }
}

// Decoupled look-back (single-pass chained scan): after this tile's total is
// published, walk back over predecessor tiles until one has published its
// inclusive prefix.  Each lane reads kLookLanes consecutive predecessors per step, so one
// L2 round trip covers 32 * kLookLanes tiles.  Tiles are claimed in order from
// an atomic counter, so every tile waited on belongs to a CTA that is already
// running and publishes its total without waiting on later tiles: the wait
// always ends.  It is still bounded; on expiry the error word gets kErrTimeout.
constexpr int kLookLanes = 4;

__device__ unsigned long long lookback(unsigned long long *status, uint32_t tile, uint32_t total, unsigned *err)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0)
            st_relaxed(status, kFlagPre | total);
        return 0;
    }
    // (the caller has published this tile's total with kFlagAgg)
    unsigned long long excl = 0;
    long long top = (long long)tile - 1;
    unsigned spins = 0;
    for (;;) {
        // lane l covers tiles top - 4l .. top - 4l - 3 (nearest first)
        unsigned long long s[kLookLanes];
#pragma unroll
        for (int j = 0; j < kLookLanes; ++j) {
            const long long k = top - (long long)(lane * kLookLanes + j);
            s[j] = (k >= 0) ? ld_relaxed(status + k) : kFlagPre;
        }
        // within the lane: the first inclusive prefix, and whether a needed slot is unpublished
        int jp = kLookLanes;
        bool hole = false;
#pragma unroll
        for (int j = kLookLanes - 1; j >= 0; --j)
            if ((s[j] >> 62) == 2)
                jp = j;
#pragma unroll
        for (int j = 0; j < kLookLanes; ++j)
            if (j <= jp && (s[j] >> 62) == 0)
                hole = true;
        const uint32_t pm = __ballot_sync(kFull, jp < kLookLanes);
        // lanes up to the first lane holding a prefix are needed
        const uint32_t need = pm ? ((pm & (0u - pm)) << 1) - 1 : kFull;
        if (__ballot_sync(kFull, hole) & need) {
            if (++spins > kSpinLimit) {
                if (lane == 0)
                    atomicOr(err, kErrTimeout);
                break;
            }
            __nanosleep(32);
            continue;
        }
        unsigned long long v = 0;
        if ((1u << lane) & need) {
#pragma unroll
            for (int j = 0; j < kLookLanes; ++j)
                if (j <= jp)
                    v += s[j] & kValMask;
        }
        excl += warp_sum64(v);
        if (pm)
            break;
        top -= 32 * kLookLanes;
    }
    if (lane == 0)
        st_relaxed(status + tile, kFlagPre | (excl + total));
    return excl;
}

// ------------------------------------------------------------ the tile kernel
// JOIN = true: pairs (sorted) + counts; JOIN = false: counts only (the
// aggregation plan that never materialises the join, §5.2).
//
// Three shared-memory tile buffers rotate: while tile k is worked on, tile
// k+1 is being bulk-copied in, and (join) tile k-1's pairs wait in their own
// buffer for their output offset.  A tile's pairs are staged in place: once
// its points are consumed, pair i of the tile (in point order) is written to
// slot i of the same buffer.  Its total is published at once, and its
// look-back runs during the next tile, by warp 0 while the other warps walk
// that tile's list points; then all threads copy the staged pairs out,
// coalesced.  A tile whose pairs do not fit in place (a point in several
// polygons) takes the look-back at once and writes directly.
template <bool FP32, bool JOIN>
__global__ void __launch_bounds__(kThreads) k_tiles(JoinLaunch a, uint32_t ntiles, int use_hist)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    int2 *s_buf = reinterpret_cast<int2 *>(dsm);                       // kBufs x kTile points (or staged pairs)
    uint2 *s_q = reinterpret_cast<uint2 *>(dsm + kBufs * kTileBytes);  // list-point queue
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(dsm + kSmemFixed); // P counters
    __shared__ __align__(8) uint64_t s_bar[kBufs];
    __shared__ uint32_t s_tile[kBufs];
    __shared__ uint32_t s_qn, s_qj, s_multi;
    __shared__ uint32_t s_off[kItems * kWarps];
    __shared__ uint32_t s_total;
    __shared__ unsigned long long s_excl, s_prev_excl;
    __shared__ uint32_t s_prev_tile, s_prev_total, s_prev_buf; // staged tile waiting for its offset

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const IndexView &ix = a.ix;
    const uint64_t keep = policy_evict_last();
    if (use_hist)
        for (uint32_t i = tid; i < ix.P; i += kThreads)
            s_hist[i] = 0;

    // copy of tile t into buffer b: TMA for the 16-byte part, a plain store for an odd last point
    auto issue = [&](uint32_t t, int b) {
        const uint64_t base = (uint64_t)t * kTile;
        const uint64_t rem = a.n - base;
        const uint32_t np = rem < (uint64_t)kTile ? (uint32_t)rem : (uint32_t)kTile;
        const uint32_t bytes = (np & ~1u) * 8u;
        int2 *dst = s_buf + b * kTile;
        if (np & 1u)
            dst[np - 1] = a.pts[base + np - 1];
        if (bytes) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(&s_bar[b], bytes);
            tma_load_1d(dst, a.pts + base, bytes, &s_bar[b], policy_evict_first());
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&s_bar[b])) : "memory");
        }
    };
    auto claim_next = [&](int b) {
        const uint32_t nt = atomicAdd(a.tile_counter, 1u);
        s_tile[b] = nt;
        if (nt < ntiles)
            issue(nt, b);
    };
    // copy a staged tile's pairs to their final place (all threads)
    auto flush = [&](uint32_t buf, uint32_t total, unsigned long long excl) {
        const uint2 *st = reinterpret_cast<const uint2 *>(s_buf + buf * kTile);
        for (uint32_t j = tid; j < total; j += kThreads)
            if (excl + j < a.cap)
                __stcs(a.pairs + excl + j, st[j]);
    };

    if (tid == 0) {
        for (int b = 0; b < kBufs; ++b)
            mbar_init(&s_bar[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_qn = 0;
        s_qj = 0;
        s_multi = 0;
        s_prev_tile = kPending; // none staged
        claim_next(0);
    }
    __syncthreads();

    uint32_t n_tests = 0, n_esc = 0, n_pts = 0, n_pairs = 0;
    for (uint32_t k = 0;; ++k) {
        const int b = int(k % kBufs);
        const uint32_t tile = s_tile[b];
        if (tile >= ntiles)
            break;
        if (tid == 0)
            claim_next(int((k + 1) % kBufs)); // that buffer's tile (k-2) was flushed during tile k-1
        {
            unsigned spins = 0;
            while (!mbar_try_wait(&s_bar[b], (k / kBufs) & 1u)) {
                if (++spins > kSpinLimit) {
                    if (tid == 0)
                        atomicOr(a.err, kErrCopy);
                    break;
                }
                __nanosleep(20);
            }
        }
        const int2 *tb = s_buf + b * kTile;
        const uint64_t base = (uint64_t)tile * kTile;
        const uint64_t rem = a.n - base;
        const uint32_t npts = rem < (uint64_t)kTile ? (uint32_t)rem : (uint32_t)kTile;

        // resolve every point's word with independent loads
        uint32_t w[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const uint32_t loc = i * kThreads + tid;
            w[i] = 0;
            if (loc < npts) {
                const int2 p = tb[loc];
                ++n_pts;
                if ((unsigned)p.x < kBox && (unsigned)p.y < kBox)
                    w[i] = coarse_word(ix, (uint32_t)p.x, (uint32_t)p.y, keep);
            }
        }
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if ((w[i] >> 30) == kCellSub) {
                const int2 p = tb[i * kThreads + tid];
                w[i] = fine_word(ix, w[i], (uint32_t)p.x, (uint32_t)p.y, keep);
            }
        }
        // one INSIDE polygon: done; a list: into the queue
        uint32_t cnt[kItems], first[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const uint32_t kind = w[i] >> 30;
            cnt[i] = kind == kCellInsideOne ? 1u : 0u;
            first[i] = w[i] & kPayloadMask;
            const bool is_list = kind == kCellList;
            const uint32_t bl = __ballot_sync(kFull, is_list);
            if (bl) {
                const int leader = __ffs(bl) - 1;
                uint32_t slot0 = 0;
                if (lane == leader)
                    slot0 = atomicAdd(&s_qn, (uint32_t)__popc(bl));
                slot0 = __shfl_sync(kFull, slot0, leader);
                if (is_list) {
                    const uint32_t slot = slot0 + __popc(bl & lanemask_lt());
                    const uint32_t loc = i * kThreads + tid;
                    if (slot < (uint32_t)kQueue) {
                        s_q[slot] = make_uint2(loc, w[i] & kPayloadMask);
                        cnt[i] = kPending;
                        first[i] = slot;
                    } else {
                        const int2 p = tb[loc];
                        uint32_t f = 0;
                        cnt[i] = walk_list<FP32>(ix, w[i] & kPayloadMask, p.x, p.y, f, n_tests, n_esc, keep);
                        first[i] = f;
                    }
                }
            }
        }
        __syncthreads();
        // walk the queued list points (dynamic assignment); in a join, warp 0
        // first settles the offset of the tile staged during the previous round
        if (JOIN && warp == 0 && s_prev_tile != kPending) {
            const unsigned long long ex = lookback(a.tile_status, s_prev_tile, s_prev_total, a.err);
            if (lane == 0)
                s_prev_excl = ex;
        }
        {
            const uint32_t qn = min(s_qn, (uint32_t)kQueue);
            for (;;) {
                const uint32_t j = atomicAdd(&s_qj, 1u);
                if (j >= qn)
                    break;
                const uint2 it = s_q[j];
                const int2 p = tb[it.x];
                uint32_t f = 0;
                const uint32_t c = walk_list<FP32>(ix, it.y, p.x, p.y, f, n_tests, n_esc, keep);
                s_q[j] = make_uint2(c, f);
            }
        }
        __syncthreads();
        bool multi = false;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if (cnt[i] == kPending) {
                const uint2 r = s_q[first[i]];
                cnt[i] = r.x;
                first[i] = r.y;
            }
            multi |= cnt[i] > 1;
        }

        if (!JOIN) {
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                if (!cnt[i])
                    continue;
                n_pairs += cnt[i];
                if (cnt[i] == 1) {
                    if (use_hist)
                        hist_add(s_hist, first[i]);
                    else
                        atomicAdd(a.counts + first[i], 1ull);
                } else {
                    const int2 p = tb[i * kThreads + tid];
                    point_emit<FP32>(ix, p.x, p.y, keep, [&](uint32_t q) {
                        if (use_hist)
                            atomicAdd(&s_hist[q], 1u);
                        else
                            atomicAdd(a.counts + q, 1ull);
                    });
                }
            }
            if (tid == 0) {
                s_qn = 0;
                s_qj = 0;
            }
            __syncthreads(); // buffer b and the queue are free for the next tile
            continue;
        }

        // tile-local exclusive offsets of every point's pairs, in point order
        multi = __any_sync(kFull, multi);
        if (multi && lane == 0)
            s_multi = 1;
        uint32_t pre[kItems];
        if (!multi) {
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                const uint32_t bl = __ballot_sync(kFull, cnt[i] != 0);
                pre[i] = __popc(bl & lanemask_lt());
                if (lane == 0)
                    s_off[i * kWarps + warp] = __popc(bl);
            }
        } else {
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                uint32_t inc = cnt[i];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(kFull, inc, o);
                    if (lane >= o)
                        inc += t;
                }
                pre[i] = inc - cnt[i];
                if (lane == 31)
                    s_off[i * kWarps + warp] = inc;
            }
        }
        __syncthreads();
        const bool staged_prev = s_prev_tile != kPending;
        if (warp == 0) {
            static_assert(kItems * kWarps == 64, "one warp scans two values per lane");
            const uint32_t v0 = s_off[2 * lane], v1 = s_off[2 * lane + 1];
            const uint32_t pair_sum = v0 + v1;
            uint32_t inc = pair_sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, inc, o);
                if (lane >= o)
                    inc += t;
            }
            const uint32_t ex = inc - pair_sum;
            const uint32_t tile_total = __shfl_sync(kFull, inc, 31);
            s_off[2 * lane] = ex;
            s_off[2 * lane + 1] = ex + v0;
            if (lane == 0)
                s_total = tile_total;
            if (tile == 0) {
                if (lane == 0) {
                    st_relaxed(a.tile_status, kFlagPre | tile_total);
                    s_excl = 0;
                }
            } else {
                if (lane == 0)
                    st_relaxed(a.tile_status + tile, kFlagAgg | tile_total);
                __syncwarp();
                if (s_multi) { // cannot stage in place: settle the offset now
                    const unsigned long long excl = lookback(a.tile_status, tile, tile_total, a.err);
                    if (lane == 0)
                        s_excl = excl;
                }
            }
        }
        __syncthreads();
        const uint32_t tile_total = s_total;
        const bool stage = !s_multi && tile != 0;
        // the previous round's staged tile goes out now that its offset is known
        if (staged_prev) {
            flush(s_prev_buf, s_prev_total, s_prev_excl);
            if (tid == 0 && s_prev_tile == ntiles - 1 && a.total)
                *a.total = s_prev_excl + s_prev_total;
        }
        if (!stage) {
            // direct writes at the settled offset
            const unsigned long long tbase = s_excl;
            if (tid == 0 && tile == ntiles - 1 && a.total)
                *a.total = tbase + tile_total;
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                if (!cnt[i])
                    continue;
                const uint32_t loc = i * kThreads + tid;
                const uint32_t pid = (uint32_t)(base + loc);
                unsigned long long o = tbase + s_off[i * kWarps + warp] + pre[i];
                n_pairs += cnt[i];
                if (cnt[i] == 1) {
                    if (o < a.cap)
                        __stcs(a.pairs + o, make_uint2(pid, first[i]));
                    if (use_hist)
                        hist_add(s_hist, first[i]);
                    else if (a.counts)
                        atomicAdd(a.counts + first[i], 1ull);
                } else {
                    const int2 p = tb[loc];
                    point_emit<FP32>(ix, p.x, p.y, keep, [&](uint32_t q) {
                        if (o < a.cap)
                            __stcs(a.pairs + o, make_uint2(pid, q));
                        ++o;
                        if (use_hist)
                            atomicAdd(&s_hist[q], 1u);
                        else if (a.counts)
                            atomicAdd(a.counts + q, 1ull);
                    });
                }
            }
        } else {
            // every point has at most one pair and all reads of this buffer's
            // points are done (the barrier above): stage pair i in slot i
            uint2 *st = reinterpret_cast<uint2 *>(s_buf + b * kTile);
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                if (!cnt[i])
                    continue;
                const uint32_t loc = i * kThreads + tid;
                st[s_off[i * kWarps + warp] + pre[i]] = make_uint2((uint32_t)(base + loc), first[i]);
                ++n_pairs;
                if (use_hist)
                    hist_add(s_hist, first[i]);
                else if (a.counts)
                    atomicAdd(a.counts + first[i], 1ull);
            }
        }
        __syncthreads(); // staged pairs complete; the previous staged buffer is free
        if (tid == 0) {
            s_qn = 0;
            s_qj = 0;
            s_multi = 0;
            if (stage) {
                s_prev_tile = tile;
                s_prev_total = tile_total;
                s_prev_buf = (uint32_t)b;
            } else {
                s_prev_tile = kPending;
            }
        }
        __syncthreads();
    }
    // the last staged tile
    if (JOIN) {
        if (warp == 0 && s_prev_tile != kPending) {
            const unsigned long long ex = lookback(a.tile_status, s_prev_tile, s_prev_total, a.err);
            if (lane == 0)
                s_prev_excl = ex;
        }
        __syncthreads();
        if (s_prev_tile != kPending) {
            flush(s_prev_buf, s_prev_total, s_prev_excl);
            if (tid == 0 && s_prev_tile == ntiles - 1 && a.total)
                *a.total = s_prev_excl + s_prev_total;
        }
    }
    add_stats(a.stats, n_pts, n_tests, n_esc, n_pairs);
    if (use_hist && a.counts) {
        __syncthreads();
        for (uint32_t i = tid; i < ix.P; i += kThreads)
            if (s_hist[i])
                atomicAdd(a.counts + i, (unsigned long long)s_hist[i]);
    }
}

// ------------------------------------------------------- plain comparison join
// Exact int64 only; one thread per point; pass 1 counts per 256-point block,
// a one-block scan makes block offsets, pass 2 recounts and writes.  Counts by
// global atomics.
__global__ void __launch_bounds__(kThreads) k_plain_count(JoinLaunch a, unsigned long long *block_cnt)
{
    __shared__ uint32_t s_w[kWarps];
    const uint64_t idx = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    uint32_t c = 0, first = 0, t = 0, e = 0;
    if (idx < a.n) {
        const int2 p = a.pts[idx];
        c = point_count<false>(a.ix, p.x, p.y, first, t, e, policy_evict_last());
    }
    uint32_t s = c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0)
        s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < kWarps; ++w)
            b += s_w[w];
        block_cnt[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(1024) k_plain_scan(unsigned long long *v, uint64_t n, unsigned long long *total)
{
    // exclusive scan of n values by one block: chunks of 1024 with a carried total
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0)
        s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t b = 0; b < n; b += 1024) {
        const uint64_t i = b + threadIdx.x;
        const unsigned long long x = i < n ? v[i] : 0ull;
        unsigned long long inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o)
                inc += t;
        }
        if (lane == 31)
            s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long w = s_w[lane];
            unsigned long long wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long t = __shfl_up_sync(kFull, wi, o);
                if (lane >= o)
                    wi += t;
            }
            s_w[lane] = wi - w;
        }
        __syncthreads();
        const unsigned long long carry = s_carry;
        if (i < n)
            v[i] = carry + s_w[warp] + inc - x;
        __syncthreads();
        if (threadIdx.x == 1023)
            s_carry = carry + s_w[warp] + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total)
        *total = s_carry;
}

__global__ void __launch_bounds__(kThreads) k_plain_write(JoinLaunch a, const unsigned long long *block_off)
{
    __shared__ uint32_t s_w[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t idx = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    uint32_t c = 0, first = 0, t = 0, e = 0;
    int2 p = make_int2(0, 0);
    const uint64_t keep = policy_evict_last();
    if (idx < a.n) {
        p = a.pts[idx];
        c = point_count<false>(a.ix, p.x, p.y, first, t, e, keep);
    }
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, inc, o);
        if (lane >= o)
            inc += v;
    }
    if (lane == 31)
        s_w[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w)
        wpre += s_w[w];
    unsigned long long o = block_off[blockIdx.x] + wpre + inc - c;
    if (c == 1) {
        if (o < a.cap)
            a.pairs[o] = make_uint2((uint32_t)idx, first);
        if (a.counts)
            atomicAdd(a.counts + first, 1ull);
    } else if (c > 1) {
        point_emit<false>(a.ix, p.x, p.y, keep, [&](uint32_t q) {
            if (o < a.cap)
                a.pairs[o] = make_uint2((uint32_t)idx, q);
            ++o;
            if (a.counts)
                atomicAdd(a.counts + q, 1ull);
        });
    }
}

template <bool FP32, bool JOIN>
cudaError_t launch_tiles(const JoinLaunch &a, uint32_t ntiles, int use_hist, cudaStream_t s)
{
    const size_t smem = kSmemFixed + (use_hist ? sizeof(uint32_t) * a.ix.P : 0);
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_tiles<FP32, JOIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(kSmemFixed + sizeof(uint32_t) * kHistMax));
        if (e != cudaSuccess)
            return e;
        if (dev < 64)
            attr_set[dev] = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tiles<FP32, JOIN>, kThreads, smem);
    if (per_sm < 1)
        per_sm = 1;
    int grid = per_sm * device_sm_count();
    if ((uint32_t)grid > ntiles)
        grid = (int)ntiles;
    k_tiles<FP32, JOIN><<<grid, kThreads, smem, s>>>(a, ntiles, use_hist);
    return cudaGetLastError();
}

} // namespace

int device_sm_count()
{
    int dev = 0;
    cudaGetDevice(&dev);
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

size_t join_scratch_bytes(uint64_t n)
{
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    return size_t(ntiles * 8 + 16);
}

size_t plain_scratch_bytes(uint64_t n)
{
    const uint64_t nb = (n + kThreads - 1) / kThreads;
    return size_t(nb * 8 + 16);
}

cudaError_t launch_join(const JoinLaunch &a, void *scratch, cudaStream_t s)
{
    const uint64_t ntiles64 = (a.n + kTile - 1) / kTile;
    if (ntiles64 >= (1ull << 31))
        return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(a.pts) & 15)
        return cudaErrorMisalignedAddress;
    const uint32_t ntiles = uint32_t(ntiles64);
    JoinLaunch b = a;
    b.tile_status = reinterpret_cast<unsigned long long *>(scratch);
    b.tile_counter = reinterpret_cast<unsigned *>(b.tile_status + ntiles);
    cudaError_t e = cudaMemsetAsync(scratch, 0, join_scratch_bytes(a.n), s);
    if (e != cudaSuccess)
        return e;
    if (a.counts && a.ix.P) {
        e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * a.ix.P, s);
        if (e != cudaSuccess)
            return e;
    }
    if (ntiles == 0) {
        if (a.total)
            return cudaMemsetAsync(a.total, 0, sizeof(unsigned long long), s);
        return cudaSuccess;
    }
    const int use_hist = (a.counts != nullptr && a.ix.P <= (uint32_t)kHistMax) ? 1 : 0;
    return a.fp32 ? launch_tiles<true, true>(b, ntiles, use_hist, s) : launch_tiles<false, true>(b, ntiles, use_hist, s);
}

cudaError_t launch_aggregate(const JoinLaunch &a, void *scratch, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * (a.ix.P ? a.ix.P : 1), s);
    if (e != cudaSuccess || a.n == 0)
        return e;
    if (reinterpret_cast<uintptr_t>(a.pts) & 15)
        return cudaErrorMisalignedAddress;
    const uint64_t ntiles64 = (a.n + kTile - 1) / kTile;
    if (ntiles64 >= (1ull << 31))
        return cudaErrorInvalidValue;
    const uint32_t ntiles = uint32_t(ntiles64);
    JoinLaunch b = a;
    b.tile_status = nullptr;
    b.tile_counter = reinterpret_cast<unsigned *>(scratch);
    e = cudaMemsetAsync(scratch, 0, 16, s);
    if (e != cudaSuccess)
        return e;
    const int use_hist = a.ix.P <= (uint32_t)kHistMax ? 1 : 0;
    return a.fp32 ? launch_tiles<true, false>(b, ntiles, use_hist, s) : launch_tiles<false, false>(b, ntiles, use_hist, s);
}

cudaError_t launch_join_plain(const JoinLaunch &a, void *scratch, cudaStream_t s)
{
    const uint64_t nb = (a.n + kThreads - 1) / kThreads;
    if (nb >= (1ull << 31))
        return cudaErrorInvalidValue;
    unsigned long long *block = reinterpret_cast<unsigned long long *>(scratch);
    cudaError_t e;
    if (a.counts && a.ix.P) {
        e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * a.ix.P, s);
        if (e != cudaSuccess)
            return e;
    }
    if (nb == 0) {
        if (a.total)
            return cudaMemsetAsync(a.total, 0, sizeof(unsigned long long), s);
        return cudaSuccess;
    }
    k_plain_count<<<(unsigned)nb, kThreads, 0, s>>>(a, block);
    k_plain_scan<<<1, 1024, 0, s>>>(block, nb, a.total);
    k_plain_write<<<(unsigned)nb, kThreads, 0, s>>>(a, block);
    return cudaGetLastError();
}

} // namespace spx
