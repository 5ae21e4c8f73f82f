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
// The join is a cached two-pass Map (§5.1).  Pass 1 (k_warp) is persistent
// and barrier-free: every warp takes its own 256-point chunks, resolves the
// coarse and fine words of all its points with independent loads, queues the
// few points whose fine cell holds an entry list in a per-warp shared-memory
// queue and walks them 32 at a time, so the edge loops run converged; it
// stores a 4-byte result per point and a pair total per chunk.  A device-wide
// scan turns the totals into offsets, and pass 3 (k_wemit) writes each
// chunk's pairs in point order.  The count aggregate is pass 1 alone.  Serving
// batches (k_multi) and the selection partition (k_part_*) follow.
#include "kernels.h"
#include "spx_internal.h"

#include <algorithm>
#include <climits>
#include <type_traits>
#include <cuda_runtime.h>

namespace spx {
namespace {

#ifndef SPX_TILE_THREADS
#define SPX_TILE_THREADS 256
#endif
constexpr int kThreads = SPX_TILE_THREADS;  // threads per CTA of the persistent kernels
constexpr int kWarps = kThreads / 32;
constexpr int kPlainThreads = 256;          // threads per CTA of the plain kernels
constexpr uint32_t kFull = 0xffffffffu;
// Pass-1 result of a point (4 bytes):
//   kResNone                            in no polygon
//   q (bit 31 clear)                    in exactly polygon q
//   kResMulti | kResCount | c<<20 | q   in c polygons (2 <= c <= 1022), the first q < 2^20
//   kResMulti | q                       in several polygons, the first q (count not stored)
constexpr uint32_t kResNone = 0xffffffffu;
constexpr uint32_t kResMulti = 0x80000000u;
constexpr uint32_t kResCount = 0x40000000u;

__host__ __device__ constexpr uint32_t res_encode(uint32_t cnt, uint32_t first)
{
    return cnt == 0 ? kResNone
                    : cnt == 1 ? first
                               : (cnt <= 1022u && first < (1u << 20)) ? (kResMulti | kResCount | (cnt << 20) | first)
                                                                      : (kResMulti | first);
}
// The narrow form (2 bytes; at most kRes16MaxP polygons), with the row bitmap
// of pass 1 as pass 1b leaves it (a row's bit stays set iff the point is in
// two or more polygons):
//   bit clear: kRes16None (in no polygon) or q (in exactly polygon q)
//   bit set:   c, the number of polygons (2 <= c <= P); the pairs are written
//              by walking the point's list again
constexpr uint16_t kRes16None = 0xffffu;
constexpr int kHistMax = 11776;             // polygons counted in shared memory (46 KB)


// ------------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
// L2 eviction policies: the index stays resident (evict_last) while the
// streamed points pass through (evict_first).
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
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
// Bulk prefetch of `bytes` (a multiple of 16) at p (16-byte aligned) into L2
// by the TMA engine: one instruction, no registers, nothing to wait for.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// mbarrier and 1-D TMA bulk copy (global -> shared) for a warp's own staging
// buffer.  The barrier counts one arrival (the expect_tx of the issuing lane)
// plus the bytes the copy delivers.
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// dst, src 16-byte aligned; bytes a multiple of 16.  The generic-proxy reads
// of dst that came before are ordered before the copy's writes.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Waits for the phase of `bar` with the given parity to complete, at most
// max_tries polls (each may suspend the thread for a short time); false if it
// gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t max_tries)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t t = 0; t < max_tries; ++t) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done)
            return true;
    }
    return false;
}
constexpr uint32_t kWaitTries = 1u << 22; // polls of a bounded wait before it reports kErrTimeout
constexpr int kWaveWords = 64; // shared words per warp of walk_list_wave: the parities of two entries per lane
// Prefetch of the line holding p into L2.
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
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
// edge list sorted by max x descending.  Edges are loaded RW at a time so a
// list costs one L2 round trip per RW edges.
template <bool FP32, int RW = 4>
__device__ __forceinline__ uint32_t row_parity(const int4 *__restrict__ e, uint32_t n, int px, int py,
                                               uint32_t &tests, uint32_t &esc, uint64_t pol)
{
    uint32_t par = 0;
    for (uint32_t k = 0; k < n; k += RW) {
        int4 v[RW];
#pragma unroll
        for (int j = 0; j < RW; ++j)
            v[j] = (k + j < n) ? ld_idx(e + k + j, pol) : make_int4(INT_MIN, 0, INT_MIN, 0);
        bool stop = false;
#pragma unroll
        for (int j = 0; j < RW; ++j) {
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

// Bounds checks of the index walks, compiled in by SPX_BOUNDS_CHECK (a debug
// build): an offset or id read from the index that points outside its array
// sets kErrInternal in the error word, and the walk treats the point as in no
// polygon of that list instead of reading there.  The host reports the word
// as SPX_EKERNEL.  In the default build the checks compile to nothing.
__device__ __forceinline__ bool in_bounds(bool ok, const IndexView &ix)
{
#ifdef SPX_BOUNDS_CHECK
    if (!ok)
        atomicOr(ix.err, kErrInternal);
    return ok;
#else
    (void)ok;
    (void)ix;
    return true;
#endif
}

__device__ __forceinline__ uint32_t coarse_word(const IndexView &ix, uint32_t px, uint32_t py, uint64_t pol)
{
    return ld_idx(ix.cell + (((py >> ix.sc) << ix.gc) | (px >> ix.sc)), pol);
}
__device__ __forceinline__ uint32_t fine_word(const IndexView &ix, uint32_t w, uint32_t px, uint32_t py,
                                              uint64_t pol)
{
    const uint32_t fm = (1u << ix.sb) - 1;
    if (!in_bounds(((uint64_t)(w & kPayloadMask) + 1) << (2 * ix.sb) <= ix.n_fine, ix))
        return 0u;
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

// Calls f(polygon) for every polygon of the entry list starting at e that
// contains (px, py), ascending.  Entries are taken two at a time: both
// entries in one round trip, then the first four edges of each in another
// (the entry array ends with sentinels, so reading two is in bounds).
template <bool FP32, class F>
__device__ __forceinline__ void walk_entries(const IndexView &ix, const uint4 *e, int px, int py, uint32_t &tests,
                                             uint32_t &esc, uint64_t pol, F f)
{
    constexpr int B = 2;
    for (bool more = true; more; e += B) {
        if (!in_bounds((uint64_t)(e - ix.ent) + 1 < ix.n_ent, ix))
            return;
        uint4 en[B];
#pragma unroll
        for (int k = 0; k < B; ++k)
            en[k] = ld_idx(e + k, pol);
#pragma unroll
        for (int k = 0; k < B; ++k)
            if ((k == 0 || !(en[0].w & kEntLast)) &&
                !in_bounds(en[k].x < ix.P && (!(en[k].w & kEntBoundary) || (uint64_t)en[k].y + en[k].z < ix.n_edge),
                           ix))
                return;
        // entries of this list among the B: up to and including the first LAST
        uint32_t live = 0;
#pragma unroll
        for (int k = 0; k < B; ++k) {
            if (more)
                live |= 1u << k;
            if (more && (en[k].w & kEntLast))
                more = false;
        }
        int4 v[B][4];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const uint32_t nk = ((live >> k) & 1u) && (en[k].w & kEntBoundary) ? min(en[k].z, 4u) : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                v[k][j] = ld_idx(ix.edge + ((uint32_t)j < nk ? en[k].y + j : 0u), pol);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((uint32_t)j >= nk)
                    v[k][j] = make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int k = 0; k < B; ++k)
            if (((live >> k) & 1u) && entry_in<FP32>(ix, en[k], v[k], px, py, tests, esc, pol))
                f(en[k].x);
    }
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
    walk_entries<FP32>(ix, ix.ent + (w & kPayloadMask), px, py, t, s, pol, f);
}

// Walk an entry list: number of polygons containing (px, py), smallest id.
// Written so that the lanes of a warp stay converged around every load: the
// common case (at most two entries, at most four edges each) issues all its
// loads unconditionally, from clamped addresses that always lie inside the
// arrays (both end with a sentinel), and selects the results; divergent lanes
// of a warp would otherwise serialise their memory round trips.  Longer lists
// finish in a loop.
template <bool FP32, int RW = 4>
__device__ __forceinline__ uint32_t walk_list(const IndexView &ix, uint32_t e0, int px, int py, uint32_t &first,
                                              uint32_t &tests, uint32_t &esc, uint64_t pol)
{
    if (!in_bounds((uint64_t)e0 + 1 < ix.n_ent, ix))
        return 0u;
    const uint4 *e = ix.ent + e0;
    const uint4 en0 = ld_idx(e, pol), en1 = ld_idx(e + 1, pol);
    const bool two = !(en0.w & kEntLast);
    if (!in_bounds(en0.x < ix.P && (!(en0.w & kEntBoundary) || (uint64_t)en0.y + en0.z < ix.n_edge) &&
                       (!two || (en1.x < ix.P && (!(en1.w & kEntBoundary) || (uint64_t)en1.y + en1.z < ix.n_edge))),
                   ix))
        return 0u;
    const uint32_t n0 = (en0.w & kEntBoundary) ? min(en0.z, 4u) : 0u;
    const uint32_t n1 = (two && (en1.w & kEntBoundary)) ? min(en1.z, 4u) : 0u;
    int4 v0[4], v1[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v0[j] = ld_idx(ix.edge + ((uint32_t)j < n0 ? en0.y + j : 0u), pol);
        v1[j] = ld_idx(ix.edge + ((uint32_t)j < n1 ? en1.y + j : 0u), pol);
    }
    uint32_t p0 = 0, p1 = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t c0 = edge_cross<FP32>(v0[j], px, py, tests, esc);
        const uint32_t c1 = edge_cross<FP32>(v1[j], px, py, tests, esc);
        p0 ^= (uint32_t)j < n0 ? c0 : 0u;
        p1 ^= (uint32_t)j < n1 ? c1 : 0u;
    }
    // lists longer than four edges: the rest, in row order
    if ((en0.w & kEntBoundary) && en0.z > 4 && max(v0[3].x, v0[3].z) > px)
        p0 ^= row_parity<FP32, RW>(ix.edge + en0.y + 4, en0.z - 4, px, py, tests, esc, pol);
    if (two && (en1.w & kEntBoundary) && en1.z > 4 && max(v1[3].x, v1[3].z) > px)
        p1 ^= row_parity<FP32, RW>(ix.edge + en1.y + 4, en1.z - 4, px, py, tests, esc, pol);
    const uint32_t in0 = (en0.w & kEntBoundary) ? p0 : 1u;
    const uint32_t in1 = two ? ((en1.w & kEntBoundary) ? p1 : 1u) : 0u;
    uint32_t c = in0 + in1;
    first = in0 ? en0.x : en1.x;
    if (two && !(en1.w & kEntLast)) {
        // three or more polygons share this fine cell (rare)
        for (const uint4 *q = e + 2;; ++q) {
            if (!in_bounds((uint64_t)(q - ix.ent) < ix.n_ent, ix))
                break;
            const uint4 en = ld_idx(q, pol);
            if (!in_bounds(en.x < ix.P && (!(en.w & kEntBoundary) || (uint64_t)en.y + en.z < ix.n_edge), ix))
                break;
            if (!(en.w & kEntBoundary) || row_parity<FP32>(ix.edge + en.y, en.z, px, py, tests, esc, pol)) {
                if (!c)
                    first = en.x;
                ++c;
            }
            if (en.w & kEntLast)
                break;
        }
    }
    return c;
}

// The polygons of an entry list that contain a point, for the 32 lanes of a
// converged warp at once, each lane with its own point (px, py) and list
// (starting at entry e0; has = false: the lane takes part but has none).
// Calls f(q) on each lane, in ascending q, for every polygon q of its list
// that contains its point.  The entries are taken two per lane per wave (one
// round trip); the edges of all the wave's boundary entries of all lanes are
// then tested by the whole warp, 64 at a time: edge k of the flattened list
// goes to lane k mod 32, which finds the lane that owns it by a binary search
// over the lanes' prefix sums, tests that lane's point, and XORs the crossing
// into that lane's parity in shared memory.  Lanes never loop on their own
// long lists (which would diverge and run one dependent load per step); the
// sorted lists' early stop is not used (an edge that ends left of the point
// counts nothing; recording where each list could stop measured slower).
// s_par: kWaveWords words of shared memory owned by this warp.
template <bool FP32, class F>
__device__ __forceinline__ void walk_list_wave(const IndexView &ix, bool has, uint32_t e0, int px, int py,
                                               uint32_t &tests, uint32_t &esc, uint64_t pol, uint32_t *s_par, F f)
{
    const int lane = threadIdx.x & 31;
    const uint4 *e = ix.ent + (has ? e0 : 0u);
    bool more = has;
    while (__any_sync(kFull, more)) {
        more = more && in_bounds((uint64_t)(e - ix.ent) + 1 < ix.n_ent, ix);
        // two entries (the entry array ends with sentinels: reading e + 1 is in bounds)
        uint4 ea = more ? ld_idx(e, pol) : make_uint4(0, 0, 0, kEntLast);
        const uint4 eb0 = more ? ld_idx(e + 1, pol) : make_uint4(0, 0, 0, kEntLast);
        const bool hb0 = more && !(ea.w & kEntLast);
        if (more && !in_bounds(ea.x < ix.P && (!(ea.w & kEntBoundary) || (uint64_t)ea.y + ea.z < ix.n_edge) &&
                                   (!hb0 || (eb0.x < ix.P &&
                                             (!(eb0.w & kEntBoundary) || (uint64_t)eb0.y + eb0.z < ix.n_edge))),
                               ix)) {
            more = false; // this lane's list ends here
            ea = make_uint4(0, 0, 0, kEntLast);
        }
        const bool hb = more && !(ea.w & kEntLast);
        const uint4 eb = hb ? eb0 : make_uint4(0, 0, 0, kEntLast);
        const uint32_t za = (more && (ea.w & kEntBoundary)) ? ea.z : 0u;
        const uint32_t zb = (hb && (eb.w & kEntBoundary)) ? eb.z : 0u;
        const uint32_t tot = za + zb;
        uint32_t pa = 0, pb = 0;
        if (__any_sync(kFull, tot != 0)) {
            uint32_t incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o)
                    incl += t;
            }
            const uint32_t T = __shfl_sync(kFull, incl, 31);
            s_par[lane] = 0u;
            s_par[32 + lane] = 0u;
            __syncwarp();
            for (uint32_t base = 0; base < T; base += 64) {
                int4 v[2];
                uint32_t slot[2], own[2];
                int ox[2], oy[2];
                bool act[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t k = base + 32 * h + lane;
                    act[h] = k < T;
                    uint32_t o = 0; // the owner: the first lane whose inclusive prefix exceeds k
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1)
                        if (__shfl_sync(kFull, incl, o + step - 1) <= k)
                            o += step;
                    o = act[h] ? o : 0u;
                    const uint32_t oi = __shfl_sync(kFull, incl, o), ot = __shfl_sync(kFull, tot, o);
                    const uint32_t oza = __shfl_sync(kFull, za, o);
                    const uint32_t oya = __shfl_sync(kFull, ea.y, o), oyb = __shfl_sync(kFull, eb.y, o);
                    ox[h] = __shfl_sync(kFull, px, o);
                    oy[h] = __shfl_sync(kFull, py, o);
                    const uint32_t t = k - (oi - ot);
                    slot[h] = t >= oza ? 1u : 0u;
                    own[h] = o;
                    const uint32_t ei = slot[h] ? oyb + (t - oza) : oya + t;
                    v[h] = act[h] ? ld_idx(ix.edge + ei, pol) : make_int4(0, 0, 0, 0); // a zero edge never straddles
                }
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (act[h] && edge_cross<FP32>(v[h], ox[h], oy[h], tests, esc))
                        atomicXor(s_par + 32 * slot[h] + own[h], 1u);
            }
            __syncwarp();
            pa = s_par[lane];
            pb = s_par[32 + lane];
            __syncwarp(); // s_par is rewritten by the next wave
        }
        if (more && (!(ea.w & kEntBoundary) || pa))
            f(ea.x);
        if (hb && (!(eb.w & kEntBoundary) || pb))
            f(eb.x);
        more = hb && !(eb.w & kEntLast);
        e += 2;
    }
}

// Shared-memory histogram update for one item of every lane of a converged
// warp (lanes with has = false add nothing).  Clustered points often put the
// whole warp on one polygon: then one atomic adds the lane count.
__device__ __forceinline__ void hist_add_warp(uint32_t *h, bool has, uint32_t q)
{
    const uint32_t m = __ballot_sync(kFull, has);
    if (!m)
        return;
    const uint32_t qmin = __reduce_min_sync(kFull, has ? q : 0xffffffffu);
    const uint32_t qmax = __reduce_max_sync(kFull, has ? q : 0u);
    if (qmin == qmax) {
        if ((int)(threadIdx.x & 31) == __ffs(m) - 1)
            atomicAdd(h + qmin, (uint32_t)__popc(m));
    } else if (has) {
        atomicAdd(h + q, 1u);
    }
}

// Global counter update for one item of every lane of a converged warp (lanes
// with has = false add nothing): one atomic per distinct polygon of the warp,
// so a clustered table's lanes do not serialise on the same counter.
__device__ __forceinline__ void global_add_warp(unsigned long long *cnt, bool has, uint32_t q)
{
    const uint32_t m = __ballot_sync(kFull, has);
    if (!m)
        return;
    // all lanes on one polygon (clustered tables): one atomic, no match
    const uint32_t qmin = __reduce_min_sync(kFull, has ? q : 0xffffffffu);
    const uint32_t qmax = __reduce_max_sync(kFull, has ? q : 0u);
    if (qmin == qmax) {
        if ((int)(threadIdx.x & 31) == __ffs(m) - 1)
            atomicAdd(cnt + qmin, (unsigned long long)__popc(m));
        return;
    }
    const uint32_t peers = __match_any_sync(kFull, has ? q : 0xffffffffu);
    if (has && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
        atomicAdd(cnt + q, (unsigned long long)__popc(peers));
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

// ------------------------------------------------------- plain comparison join
// Exact int64 only; one thread per point; pass 1 counts per 256-point block,
// a one-block scan makes block offsets, pass 2 recounts and writes.  Counts by
// global atomics.
__global__ void __launch_bounds__(kPlainThreads) k_plain_count(JoinLaunch a, unsigned long long *block_cnt)
{
    __shared__ uint32_t s_w[(kPlainThreads / 32)];
    const uint64_t idx = (uint64_t)blockIdx.x * kPlainThreads + threadIdx.x;
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
        for (int w = 0; w < (kPlainThreads / 32); ++w)
            b += s_w[w];
        block_cnt[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(1024) k_scan(unsigned long long *v, uint64_t n, unsigned long long *total)
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

// Device-wide exclusive scan for long arrays: per-chunk sums, a one-block scan
// of the sums, then every chunk rescanned from its base.
constexpr int kScanItems = 8;
constexpr uint64_t kScanChunk = 1024 * kScanItems;

__device__ __forceinline__ unsigned long long block_exclusive_scan_1024(unsigned long long x, unsigned long long &total,
                                                                        unsigned long long *s_w)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
        if (lane == 31)
            s_w[32] = wi;
    }
    __syncthreads();
    total = s_w[32];
    const unsigned long long ex = s_w[warp] + inc - x;
    __syncthreads();
    return ex;
}

__global__ void __launch_bounds__(1024) k_scan_partials(const unsigned long long *v, uint64_t n,
                                                        unsigned long long *part)
{
    __shared__ unsigned long long s_w[33];
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanChunk + (uint64_t)threadIdx.x * kScanItems;
    unsigned long long sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        sum += (b0 + j < n) ? v[b0 + j] : 0ull;
    unsigned long long total;
    block_exclusive_scan_1024(sum, total, s_w);
    if (threadIdx.x == 0)
        part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_apply(unsigned long long *v, uint64_t n,
                                                     const unsigned long long *part_off)
{
    __shared__ unsigned long long s_w[33];
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanChunk + (uint64_t)threadIdx.x * kScanItems;
    unsigned long long x[kScanItems], sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        x[j] = (b0 + j < n) ? v[b0 + j] : 0ull;
        sum += x[j];
    }
    unsigned long long total;
    unsigned long long run = part_off[blockIdx.x] + block_exclusive_scan_1024(sum, total, s_w);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (b0 + j < n)
            v[b0 + j] = run;
        run += x[j];
    }
}

__device__ __forceinline__ uint32_t warp_sum32(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// ---------------------------------------------- count-only aggregate
// The count-only aggregation that never materialises the join (§5.2 "Spatial
// Aggregations").  No CTA barrier in its loop: every warp works alone on
// chunks of 32 x kWItems consecutive points (chunk c goes to warp c mod
// #warps), loads its points with coalesced 8-byte loads, resolves the coarse
// and fine words of all of a lane's points with independent loads, and queues
// its list points in a per-warp shared-memory queue that it walks 32 at a time
// once the whole chunk is resolved (the chunk's points and words are dead by
// then, which keeps the kernel at 64 registers and 4 CTAs per SM).  A warp
// never waits for another warp, so a slow walk or an index miss only stalls
// its own warp.  The chunks (256 points) are those of the join's passes.
#ifndef SPX_WARP_ITEMS
#define SPX_WARP_ITEMS 8
#endif
#ifndef SPX_WARP_MIN_BLOCKS
#define SPX_WARP_MIN_BLOCKS 4
#endif
constexpr int kWItems = SPX_WARP_ITEMS; // points per lane per chunk (8: 256-point chunks)
constexpr int kWChunk = 32 * kWItems;   // consecutive points per warp chunk
constexpr int kWQueue = kWChunk;        // list points queued per warp: a whole chunk
// per warp: the queue, then the words of walk_list_wave
constexpr size_t kWarpSmem = size_t(kWarps) * (kWQueue * sizeof(uint4) + kWaveWords * sizeof(uint32_t));

// With DIR (a cell-clustered table and its directory, the directory grid at
// least as fine as the coarse grid), k_agg_cells has already counted every
// point of a coarse cell INSIDE one polygon from the cell's row range, and
// marked the chunks that hold points of mixed coarse cells: the others are
// skipped unread, and INSIDE coarse words count nothing here.
template <bool FP32, bool CLUSTERED, bool DIR = false>
__global__ void __launch_bounds__(kThreads, SPX_WARP_MIN_BLOCKS)
    k_warp(JoinLaunch a, uint32_t nchunks, int use_hist, const uint32_t *chunk_mask)
{
    extern __shared__ __align__(16) unsigned char s_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4 *s_q = reinterpret_cast<uint4 *>(s_raw) + warp * kWQueue; // (x, y, first entry, chunk index)
    uint32_t *s_par = reinterpret_cast<uint32_t *>(s_raw + size_t(kWarps) * kWQueue * sizeof(uint4)) + warp * kWaveWords;
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_raw + kWarpSmem);
    const IndexView &ix = a.ix;
    const uint64_t keep = policy_evict_last();
    const bool hist = use_hist && a.counts;
    if (hist)
        for (uint32_t i = threadIdx.x; i < ix.P; i += kThreads)
            s_hist[i] = 0;
    __syncthreads();
    uint32_t n_tests = 0, n_esc = 0, n_pts = 0, n_pairs = 0;
    // count one polygon for every lane with has (converged warp)
    auto count1 = [&](bool has, uint32_t q) {
        if (!a.counts)
            return;
        if (!hist)
            global_add_warp(a.counts, has, q);
        else if (CLUSTERED) // lanes mostly share a counter: one atomic per distinct polygon
            hist_add_warp(s_hist, has, q);
        else if (has) // lanes mostly hit different counters: one atomic each, no vote
            atomicAdd(s_hist + q, 1u);
    };
    const uint32_t nw = gridDim.x * kWarps;
    for (uint32_t ch = blockIdx.x * kWarps + warp; ch < nchunks; ch += nw) {
        if (DIR && !((chunk_mask[ch >> 5] >> (ch & 31)) & 1u))
            continue; // no point of a mixed coarse cell here
        const uint64_t base = (uint64_t)ch * kWChunk;
        const uint32_t npts = (uint32_t)min((uint64_t)kWChunk, a.n - base);
        int2 p[kWItems];
        uint32_t w[kWItems];
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            const uint32_t loc = j * 32 + lane;
            p[j] = loc < npts ? __ldcs(a.pts + base + loc) : make_int2(-1, -1);
            n_pts += (!DIR && loc < npts) ? 1u : 0u;
        }
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            const bool ok = (unsigned)p[j].x < kBox && (unsigned)p[j].y < kBox;
            const uint32_t cw = coarse_word(ix, ok ? (uint32_t)p[j].x : 0u, ok ? (uint32_t)p[j].y : 0u, keep);
            w[j] = ok ? cw : 0u;
            if (DIR) { // INSIDE and empty coarse cells were counted from the directory
                n_pts += ok && (cw >> 30) == kCellSub ? 1u : 0u;
                w[j] = (cw >> 30) == kCellSub ? w[j] : 0u;
            }
        }
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            const bool sub = (w[j] >> 30) == kCellSub;
            if (sub)
                w[j] = fine_word(ix, w[j], (uint32_t)p[j].x, (uint32_t)p[j].y, keep);
        }
        uint32_t total = 0, qn = 0;
        // walk m <= 32 queued points starting at k0, one per lane
        auto walk = [&](uint32_t k0, uint32_t m) {
            __syncwarp();
            const bool has = (uint32_t)lane < m;
            const uint4 it = s_q[k0 + (has ? lane : 0)]; // idle lanes walk nothing
            // the warp walks its lanes' lists together; a point's first polygon is
            // counted with the warp below, any further ones at once
            uint32_t f = 0, c = 0;
            walk_list_wave<FP32>(ix, has, it.z, (int)it.x, (int)it.y, n_tests, n_esc, keep, s_par, [&](uint32_t q) {
                if (c == 0)
                    f = q;
                else if (a.counts)
                    hist ? (void)atomicAdd(s_hist + q, 1u) : (void)atomicAdd(a.counts + q, 1ull);
                ++c;
            });
            total += c;
            count1(c >= 1, f);
            __syncwarp();
        };
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            const uint32_t kind = w[j] >> 30, loc = j * 32 + lane;
            const bool one = kind == kCellInsideOne && in_bounds((w[j] & kPayloadMask) < ix.P, ix),
                       lst = kind == kCellList;
            total += one ? 1u : 0u;
            count1(one, w[j] & kPayloadMask);
            const uint32_t bl = __ballot_sync(kFull, lst);
            if (lst)
                s_q[qn + __popc(bl & lanemask_lt())] =
                    make_uint4((uint32_t)p[j].x, (uint32_t)p[j].y, w[j] & kPayloadMask, loc);
            qn += __popc(bl);
        }
        for (uint32_t k0 = 0; k0 < qn; k0 += 32)
            walk(k0, min(qn - k0, 32u));
        n_pairs += total;
    }
    if (hist) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < ix.P; i += kThreads)
            if (s_hist[i])
                atomicAdd(a.counts + i, (unsigned long long)s_hist[i]);
    }
    add_stats(a.stats, n_pts, n_tests, n_esc, n_pairs);
}

// ---------------------------------------------- join pass 1 as two kernels
// Pass 1a (k_resolve) is the streaming half of the first pass of the Map:
// every warp takes its own 256-point chunks (chunk c goes to warp c mod
// #warps), loads the points with coalesced 8-byte loads, reads the coarse
// word of every point and, in mixed coarse cells, the fine word, all with
// independent loads, and stores each point's result at once: none, its one
// INSIDE polygon (counted here: §4.3, interior pixels need no test), or, for
// a point whose fine cell holds an entry list, the list's first entry.  Those
// points need the exact boundary test.  Pass 1a marks them in a bitmap over
// the rows: the ballot of the list points of a round of 32 rows is the
// bitmap word of those rows.  It stores each chunk's pair total without
// them.  With no walk in it, the kernel is a short stream of independent
// loads and stores that keeps many warps per SM busy.
//
// Pass 1b (k_walk) runs the exact tests of the marked rows (§4.3 boundary
// index): every warp takes a contiguous range of bitmap words, a lane per
// word, gathers the marked rows into its shared-memory queue and walks them
// in full rounds of 32, one row per lane (the point and its stored first
// entry, two independent loads, then the entry list).  It rewrites the row's
// result, adds the row's pairs to its chunk's total and counts them.
#ifndef SPX_RESOLVE_MIN_BLOCKS
#define SPX_RESOLVE_MIN_BLOCKS 8
#endif
constexpr int kResolveMinBlocks = SPX_RESOLVE_MIN_BLOCKS;
#ifndef SPX_WALK_MIN_BLOCKS
#define SPX_WALK_MIN_BLOCKS 3
#endif
constexpr int kWalkMinBlocks = SPX_WALK_MIN_BLOCKS;
constexpr int kWalkQueue = 64; // < 32 rows carried over + one gather step of 32
#ifndef SPX_WALK_BATCH
#define SPX_WALK_BATCH 4
#endif
constexpr int kWalkBatch = SPX_WALK_BATCH;
#ifndef SPX_WALK_RANGE
#define SPX_WALK_RANGE 512
#endif
constexpr int kWalkRange = SPX_WALK_RANGE; // bitmap words (of 32 rows) per warp of pass 1b
static_assert(kWalkRange % (32 * SPX_WALK_BATCH) == 0, "a warp's range is whole steps");

// With the block summary (SUM), a CTA of 1024 threads (one per SM) first
// copies the summary into shared memory; a point whose block is empty or
// INSIDE one polygon is resolved there and reads no index word.  Random
// 4-byte index loads are what bounds this pass (every lane's word lies in
// another cache line, and the L1 looks up one line at a time), and a
// shared-memory lookup costs a fraction of one.
constexpr int kResolveSumThreads = 1024;
#ifndef SPX_PREFETCH_CHUNKS
#define SPX_PREFETCH_CHUNKS 1
#endif
constexpr int kPrefetchChunks = SPX_PREFETCH_CHUNKS; // L2 prefetch distance of pass 1a, in a warp's chunks
#ifndef SPX_TMA_POINTS
#define SPX_TMA_POINTS 1
#endif
constexpr bool kTmaPoints = SPX_TMA_POINTS != 0; // pass 1a stages points with bulk copies when they fit
#ifndef SPX_RESOLVE_PIPE
#define SPX_RESOLVE_PIPE 1
#endif
// pass 1a with the block summary loads a warp's next chunk of points into
// registers before the current chunk's cell words
constexpr bool kResolvePipe = SPX_RESOLVE_PIPE != 0;

// Shared memory of pass 1a: [summary][TMA: per warp a chunk buffer, then per
// warp an mbarrier][counters].
__host__ __device__ constexpr size_t resolve_smem_head(int warps, bool sum, int sg, bool tma)
{
    return (sum ? ((size_t(2) << (2 * sg)) + 15) & ~size_t(15) : 0) +
           (tma ? size_t(warps) * (kWChunk * sizeof(int2) + sizeof(uint64_t)) : 0);
}

// With TMA, every warp stages its next chunk's points in its own shared-memory
// buffer with one bulk copy, issued as soon as it has read the current chunk
// from there: the points arrive while the chunk is resolved, and their loads
// cost the L1 nothing.  A warp's last chunk, when it is not full, is loaded
// with plain loads.
template <int THREADS, bool SUM, bool TMA, bool R16>
__global__ void __launch_bounds__(THREADS, SUM ? 1 : (TMA ? 6 : kResolveMinBlocks))
    k_resolve(const __grid_constant__ JoinLaunch a, uint32_t *pend, uint32_t nchunks, int use_hist)
{
    constexpr int WARPS = THREADS / 32;
    extern __shared__ __align__(16) unsigned char s_raw[];
    const IndexView &ix = a.ix;
    const uint32_t sum_words = SUM ? (1u << (2 * ix.sg)) : 0u; // 16-bit words
    const uint16_t *s_sum = reinterpret_cast<const uint16_t *>(s_raw);
    const size_t sum_bytes = SUM ? ((size_t(sum_words) * 2 + 15) & ~size_t(15)) : 0;
    int2 *s_buf = reinterpret_cast<int2 *>(s_raw + sum_bytes) + (size_t)(threadIdx.x >> 5) * kWChunk;
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(s_raw + sum_bytes + size_t(WARPS) * kWChunk * sizeof(int2)) +
                      (threadIdx.x >> 5);
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_raw + resolve_smem_head(WARPS, SUM, SUM ? ix.sg : 0, TMA));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t keep = policy_evict_last();
    const bool hist = use_hist && a.counts;
    const uint32_t nw = gridDim.x * WARPS;
    auto full = [&](uint32_t c) { return (uint64_t)(c + 1) * kWChunk <= a.n; };
    if constexpr (SUM) {
        uint4 *d = reinterpret_cast<uint4 *>(s_raw);
        for (uint32_t i = threadIdx.x; i < (sum_words + 7) / 8; i += THREADS)
            d[i] = ld_idx(ix.sum + i, keep);
    }
    if constexpr (TMA) {
        const uint32_t c0 = blockIdx.x * WARPS + warp;
        if (lane == 0) {
            mbar_init(s_bar, 1);
            if (c0 < nchunks && full(c0))
                bulk_load(s_buf, a.pts + (uint64_t)c0 * kWChunk, kWChunk * sizeof(int2), s_bar);
        }
    }
    if (hist)
        for (uint32_t i = threadIdx.x; i < ix.P; i += THREADS)
            s_hist[i] = 0;
    __syncthreads();
    uint32_t n_pts = 0, n_pairs = 0, phase = 0;
    constexpr bool PIPE = SUM && !TMA && kResolvePipe;
    int2 pn[kWItems]; // PIPE: the points of this warp's next chunk
    auto load_chunk = [&](uint32_t c, int2(&q)[kWItems]) {
        const uint64_t b = (uint64_t)c * kWChunk;
        const uint32_t m = c < nchunks ? (uint32_t)min((uint64_t)kWChunk, a.n - b) : 0u;
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            const uint32_t loc = j * 32 + lane;
            q[j] = loc < m ? __ldcs(a.pts + b + loc) : make_int2(-1, -1);
        }
    };
    if (PIPE)
        load_chunk(blockIdx.x * WARPS + warp, pn);
    for (uint32_t ch = blockIdx.x * WARPS + warp; ch < nchunks; ch += nw) {
        const uint64_t base = (uint64_t)ch * kWChunk;
        const uint32_t npts = (uint32_t)min((uint64_t)kWChunk, a.n - base);
        const int2 *pts = a.pts + base;
        uint32_t *res = a.res + base;
        uint16_t *res16 = reinterpret_cast<uint16_t *>(a.res) + base;
        int2 p[kWItems];
        uint32_t w[kWItems];
        if (PIPE) {
            if (kPrefetchChunks > 0 && lane == 0) {
                // the chunk after the next goes to L2; the next one to registers now
                const uint64_t nb = base + (uint64_t)(kPrefetchChunks + 1) * nw * kWChunk;
                if (nb + kWChunk <= a.n)
                    prefetch_l2_bulk(a.pts + nb, kWChunk * sizeof(int2));
            }
#pragma unroll
            for (int j = 0; j < kWItems; ++j)
                p[j] = pn[j];
            load_chunk(ch + nw, pn);
        } else if (TMA && npts == kWChunk) {
            if (!mbar_wait(s_bar, phase, kWaitTries)) {
                // the copy did not arrive: report it, give it one more bounded wait, stop
                if (lane == 0)
                    atomicOr(a.err, kErrTimeout);
                mbar_wait(s_bar, phase, kWaitTries);
                break;
            }
            phase ^= 1u;
#pragma unroll
            for (int j = 0; j < kWItems; ++j)
                p[j] = s_buf[j * 32 + lane];
            __syncwarp();
            const uint32_t nx = ch + nw;
            if (lane == 0 && nx < nchunks && full(nx))
                bulk_load(s_buf, a.pts + (uint64_t)nx * kWChunk, kWChunk * sizeof(int2), s_bar);
        } else {
            if (kPrefetchChunks > 0 && lane == 0) {
                // this warp's chunk kPrefetchChunks ahead goes to L2 while this one is resolved
                const uint64_t nb = base + (uint64_t)kPrefetchChunks * nw * kWChunk;
                if (nb + kWChunk <= a.n)
                    prefetch_l2_bulk(a.pts + nb, kWChunk * sizeof(int2));
            }
#pragma unroll
            for (int j = 0; j < kWItems; ++j) {
                const uint32_t loc = j * 32 + lane;
                p[j] = loc < npts ? __ldcs(pts + loc) : make_int2(-1, -1);
            }
        }
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            // x, y >= 0 and both < 2^30 iff their bitwise or is below 2^30
            const bool ok = (uint32_t)(p[j].x | p[j].y) < kBox;
            const uint32_t px = ok ? (uint32_t)p[j].x : 0u, py = ok ? (uint32_t)p[j].y : 0u;
            bool look = ok;
            if (SUM) {
                const uint32_t sv = s_sum[((py >> ix.ssh) << ix.sg) | (px >> ix.ssh)];
                look = ok && sv == kSumMixed;
                w[j] = !ok || sv == kSumEmpty ? 0u : (kCellInsideOne << 30) | sv;
            }
            if (look)
                w[j] = coarse_word(ix, px, py, keep);
            else if (!SUM)
                w[j] = 0u;
        }
#pragma unroll
        for (int j = 0; j < kWItems; ++j)
            if ((w[j] >> 30) == kCellSub)
                w[j] = fine_word(ix, w[j], (uint32_t)p[j].x, (uint32_t)p[j].y, keep);
        uint32_t total = 0, mask = 0;
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            const uint32_t kind = w[j] >> 30, loc = j * 32 + lane, pay = w[j] & kPayloadMask;
            const bool one = kind == kCellInsideOne && in_bounds(pay < ix.P, ix);
            total += one ? 1u : 0u;
            if (a.counts) {
                if (!hist)
                    global_add_warp(a.counts, one, pay);
                else if (one)
                    atomicAdd(s_hist + pay, 1u);
            }
            // one: the polygon; list: its first entry (narrow: none; rewritten
            // by pass 1b); empty: none
            if (loc < npts) {
                if (R16)
                    __stcg(reinterpret_cast<unsigned short *>(res16 + loc),
                           (unsigned short)(kind == kCellInsideOne ? pay : kRes16None));
                else
                    __stcg(res + loc, kind == kCellEmpty ? kResNone : pay);
            }
            const uint32_t bl = __ballot_sync(kFull, kind == kCellList);
            mask = lane == j ? bl : mask;
        }
        if (lane < kWItems)
            __stcg(pend + (uint64_t)ch * kWItems + lane, mask);
        n_pts += lane == 0 ? npts : 0u;
        n_pairs += total;
        total = warp_sum32(total);
        if (lane == 0)
            a.tile_tot[ch] = total; // the chunk's total without its list points; pass 1b adds theirs
    }
    if (hist) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < ix.P; i += THREADS)
            if (s_hist[i])
                atomicAdd(a.counts + i, (unsigned long long)s_hist[i]);
    }
    add_stats(a.stats, n_pts, 0u, 0u, n_pairs);
}

template <bool FP32, bool R16>
__global__ void __launch_bounds__(kThreads, kWalkMinBlocks) k_walk(JoinLaunch a, uint32_t *pend, uint32_t nwords)
{
    __shared__ uint32_t s_qa[kWarps * kWalkQueue];
    __shared__ uint32_t s_pa[kWarps * kWaveWords];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *s_q = s_qa + warp * kWalkQueue; // rows
    uint32_t *s_par = s_pa + warp * kWaveWords;
    const IndexView &ix = a.ix;
    const uint64_t keep = policy_evict_last();
    uint32_t n_tests = 0, n_esc = 0, n_pairs = 0;
    // walk the queued rows [0, m), m <= 32, one per lane
    auto walk = [&](uint32_t m) {
        __syncwarp();
        const bool has = (uint32_t)lane < m;
        const uint32_t row = s_q[has ? lane : 0]; // idle lanes load lane 0's row and walk nothing
        const int2 p = a.pts[row];
        // the list's first entry: stored by pass 1a, or (narrow results) the
        // cell resolved again
        uint32_t e0;
        bool lst = has;
        if (R16) {
            const uint32_t w = resolve(ix, (uint32_t)p.x, (uint32_t)p.y, keep); // a marked row's point is in the box
            e0 = w & kPayloadMask;
            lst = has && in_bounds((w >> 30) == kCellList, ix);
        } else {
            e0 = __ldcg(a.res + row);
        }
        uint32_t f = 0, c = 0;
        uint64_t ids = 0; // R16 and a.aux: the first four polygons, 16 bits each
        walk_list_wave<FP32>(ix, lst, e0, p.x, p.y, n_tests, n_esc, keep, s_par, [&](uint32_t q) {
            if (R16 && c < 4)
                ids |= (uint64_t)q << (16 * c);
            f = c ? f : q;
            ++c;
            if (a.counts)
                atomicAdd(a.counts + q, 1ull);
        });
        n_pairs += c;
        if (has) {
            if (R16) {
                __stcg(reinterpret_cast<unsigned short *>(a.res) + row,
                       (unsigned short)(c == 0 ? kRes16None : c == 1 ? f : c));
                // the row's bit stays set iff the point is in several polygons;
                // only this warp reads or writes the bitmap words of its range
                if (c < 2)
                    atomicAnd(pend + (row >> 5), ~(1u << (row & 31)));
                else if (a.aux && c <= 4)
                    __stcg(reinterpret_cast<unsigned long long *>(a.aux) + row, (unsigned long long)ids);
            } else {
                __stcg(a.res + row, res_encode(c, f));
            }
            if (c)
                atomicAdd(a.tile_tot + row / kWChunk, (unsigned long long)c);
        }
        __syncwarp(); // the queue is rewritten after the round
    };
    constexpr int B = kWalkBatch; // bitmap words per lane per step, the next step's loaded ahead
    const uint64_t w0 = ((uint64_t)blockIdx.x * kWarps + warp) * kWalkRange;
    const uint64_t w1 = min((uint64_t)nwords, w0 + kWalkRange);
    uint32_t qn = 0;
    uint32_t nxt[B];
#pragma unroll
    for (int k = 0; k < B; ++k)
        nxt[k] = w0 + k * 32 + lane < w1 ? __ldcs(pend + w0 + k * 32 + lane) : 0u;
    for (uint64_t wb = w0; wb < w1; wb += 32 * B) {
        uint32_t cur[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            cur[k] = nxt[k];
            const uint64_t wn = wb + 32 * B + k * 32 + lane;
            nxt[k] = wn < w1 ? __ldcs(pend + wn) : 0u;
        }
#pragma unroll 1
        for (int k = 0; k < B; ++k) { // not unrolled: one copy of the walk
            const uint64_t wi = wb + k * 32 + lane;
            uint32_t m = cur[0];
#pragma unroll
            for (int t = 0; t + 1 < B; ++t)
                cur[t] = cur[t + 1];
            while (__any_sync(kFull, m != 0)) {
                const bool has = m != 0;
                const uint32_t b = (uint32_t)__ffs(m) - 1u;
                m &= m - 1u;
                const uint32_t bl = __ballot_sync(kFull, has);
                if (has) {
                    const uint32_t row = (uint32_t)(wi * 32 + b);
                    s_q[qn + __popc(bl & lanemask_lt())] = row;
                    prefetch_l2(a.pts + row); // loaded when its round is walked
                }
                qn += __popc(bl);
                if (qn >= 32) {
                    walk(32);
                    const uint32_t rem = qn - 32; // move the rest (< 32) to the front
                    const uint32_t it = (uint32_t)lane < rem ? s_q[32 + lane] : 0u;
                    __syncwarp();
                    if ((uint32_t)lane < rem)
                        s_q[lane] = it;
                    qn = rem;
                    __syncwarp();
                }
            }
        }
    }
    if (qn)
        walk(qn);
    add_stats(a.stats, 0u, n_tests, n_esc, n_pairs);
}

// Pass 3 of the join with warp chunks: every warp writes the pairs of its
// chunks from the stored per-point results at the chunk's scanned offset.
// Lane order within a round of 32 points, rounds in order: point order.  A
// point in one polygon is written at once; a point in several is queued (its
// row and its offset; its count comes with its stored result), and the warp
// walks its queue 32 points at a time afterwards (all lanes busy, as in pass
// 1), loading the queued points' coordinates then, one independent load per
// lane, to write their pairs.
constexpr size_t kEmitSmem = size_t(kWarps) * kWChunk * (sizeof(uint32_t) + sizeof(unsigned long long)) +
                             size_t(kWarps) * kWaveWords * sizeof(uint32_t);

template <bool FP32, bool R16>
__global__ void __launch_bounds__(kThreads, 3) k_wemit(JoinLaunch a, const unsigned long long *chunk_off,
                                                       uint32_t nchunks, const uint32_t *pend)
{
    extern __shared__ __align__(16) unsigned char s_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long *s_o = reinterpret_cast<unsigned long long *>(s_raw) + warp * kWChunk;
    uint32_t *s_q = reinterpret_cast<uint32_t *>(s_raw + size_t(kWarps) * kWChunk * sizeof(unsigned long long)) +
                    warp * kWChunk; // rows within the chunk
    uint32_t *s_par = reinterpret_cast<uint32_t *>(s_raw + size_t(kWarps) * kWChunk *
                                                               (sizeof(unsigned long long) + sizeof(uint32_t))) +
                      warp * kWaveWords; // words of walk_list_wave
    const uint64_t keep = policy_evict_last();
    const uint32_t nw = gridDim.x * kWarps;
    for (uint32_t ch = blockIdx.x * kWarps + warp; ch < nchunks; ch += nw) {
        const uint64_t base = (uint64_t)ch * kWChunk;
        const uint32_t npts = (uint32_t)min((uint64_t)kWChunk, a.n - base);
        unsigned long long run = chunk_off[ch] + (a.pair_base ? *a.pair_base : 0ull);
        uint32_t res[kWItems], mw = 0;
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            const uint32_t loc = j * 32 + lane;
            if (R16) {
                const uint16_t r = loc < npts ? __ldcs(reinterpret_cast<const unsigned short *>(a.res) + base + loc)
                                              : kRes16None;
                res[j] = r == kRes16None ? kResNone : r;
            } else {
                res[j] = loc < npts ? __ldcs(a.res + base + loc) : kResNone;
            }
        }
        if (R16 && lane < kWItems) // lane j: the bitmap word of round j (rows in several polygons)
            mw = __ldcs(pend + (uint64_t)ch * kWItems + lane);
        uint32_t qn = 0;
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            const uint32_t loc = j * 32 + lane;
            uint32_t r = res[j];
            const uint32_t pid = a.pid0 + (uint32_t)(base + loc);
            bool multi;
            if (R16) {
                multi = (__shfl_sync(kFull, mw, j) >> lane) & 1u;
                if (multi) // the count; the polygons come from walking the list again
                    r = kResMulti | kResCount;
            } else {
                multi = r != kResNone && (r & kResMulti);
            }
            uint32_t c = r == kResNone ? 0u : 1u, pre, tot;
            if (!__any_sync(kFull, multi)) {
                const uint32_t bl = __ballot_sync(kFull, c != 0);
                pre = __popc(bl & lanemask_lt());
                tot = __popc(bl);
            } else {
                if (multi) {
                    if (R16) {
                        c = res[j];
                    } else if (r & kResCount) {
                        c = (r >> 20) & 0x3ffu;
                    } else { // count not stored: count again
                        const int2 p = a.pts[base + loc];
                        uint32_t f = 0, t = 0, e = 0;
                        c = point_count<FP32>(a.ix, p.x, p.y, f, t, e, keep);
                    }
                }
                uint32_t inc = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(kFull, inc, o);
                    if (lane >= o)
                        inc += v;
                }
                pre = inc - c;
                tot = __shfl_sync(kFull, inc, 31);
                // a point whose polygons pass 1b packed: written from them
                const bool packed = R16 && multi && a.aux && c <= 4;
                if (packed) {
                    const unsigned long long ids = __ldcs(reinterpret_cast<const unsigned long long *>(a.aux) + base + loc);
                    for (uint32_t t = 0; t < c; ++t)
                        if (run + pre + t < a.cap)
                            __stcs(a.pairs + run + pre + t, make_uint2(pid, uint32_t(ids >> (16 * t)) & 0xffffu));
                }
                const uint32_t bl = __ballot_sync(kFull, multi && !packed);
                if (multi) {
                    if (!packed) {
                        const uint32_t slot = qn + __popc(bl & lanemask_lt());
                        s_q[slot] = loc;
                        s_o[slot] = run + pre;
                    }
                    c = 0; // written above or from the queue
                }
                qn += __popc(bl);
            }
            if (c) {
                const unsigned long long o = run + pre;
                if (o < a.cap)
                    __stcs(a.pairs + o, make_uint2(pid, r));
            }
            run += tot;
        }
        __syncwarp();
        for (uint32_t k0 = 0; k0 < qn; k0 += 32) {
            // the whole warp walks the queued points' lists together
            const bool has = k0 + lane < qn;
            const uint32_t loc = has ? s_q[k0 + lane] : 0u;
            unsigned long long o = has ? s_o[k0 + lane] : 0ull;
            const int2 p = has ? a.pts[base + loc] : make_int2(0, 0);
            const uint32_t pid = a.pid0 + (uint32_t)(base + loc);
            const uint32_t w = has ? resolve(a.ix, (uint32_t)p.x, (uint32_t)p.y, keep) : 0u;
            uint32_t t = 0, e = 0;
            walk_list_wave<FP32>(a.ix, (w >> 30) == kCellList, w & kPayloadMask, p.x, p.y, t, e, keep, s_par,
                                 [&](uint32_t q) {
                                     if (o < a.cap)
                                         __stcs(a.pairs + o, make_uint2(pid, q));
                                     ++o;
                                 });
        }
        __syncwarp(); // the queue is rewritten by the next chunk
    }
}

// ------------------------------------------------------ multi-request batches
// Serving answers several requests, each with its own index, in one pass over
// the points: the point table is read once per pass for the whole batch
// instead of once per request (the one-pass batched selection of §5.2,
// applied across requests).  Two passes, as in the Map of §5.1: the count pass
// counts every request's pairs per warp chunk (and the join requests'
// per-polygon counts); the per-request chunk totals are scanned; the emit pass
// resolves again and writes every request's pairs in (point, polygon) order
// from its chunk's offset.  As in k_warp, every warp works alone on its
// chunks (loaded once for all requests) and walks list points from a
// per-warp queue; the output never depends on the schedule.
constexpr uint32_t kMPending = 0xffffffffu; // a list point whose walk is queued
#ifndef SPX_MULTI_ITEMS
#define SPX_MULTI_ITEMS 4
#endif
constexpr int kMItems = SPX_MULTI_ITEMS;                      // points per lane per chunk
constexpr int kMChunk = 32 * kMItems;                         // consecutive points per warp chunk
// queues and offsets, then the words of walk_list_wave, per warp
constexpr size_t kMultiSmem =
    size_t(kWarps) * (kMChunk * (sizeof(uint4) + sizeof(unsigned long long)) + kWaveWords * sizeof(uint32_t));

// Does the cover bitmap let (px, py) reach a non-empty coarse cell?  False for
// points outside the box.
__device__ __forceinline__ bool covered(const IndexView &ix, int px, int py)
{
    if ((unsigned)px >= kBox || (unsigned)py >= kBox)
        return false;
    const uint32_t b = (((uint32_t)py >> ix.scv) << ix.cg) | ((uint32_t)px >> ix.scv);
    return (__ldg(ix.cover + (b >> 5)) >> (b & 31)) & 1u;
}

template <bool FP32, bool EMIT>
__global__ void __launch_bounds__(kThreads, 3) k_multi(const __grid_constant__ MultiLaunch m,
                                                    unsigned long long *chunk_tot, uint32_t nchunks, int use_hist)
{
    extern __shared__ __align__(16) unsigned char s_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4 *s_q = reinterpret_cast<uint4 *>(s_raw) + warp * kMChunk; // (x, y, first entry) -> (count, first)
    unsigned long long *s_o = // emit pass: output offsets of queued points
        reinterpret_cast<unsigned long long *>(s_raw + size_t(kWarps) * kMChunk * sizeof(uint4)) + warp * kMChunk;
    uint32_t *s_par = reinterpret_cast<uint32_t *>(
                          s_raw + size_t(kWarps) * kMChunk * (sizeof(uint4) + sizeof(unsigned long long))) +
                      warp * kWaveWords;
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_raw + kMultiSmem); // count pass: qbase[K] counters
    const uint64_t keep = policy_evict_last();
    const int K = m.K;
    uint32_t tests = 0, esc = 0, scanned = 0, emitted = 0;
    if (!EMIT && use_hist)
        for (uint32_t i = threadIdx.x; i < m.qbase[K]; i += kThreads)
            s_hist[i] = 0;
    __syncthreads();
    const uint32_t nw = gridDim.x * kWarps;
    for (uint32_t ch = blockIdx.x * kWarps + warp; ch < nchunks; ch += nw) {
        const uint64_t base = (uint64_t)ch * kMChunk;
        const uint32_t npts = (uint32_t)min((uint64_t)kMChunk, m.n - base);
        int2 p[kMItems];
#pragma unroll
        for (int j = 0; j < kMItems; ++j) {
            const uint32_t loc = j * 32 + lane;
            p[j] = loc < npts ? __ldcs(m.pts + base + loc) : make_int2(-1, -1);
            if (!EMIT)
                scanned += loc < npts ? (uint32_t)K : 0u;
        }
        for (int r = 0; r < K; ++r) {
            const IndexView &ix = m.ix[r];
            uint32_t c[kMItems], f[kMItems];
#pragma unroll
            for (int j = 0; j < kMItems; ++j) {
                const bool ok = covered(ix, p[j].x, p[j].y);
                const uint32_t cw = coarse_word(ix, ok ? (uint32_t)p[j].x : 0u, ok ? (uint32_t)p[j].y : 0u, keep);
                f[j] = ok ? cw : 0u;
            }
#pragma unroll
            for (int j = 0; j < kMItems; ++j) {
                const bool sub = (f[j] >> 30) == kCellSub;
                const uint32_t fw = fine_word(ix, sub ? f[j] : 0u, sub ? (uint32_t)p[j].x : 0u,
                                              sub ? (uint32_t)p[j].y : 0u, keep);
                f[j] = sub ? fw : f[j];
            }
            // one INSIDE polygon: done; a list: queued
            uint32_t qn = 0;
#pragma unroll
            for (int j = 0; j < kMItems; ++j) {
                const uint32_t kind = f[j] >> 30;
                const bool lst = kind == kCellList;
                c[j] = kind == kCellInsideOne ? 1u : 0u;
                const uint32_t bl = __ballot_sync(kFull, lst);
                if (lst) {
                    const uint32_t slot = qn + __popc(bl & lanemask_lt());
                    s_q[slot] = make_uint4((uint32_t)p[j].x, (uint32_t)p[j].y, f[j] & kPayloadMask, 0u);
                    c[j] = kMPending;
                    f[j] = slot;
                } else {
                    f[j] &= kPayloadMask;
                }
                qn += __popc(bl);
            }
            __syncwarp();
            unsigned long long *cnt = m.counts[r];
            uint32_t *h = s_hist + m.qbase[r];
            for (uint32_t k0 = 0; k0 < qn; k0 += 32) {
                const bool has = k0 + lane < qn;
                const uint4 it = s_q[has ? k0 + lane : k0]; // idle lanes walk nothing
                // the warp walks its lanes' lists together; the count pass counts a
                // point's further polygons here, its first one with the warp below
                uint32_t fq = 0, cq = 0, t_l = 0, e_l = 0;
                walk_list_wave<FP32>(ix, has, it.z, (int)it.x, (int)it.y, t_l, e_l, keep, s_par, [&](uint32_t q) {
                    if (cq == 0)
                        fq = q;
                    else if (!EMIT && cnt)
                        use_hist ? (void)atomicAdd(h + q, 1u) : (void)atomicAdd(cnt + q, 1ull);
                    ++cq;
                });
                if (!EMIT) {
                    tests += t_l;
                    esc += e_l;
                }
                __syncwarp();
                if (has)
                    s_q[k0 + lane] = make_uint4(cq, fq, 0u, 0u);
                __syncwarp();
            }
#pragma unroll
            for (int j = 0; j < kMItems; ++j)
                if (c[j] == kMPending) {
                    const uint4 q = s_q[f[j]];
                    c[j] = q.x;
                    f[j] = q.y;
                }
            __syncwarp(); // s_q is rewritten for the next request
            if (!EMIT) {
                uint32_t total = 0;
#pragma unroll
                for (int j = 0; j < kMItems; ++j) {
                    total += c[j];
                    if (!cnt)
                        continue;
                    // the first polygon of every point in any (further ones were counted by the walk)
                    if (!use_hist) // served tables are in row order: lanes rarely share a counter
                        global_add_warp(cnt, c[j] >= 1, f[j]);
                    else if (c[j] >= 1)
                        atomicAdd(h + f[j], 1u);
                }
                total = warp_sum32(total);
                if (lane == 0)
                    chunk_tot[(uint64_t)r * nchunks + ch] = total;
                continue;
            }
            // emit: pairs of request r in point order from the chunk's offset;
            // points in several polygons are queued and walked 32 at a time
            uint2 *out = m.pairs[r];
            const uint64_t cap = m.cap[r];
            unsigned long long run = chunk_tot[(uint64_t)r * nchunks + ch];
            uint32_t mq = 0;
#pragma unroll
            for (int j = 0; j < kMItems; ++j) {
                const uint32_t loc = j * 32 + lane, cj = c[j];
                uint32_t inc = cj;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(kFull, inc, o);
                    if (lane >= o)
                        inc += v;
                }
                const uint32_t wtot = __shfl_sync(kFull, inc, 31);
                const unsigned long long o = run + inc - cj;
                const uint32_t pid = (uint32_t)(base + loc);
                if (cj == 1 && o < cap)
                    out[o] = make_uint2(pid, f[j]);
                const uint32_t bl = __ballot_sync(kFull, cj > 1);
                if (cj > 1) {
                    const uint32_t slot = mq + __popc(bl & lanemask_lt());
                    s_q[slot] = make_uint4((uint32_t)p[j].x, (uint32_t)p[j].y, pid, 0u);
                    s_o[slot] = o;
                }
                mq += __popc(bl);
                emitted += cj;
                run += wtot;
            }
            __syncwarp();
            for (uint32_t k0 = 0; k0 < mq; k0 += 32) {
                // the whole warp walks the queued points' lists together
                const bool has = k0 + lane < mq;
                const uint4 it = has ? s_q[k0 + lane] : make_uint4(0u, 0u, 0u, 0u);
                unsigned long long o = has ? s_o[k0 + lane] : 0ull;
                const uint32_t w = has ? resolve(ix, it.x, it.y, keep) : 0u;
                uint32_t t_l = 0, e_l = 0;
                walk_list_wave<FP32>(ix, (w >> 30) == kCellList, w & kPayloadMask, (int)it.x, (int)it.y, t_l, e_l, keep,
                                     s_par, [&](uint32_t q) {
                                         if (o < cap)
                                             out[o] = make_uint2(it.z, q);
                                         ++o;
                                     });
            }
            __syncwarp(); // s_q is rewritten for the next request
        }
    }
    if (!EMIT && use_hist) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < m.qbase[K]; i += kThreads) {
            const uint32_t v = s_hist[i];
            if (!v)
                continue;
            int r = 0;
            while (r + 1 < K && i >= m.qbase[r + 1])
                ++r;
            atomicAdd(m.counts[r] + (i - m.qbase[r]), (unsigned long long)v);
        }
    }
    add_stats(m.stats, scanned, tests, esc, emitted);
}

// ------------------------------------------------------ batched selection
// Selection of points by many query polygons at once (§5.2 "Spatial
// Selection", one pass over the points for all queries).  The join runs once
// and yields (point, query) pairs in point order; the pairs are then
// partitioned by query, keeping point order: each super-tile of kSuperTile
// pairs counts its pairs per query into a query-major table; an exclusive scan
// of the table in query-major order makes entry (q, s) the output position of
// super-tile s's first pair of query q; the emit kernel writes the point ids.
constexpr int kSuperTile = 32768;
constexpr int kSelMaxQ = 1024;                      // queries per index (shared-memory counters)
constexpr int kSelWarpRange = kSuperTile / kWarps;  // pairs per warp of a super-tile

__global__ void __launch_bounds__(kThreads) k_part_count(const uint2 *__restrict__ pairs,
                                                         const unsigned long long *total, uint64_t cap, uint32_t P,
                                                         unsigned long long *table, uint32_t n_super)
{
    extern __shared__ uint32_t s_cnt[]; // P counters
    for (uint32_t q = threadIdx.x; q < P; q += kThreads)
        s_cnt[q] = 0;
    __syncthreads();
    const unsigned long long n = min(*total, (unsigned long long)cap); // pairs past cap were not written
    const uint64_t base = (uint64_t)blockIdx.x * kSuperTile;
    for (uint32_t j = threadIdx.x; j < (uint32_t)kSuperTile; j += kThreads) {
        const bool has = base + j < n;
        const uint32_t q = has ? __ldcg(&pairs[base + j].y) : 0u;
        hist_add_warp(s_cnt, has, q);
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < P; q += kThreads)
        table[(uint64_t)q * n_super + blockIdx.x] = s_cnt[q];
}

__global__ void __launch_bounds__(kThreads) k_part_emit(const uint2 *__restrict__ pairs,
                                                        const unsigned long long *total, uint32_t P,
                                                        const unsigned long long *table, uint32_t n_super,
                                                        uint32_t *ids, uint64_t cap)
{
    extern __shared__ unsigned long long s_run[]; // kWarps x P running positions
    uint32_t *s_wc = reinterpret_cast<uint32_t *>(s_run + (size_t)kWarps * P); // kWarps x P counts
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t i = threadIdx.x; i < kWarps * P; i += kThreads)
        s_wc[i] = 0;
    __syncthreads();
    const unsigned long long n = min(*total, (unsigned long long)cap); // pairs past cap were not written
    const uint64_t base = (uint64_t)blockIdx.x * kSuperTile + (uint64_t)warp * kSelWarpRange;
    // 1. every warp counts its range per query
    for (uint32_t j = lane; j < (uint32_t)kSelWarpRange; j += 32) {
        const bool has = base + j < n;
        const uint32_t q = has ? __ldcg(&pairs[base + j].y) : 0u;
        hist_add_warp(s_wc + warp * P, has, q);
    }
    __syncthreads();
    // 2. start positions per (warp, query)
    for (uint32_t q = threadIdx.x; q < P; q += kThreads) {
        unsigned long long pos = table[(uint64_t)q * n_super + blockIdx.x];
        for (int w = 0; w < kWarps; ++w) {
            s_run[w * P + q] = pos;
            pos += s_wc[w * P + q];
        }
    }
    __syncthreads();
    // 3. every warp writes its range in pair (= point) order: lanes with the
    //    same query take consecutive positions in lane order
    for (uint32_t j0 = 0; j0 < (uint32_t)kSelWarpRange; j0 += 32) {
        if (base + j0 >= n)
            break;
        const bool has = base + j0 + lane < n;
        const uint2 pr = has ? __ldcg(&pairs[base + j0 + lane]) : make_uint2(0u, 0xffffffffu);
        const uint32_t peers = __match_any_sync(kFull, pr.y);
        const unsigned long long start = has ? s_run[warp * P + pr.y] : 0ull;
        __syncwarp();
        if (has) {
            const unsigned long long o = start + __popc(peers & lanemask_lt());
            if (o < cap)
                ids[o] = pr.x;
            if ((int)lane == __ffs(peers) - 1)
                s_run[warp * P + pr.y] = start + __popc(peers);
        }
        __syncwarp();
    }
}

// offsets[q] = first position of query q (table entry (q, 0)), offsets[P] = total
__global__ void k_sel_offsets(const unsigned long long *table, uint32_t n_super, uint32_t P,
                              const unsigned long long *total, unsigned long long *offsets)
{
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= P; q += gridDim.x * blockDim.x)
        offsets[q] = q < P ? table[(uint64_t)q * n_super] : *total;
}

__global__ void __launch_bounds__(kPlainThreads) k_plain_write(JoinLaunch a, const unsigned long long *block_off)
{
    __shared__ uint32_t s_w[(kPlainThreads / 32)];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t idx = (uint64_t)blockIdx.x * kPlainThreads + threadIdx.x;
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

// ------------------------------------------------------- buffered polygons
// Is (px, py) within distance r of the closed segment v = (a, b)?  With
// d = b - a, w = p - a and t = w . d: the distance is |w| when t <= 0, |p - b|
// when t >= |d|^2, else |d x w| / |d|.  Coordinates lie in [0, 2^30], so every
// product of two differences is below 2^60 in magnitude (int64 sums stay
// exact); the last case compares (d x w)^2 with r^2 |d|^2 as 128-bit
// products.  A zero-length edge takes the first case.
__device__ __forceinline__ bool seg_near(const int4 &v, int px, int py, int64_t r)
{
    const int64_t dx = (int64_t)v.z - v.x, dy = (int64_t)v.w - v.y;
    const int64_t wx = (int64_t)px - v.x, wy = (int64_t)py - v.y, rr = r * r;
    const int64_t t = wx * dx + wy * dy;
    if (t <= 0)
        return wx * wx + wy * wy <= rr;
    const int64_t dd = dx * dx + dy * dy;
    if (t >= dd) {
        const int64_t ux = (int64_t)px - v.z, uy = (int64_t)py - v.w;
        return ux * ux + uy * uy <= rr;
    }
    const int64_t c = dx * wy - dy * wx;
    const uint64_t ca = (uint64_t)(c < 0 ? -c : c);
    const uint64_t lh = __umul64hi(ca, ca), ll = ca * ca;
    const uint64_t rh = __umul64hi((uint64_t)rr, (uint64_t)dd), rl = (uint64_t)rr * (uint64_t)dd;
    return lh < rh || (lh == rh && ll <= rl);
}

// Calls f(q) for every buffered polygon q that the in-box point (px, py)
// meets, ascending, and returns their number: the polygons that contain the
// point (its polygon index's cell, ascending), merged with the polygons of its
// edge-grid cell that have an edge within r[q] of it (the cell's items are
// sorted by polygon, each polygon's edges together; a polygon that contains
// the point needs no edge test).
template <bool FP32, class F>
__device__ __forceinline__ uint32_t buffer_point(const IndexView &ix, const BufferView &bv, int px, int py,
                                                 uint32_t &tests, uint32_t &esc, uint64_t pol, F f)
{
    const uint32_t c = (((uint32_t)py >> bv.sc) << bv.g) | ((uint32_t)px >> bv.sc);
    if (!((__ldg(bv.mask + (c >> 5)) >> (c & 31)) & 1u))
        return 0u; // no edge near the cell, no polygon in it: a small L2-resident screen
    uint32_t k = __ldg(bv.cell_off + c);
    const uint32_t kend = __ldg(bv.cell_off + c + 1);
    if (!in_bounds(k <= kend && kend <= bv.n_items, ix))
        return 0u;
    uint32_t n = 0;
    // the cell's polygons below `bound` that have an edge within r (an item
    // flagged kBufferFull: the polygon's r-region holds the whole cell)
    auto near_below = [&](uint32_t bound) {
        while (k < kend) {
            const uint32_t raw = __ldg(bv.item_q + k), q = raw & ~kBufferFull;
            if (q >= bound || !in_bounds(q < bv.P, ix))
                break;
            bool hit = (raw & kBufferFull) != 0;
            if (hit) {
                ++k;
            } else {
                const int64_t r = __ldg(bv.rad + q);
                for (; k < kend && __ldg(bv.item_q + k) == q; ++k)
                    hit = hit || seg_near(ld_idx(bv.item_seg + k, pol), px, py, r);
            }
            if (hit) {
                f(q);
                ++n;
            }
        }
    };
    auto inside = [&](uint32_t q) {
        near_below(q);
        while (k < kend && (__ldg(bv.item_q + k) & ~kBufferFull) == q) // met already: no test
            ++k;
        f(q);
        ++n;
    };
    const uint32_t w = resolve(ix, (uint32_t)px, (uint32_t)py, pol);
    const uint32_t kind = w >> 30, pay = w & kPayloadMask;
    if (kind == kCellInsideOne && in_bounds(pay < ix.P, ix))
        inside(pay);
    else if (kind == kCellList && in_bounds((uint64_t)pay + 1 < ix.n_ent, ix))
        walk_entries<FP32>(ix, ix.ent + pay, px, py, tests, esc, pol, inside);
    near_below(0xffffffffu);
    return n;
}

// Pass 1: per-point pair counts (kept for pass 2), per-polygon counts, and
// the pair total of every 256-point block (block_cnt null: counts only).
template <bool FP32>
__global__ void __launch_bounds__(kPlainThreads) k_buf_count(BufferLaunch a, uint32_t *pt_cnt,
                                                             unsigned long long *block_cnt)
{
    __shared__ uint32_t s_w[kPlainThreads / 32];
    const uint64_t i = (uint64_t)blockIdx.x * kPlainThreads + threadIdx.x;
    const uint64_t keep = policy_evict_last();
    uint32_t c = 0, t = 0, e = 0;
    if (i < a.n) {
        const int2 p = a.pts[i];
        if ((uint32_t)(p.x | p.y) < kBox)
            c = buffer_point<FP32>(a.ix, a.bv, p.x, p.y, t, e, keep, [&](uint32_t q) {
                if (a.counts)
                    atomicAdd(a.counts + q, 1ull);
            });
        if (pt_cnt)
            pt_cnt[i] = c;
    }
    add_stats(a.stats, i < a.n ? 1u : 0u, t, e, c);
    if (!block_cnt)
        return;
    const uint32_t s = warp_sum32(c);
    if ((threadIdx.x & 31) == 0)
        s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < kPlainThreads / 32; ++w)
            b += s_w[w];
        block_cnt[blockIdx.x] = b;
    }
}

// Pass 2: each point's pairs at its block's scanned offset plus the counts
// of the block's earlier points.
template <bool FP32>
__global__ void __launch_bounds__(kPlainThreads) k_buf_write(BufferLaunch a, const uint32_t *pt_cnt,
                                                             const unsigned long long *block_off)
{
    __shared__ uint32_t s_w[kPlainThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t i = (uint64_t)blockIdx.x * kPlainThreads + threadIdx.x;
    const uint32_t c = i < a.n ? pt_cnt[i] : 0u;
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
    if (!c)
        return;
    unsigned long long o = block_off[blockIdx.x] + wpre + inc - c;
    const int2 p = a.pts[i];
    uint32_t t = 0, e = 0;
    buffer_point<FP32>(a.ix, a.bv, p.x, p.y, t, e, policy_evict_last(), [&](uint32_t q) {
        if (o < a.cap)
            a.pairs[o] = make_uint2((uint32_t)i, q);
        ++o;
    });
}

// Opt a kernel in to the shared memory it needs (once per device).
template <class K>
cudaError_t smem_opt_in(K kernel, size_t bytes, bool (&done)[64])
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && done[dev])
        return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess && dev < 64)
        done[dev] = true;
    return e;
}

template <class K>
int persistent_grid(K kernel, int threads, size_t smem, uint32_t ntiles)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1)
        per_sm = 1;
    int grid = per_sm * device_sm_count();
    if ((uint32_t)grid > ntiles)
        grid = (int)ntiles;
    return grid;
}

template <bool FP32, bool CLUSTERED, bool DIR = false>
cudaError_t launch_warp_kernel(const JoinLaunch &a, int use_hist, cudaStream_t s, const uint32_t *chunk_mask = nullptr)
{
    static bool done[64] = {};
    const uint64_t nchunks = (a.n + kWChunk - 1) / kWChunk;
    if (nchunks >= (1ull << 32))
        return cudaErrorInvalidValue;
    const size_t smem = kWarpSmem + (use_hist ? sizeof(uint32_t) * a.ix.P : 0);
    auto kern = k_warp<FP32, CLUSTERED, DIR>;
    cudaError_t e = smem_opt_in(kern, kWarpSmem + sizeof(uint32_t) * kHistMax, done);
    if (e != cudaSuccess)
        return e;
    const uint32_t nblk = uint32_t((nchunks + kWarps - 1) / kWarps);
    kern<<<persistent_grid(kern, kThreads, smem, nblk), kThreads, smem, s>>>(a, uint32_t(nchunks), use_hist,
                                                                             chunk_mask);
    return cudaGetLastError();
}

// The directory stage of the count aggregate over a cell-clustered table:
// a thread per cell of the directory grid (2^c, c >= g).  A cell inside a
// coarse cell INSIDE one polygon adds its whole row range to that polygon
// (its points need not be read); an empty one adds nothing; one in a mixed
// coarse cell marks the 256-point chunks its range touches, for k_warp<DIR>.
// The points of the cells counted here, and of the bin outside the box, go
// into the scanned-points counter.
__global__ void __launch_bounds__(256) k_agg_cells(const unsigned long long *cell_end, int c, IndexView ix,
                                                   unsigned long long *counts, uint32_t *chunk_mask,
                                                   unsigned long long *stats)
{
    const uint32_t ncell = 1u << (2 * c);
    const int sh = c - ix.gc;
    unsigned long long done_pts = 0;
    for (uint32_t k0 = blockIdx.x * 256 + (threadIdx.x & ~31u); k0 < ncell; k0 += gridDim.x * 256) {
        const uint32_t k = k0 + (threadIdx.x & 31);
        const bool in = k < ncell;
        const unsigned long long s0 = in && k ? cell_end[k - 1] : 0ull, s1 = in ? cell_end[k] : 0ull;
        const bool has = s1 > s0;
        uint32_t w = 0;
        if (has) {
            const uint32_t cx = k & ((1u << c) - 1), cy = k >> c;
            w = ix.cell[((cy >> sh) << ix.gc) | (cx >> sh)];
        }
        const uint32_t kind = w >> 30, q = w & kPayloadMask;
        const bool one = has && kind == kCellInsideOne && in_bounds(q < ix.P, ix);
        done_pts += has && kind != kCellSub ? s1 - s0 : 0ull;
        // counts: one atomic for the warp when its cells share the polygon
        const uint32_t m = __ballot_sync(kFull, one);
        if (m) {
            const uint32_t qmin = __reduce_min_sync(kFull, one ? q : 0xffffffffu);
            const uint32_t qmax = __reduce_max_sync(kFull, one ? q : 0u);
            if (qmin == qmax) {
                const unsigned long long t = warp_sum64(one ? s1 - s0 : 0ull);
                if ((int)(threadIdx.x & 31) == __ffs(m) - 1)
                    atomicAdd(counts + qmin, t);
            } else if (one) {
                atomicAdd(counts + q, s1 - s0);
            }
        }
        if (has && kind == kCellSub) {
            const uint64_t c0 = s0 / kWChunk, c1 = (s1 - 1) / kWChunk;
            for (uint64_t wd = c0 >> 5; wd <= (c1 >> 5); ++wd) {
                const uint64_t lo = max(c0, wd << 5), hi = min(c1, (wd << 5) + 31);
                const uint32_t bits = (hi - lo == 31) ? 0xffffffffu : (((1u << (hi - lo + 1)) - 1u) << (lo & 31));
                atomicOr(chunk_mask + wd, bits);
            }
        }
    }
    // the bin of points outside the box: in no polygon
    if (blockIdx.x == 0 && threadIdx.x == 0)
        done_pts += cell_end[ncell] - cell_end[ncell - 1];
    done_pts = warp_sum64(done_pts);
    if ((threadIdx.x & 31) == 0 && done_pts) {
        atomicAdd(stats + kStatPoints, done_pts);
        atomicAdd(stats + kStatDirPoints, done_pts);
    }
}

// Pass 1 of the join (1a resolve, 1b walk).  pend: 8 words per chunk (the
// bitmap of the rows pass 1b tests).  mid (or null): an event recorded between
// the two kernels.
template <bool FP32>
cudaError_t launch_pass1(const JoinLaunch &a, uint32_t *pend, cudaStream_t s, cudaEvent_t mid)
{
    static bool done_r[8][64] = {};
    const uint64_t nchunks = (a.n + kWChunk - 1) / kWChunk;
    if (a.n >= (1ull << 32))
        return cudaErrorInvalidValue; // rows are 32-bit
    const int use_hist = (a.counts != nullptr && a.ix.P <= (uint32_t)kHistMax) ? 1 : 0;
    const size_t hsm = use_hist ? sizeof(uint32_t) * a.ix.P : 0;
    cudaError_t e;
    if (reinterpret_cast<uintptr_t>(a.pts) & 15)
        return cudaErrorMisalignedAddress; // bulk copies of whole chunks start 16-byte aligned
    // the largest shared memory a CTA may take
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // head: this launch's shared memory before the counters; head_max: the
    // most any launch of the kernel takes (the opt-in, set once per device,
    // must cover every later call, whatever its index)
    auto launch = [&](auto kr, int threads, size_t head, size_t head_max, bool (&done)[64]) -> cudaError_t {
        const size_t smem = head + hsm;
        cudaError_t err =
            smem_opt_in(kr, std::min<size_t>(size_t(smem_max), head_max + sizeof(uint32_t) * kHistMax), done);
        if (err != cudaSuccess)
            return err;
        const uint32_t nblk = uint32_t((nchunks + threads / 32 - 1) / (threads / 32));
        kr<<<persistent_grid(kr, threads, smem, nblk), threads, smem, s>>>(a, pend, uint32_t(nchunks), use_hist);
        return cudaGetLastError();
    };
    constexpr int WS = kResolveSumThreads / 32;
    auto pass1a = [&](auto r16) -> cudaError_t {
        constexpr bool R16 = decltype(r16)::value;
        bool(*d)[64] = done_r + (R16 ? 4 : 0);
        if (a.ix.use_sum) {
            // beside the summary, shared memory holds one chunk buffer per warp
            // at most, too shallow to hide a bulk copy: L2 prefetches instead
            return launch(k_resolve<kResolveSumThreads, true, false, R16>, kResolveSumThreads,
                          resolve_smem_head(WS, true, a.ix.sg, false), resolve_smem_head(WS, true, kSumLog2, false),
                          d[2]);
        }
        const size_t head = kTmaPoints ? resolve_smem_head(kWarps, false, 0, true) : 0;
        if (kTmaPoints)
            return launch(k_resolve<kThreads, false, true, R16>, kThreads, head, head, d[3]);
        return launch(k_resolve<kThreads, false, false, R16>, kThreads, head, head, d[0]);
    };
    e = a.narrow ? pass1a(std::true_type{}) : pass1a(std::false_type{});
    if (e != cudaSuccess) // pass 1b must not run on what an earlier call left in the scratch
        return e;
    if (mid)
        cudaEventRecord(mid, s);
    // pass 1b: a warp per kWalkRange bitmap words, as many CTAs as that takes
    const uint64_t nwords = nchunks * kWItems;
    const uint64_t wblk = (nwords + uint64_t(kWarps) * kWalkRange - 1) / (uint64_t(kWarps) * kWalkRange);
    if (a.narrow)
        k_walk<FP32, true><<<unsigned(wblk), kThreads, 0, s>>>(a, pend, uint32_t(nwords));
    else
        k_walk<FP32, false><<<unsigned(wblk), kThreads, 0, s>>>(a, pend, uint32_t(nwords));
    return cudaGetLastError();
}

// Exclusive scan of n values in place; the total goes to *total.  part: at
// least scan_partials(n) + 1 values of scratch.
uint64_t scan_partials(uint64_t n) { return (n + kScanChunk - 1) / kScanChunk; }

cudaError_t launch_scan(unsigned long long *v, uint64_t n, unsigned long long *total, unsigned long long *part,
                        cudaStream_t s)
{
    if (n <= 4 * kScanChunk) {
        k_scan<<<1, 1024, 0, s>>>(v, n, total);
        return cudaGetLastError();
    }
    const uint64_t nb = scan_partials(n);
    if (nb >= (1ull << 31))
        return cudaErrorInvalidValue;
    k_scan_partials<<<(unsigned)nb, 1024, 0, s>>>(v, n, part);
    k_scan<<<1, 1024, 0, s>>>(part, nb, total);
    k_scan_apply<<<(unsigned)nb, 1024, 0, s>>>(v, n, part);
    return cudaGetLastError();
}

} // namespace

// The bounded wait of pass 1a's bulk-copy staging on a barrier that nothing
// completes (no copy is issued): after `tries` polls it reports kErrTimeout.
__global__ void k_wait_check(unsigned *err, uint32_t tries)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0)
        mbar_init(&bar, 1);
    __syncwarp();
    if (!mbar_wait(&bar, 0, tries) && threadIdx.x == 0)
        atomicOr(err, kErrTimeout);
}

cudaError_t launch_wait_check(unsigned *err, uint32_t tries, cudaStream_t s)
{
    k_wait_check<<<1, 32, 0, s>>>(err, tries);
    return cudaGetLastError();
}

uint64_t scan_part_words(uint64_t n) { return scan_partials(n) + 2; }
cudaError_t launch_exclusive_scan(unsigned long long *v, uint64_t n, unsigned long long *total,
                                  unsigned long long *part, cudaStream_t s)
{
    return launch_scan(v, n, total, part, s);
}

// Deterministic sample for the tuner: dst[i] = src[i * stride], i < m.
__global__ void __launch_bounds__(256) k_gather_stride(const int2 *__restrict__ src, uint64_t stride,
                                                     int2 *__restrict__ dst, uint64_t m)
{
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < m; i += (uint64_t)gridDim.x * 256)
        dst[i] = src[i * stride];
}

cudaError_t launch_gather_stride(const int2 *src, uint64_t n, int2 *dst, uint64_t m, cudaStream_t s)
{
    if (m == 0)
        return cudaSuccess;
    if (m > n)
        return cudaErrorInvalidValue;
    const uint64_t stride = n / m; // (m - 1) * stride < n
    const uint64_t blocks = std::min<uint64_t>((m + 255) / 256, uint64_t(device_sm_count()) * 8);
    k_gather_stride<<<unsigned(blocks), 256, 0, s>>>(src, stride, dst, m);
    return cudaGetLastError();
}

// ------------------------------------------------------ distance queries (disks)
// A point is within distance r of a centre c iff (px-cx)^2 + (py-cy)^2 <= r^2,
// exact in int64 (differences < 2^31; r < 2^30; the x term is compared with
// r^2 before the sum, so the sum cannot overflow).  A point reads the word of
// its cell in the disks' grid; INSIDE entries count at once and BOUNDARY
// entries take the exact test; lists are in disk order.
__device__ __forceinline__ bool in_disk(const int4 &d, int px, int py)
{
    const long long dx = (long long)px - d.x, dy = (long long)py - d.y, rr = (long long)d.z * d.z;
    const long long dx2 = dx * dx;
    return dx2 <= rr && dx2 + dy * dy <= rr;
}

template <class F>
__device__ __forceinline__ uint32_t disk_walk(const DiskView &d, int px, int py, uint32_t &first, uint32_t &tests,
                                              uint64_t pol, F f)
{
    if ((unsigned)px >= kBox || (unsigned)py >= kBox)
        return 0;
    const uint32_t w = ld_idx(d.cell + ((((uint32_t)py >> d.sc) << d.g) | ((uint32_t)px >> d.sc)), pol);
    const uint32_t kind = w >> 30;
    if (kind == kCellInsideOne) {
        first = w & kPayloadMask;
        f(first);
        return 1;
    }
    if (kind != kCellList)
        return 0;
    const uint32_t *e = d.ent + (w & kPayloadMask);
    const uint32_t n = ld_idx(e, pol);
    uint32_t c = 0;
    for (uint32_t k = 1; k <= n; ++k) {
        const uint32_t en = ld_idx(e + k, pol), q = en >> 1;
        bool in = true;
        if (en & 1u) {
            ++tests;
            in = in_disk(__ldg(d.disk + q), px, py);
        }
        if (in) {
            if (!c)
                first = q;
            ++c;
            f(q);
        }
    }
    return c;
}

// Distance join with warp chunks (the design of k_warp / k_wemit): pass 1
// resolves every point once: the cover bitmap (in shared memory) sends the
// points of blocks without any disk away without an index read; the others
// read their cell word, and the points of list cells are queued in shared
// memory.  The queue carries over from chunk to chunk and the warp walks it
// in full rounds of 32 (one chain of dependent loads per 32 list points); a
// walked point adds its pairs to its own chunk's total (stored by lane 0
// before any of the chunk's points is walked; __syncwarp orders the two).
// It stores a 4-byte result per point and a pair total per 256-point chunk,
// and counts per disk (in shared memory when Q <= kHistMax); pass 3 writes
// the pairs from the results.
constexpr int kDiskMinBlocks = 4;
constexpr uint32_t kDiskCoverWords = 1u << (2 * kCoverLog2 - 5); // cover bitmap in shared memory
constexpr int kDQueue = kWChunk + 32; // a chunk's points plus a partial round
constexpr size_t kDWarpSmem = size_t(kWarps) * kDQueue * sizeof(uint4);

template <bool RESOLVE>
__global__ void __launch_bounds__(kThreads, kDiskMinBlocks) k_dwarp(DiskLaunch a, unsigned long long *chunk_tot, uint32_t *res,
                                                       uint32_t nchunks, int use_hist)
{
    extern __shared__ __align__(16) unsigned char s_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4 *s_q = reinterpret_cast<uint4 *>(s_raw) + warp * kDQueue; // (x, y, list offset, point index)
    uint32_t *s_cov = reinterpret_cast<uint32_t *>(s_raw + kDWarpSmem);
    uint32_t *s_hist = s_cov + kDiskCoverWords;
    const DiskView &d = a.dv;
    const uint64_t keep = policy_evict_last();
    const bool hist = use_hist && a.counts;
    const uint32_t ncov = max(1u, (1u << (2 * d.cg)) >> 5);
    for (uint32_t i = threadIdx.x; i < ncov; i += kThreads)
        s_cov[i] = __ldg(d.cover + i);
    if (hist)
        for (uint32_t i = threadIdx.x; i < d.Q; i += kThreads)
            s_hist[i] = 0;
    __syncthreads();
    // count one disk for every lane with has (converged warp)
    auto count1 = [&](bool has, uint32_t q) {
        if (!a.counts)
            return;
        if (!hist)
            global_add_warp(a.counts, has, q);
        else if (has)
            atomicAdd(s_hist + q, 1u);
    };
    uint32_t n_tests = 0, n_pts = 0, n_pairs = 0;
    // walk queued list points [k0, k0 + m), m <= 32, one per lane; their pairs
    // are added to their chunk's total
    auto walk = [&](uint32_t k0, uint32_t m) {
        const bool has = (uint32_t)lane < m;
        const uint4 it = s_q[k0 + (has ? lane : 0)]; // idle lanes repeat lane 0's walk, uncounted
        const uint32_t *e = d.ent + it.z;
        const uint32_t n = ld_idx(e, keep);
        uint32_t c = 0, f = 0, t_l = 0;
        for (uint32_t k = 1; k <= n; ++k) {
            const uint32_t en = ld_idx(e + k, keep), q = en >> 1;
            bool in = true;
            if (en & 1u) {
                ++t_l;
                in = in_disk(__ldg(d.disk + q), (int)it.x, (int)it.y);
            }
            if (in) {
                if (!c)
                    f = q;
                else if (has && a.counts) // the first disk is counted with the warp below
                    hist ? (void)atomicAdd(s_hist + q, 1u) : (void)atomicAdd(a.counts + q, 1ull);
                ++c;
            }
        }
        c = has ? c : 0u;
        n_tests += has ? t_l : 0u;
        n_pairs += c;
        count1(c >= 1, f);
        if (RESOLVE && has) {
            __stcg(res + it.w, res_encode(c, f));
            if (c)
                atomicAdd(chunk_tot + it.w / kWChunk, (unsigned long long)c);
        }
        __syncwarp();
    };
    const uint32_t nw = gridDim.x * kWarps;
    uint32_t qn = 0; // queued list points, < 32 between chunks
    for (uint32_t ch = blockIdx.x * kWarps + warp; ch < nchunks; ch += nw) {
        const uint64_t base = (uint64_t)ch * kWChunk;
        const uint32_t npts = (uint32_t)min((uint64_t)kWChunk, a.n - base);
        if (lane == 0)
            n_pts += npts;
        int2 p[kWItems];
        uint32_t w[kWItems];
        // rows past the table's end read as outside the box
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            const uint32_t loc = j * 32 + lane;
            p[j] = loc < npts ? __ldcs(a.pts + base + loc) : make_int2(-1, -1);
        }
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            // points outside the box or in a block of empty cells read no cell word
            const uint32_t px = (uint32_t)p[j].x, py = (uint32_t)p[j].y;
            const uint32_t b = (((py & (kBox - 1)) >> d.scv) << d.cg) | ((px & (kBox - 1)) >> d.scv);
            const bool ok = px < kBox && py < kBox && ((s_cov[b >> 5] >> (b & 31)) & 1u);
            w[j] = ok ? ld_idx(d.cell + ((((py & (kBox - 1)) >> d.sc) << d.g) | ((px & (kBox - 1)) >> d.sc)), keep)
                      : 0u;
        }
        uint32_t total = 0;
#pragma unroll
        for (int j = 0; j < kWItems; ++j) {
            const uint32_t kind = w[j] >> 30, loc = j * 32 + lane;
            const bool one = kind == kCellInsideOne, lst = kind == kCellList;
            total += one ? 1u : 0u;
            count1(one, w[j] & kPayloadMask);
            if (RESOLVE && loc < npts && !lst)
                __stcg(res + base + loc, one ? (w[j] & kPayloadMask) : kResNone);
            const uint32_t bl = __ballot_sync(kFull, lst);
            if (lst)
                s_q[qn + __popc(bl & lanemask_lt())] =
                    make_uint4((uint32_t)p[j].x, (uint32_t)p[j].y, w[j] & kPayloadMask, (uint32_t)(base + loc));
            qn += __popc(bl);
        }
        n_pairs += total;
        total = warp_sum32(total);
        if (RESOLVE && lane == 0)
            chunk_tot[ch] = total; // the chunk's pair total so far; its queued points add theirs
        __syncwarp();
        if (qn >= 32) {
            uint32_t k0 = 0;
            for (; qn - k0 >= 32; k0 += 32)
                walk(k0, 32);
            // move the partial round (< 32, from k0 >= 32) to the front
            const uint32_t rem = qn - k0;
            const uint4 it = (uint32_t)lane < rem ? s_q[k0 + lane] : make_uint4(0, 0, 0, 0);
            __syncwarp();
            if ((uint32_t)lane < rem)
                s_q[lane] = it;
            qn = rem;
            __syncwarp();
        }
    }
    __syncwarp();
    if (qn)
        walk(0, qn);
    if (hist) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < d.Q; i += kThreads)
            if (s_hist[i])
                atomicAdd(a.counts + i, (unsigned long long)s_hist[i]);
    }
    add_stats(a.stats, n_pts, n_tests, 0u, n_pairs);
}

// Pass 3 of the distance join.  Lane-major: lane l owns rows 8l .. 8l + 7 of
// the warp's 256-row chunk (two 16-byte loads of stored results), so one warp
// scan of the lanes' pair counts gives every row its offset in point order.
// A point in one disk is written at once; a point in several is queued (its
// row and its offset; its count comes with its stored result).  Such points
// are rare, so the queue carries over from chunk to chunk and the warp walks
// it only in full rounds of 32 (and what is left at the end), loading the
// queued points' coordinates then, one independent load per lane.  The next
// chunk's results are loaded while this one is written.
constexpr size_t kDEmitSmem = size_t(kWarps) * kDQueue * (sizeof(uint32_t) + sizeof(unsigned long long));
static_assert(kWItems == 8, "lane-major emit: two 16-byte loads of 4-byte results per lane");

__global__ void __launch_bounds__(kThreads, 4) k_dwemit(DiskLaunch a, const unsigned long long *chunk_off,
                                                        const uint32_t *res_in, uint32_t nchunks)
{
    extern __shared__ __align__(16) unsigned char s_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long *s_o = reinterpret_cast<unsigned long long *>(s_raw) + warp * kDQueue;
    uint32_t *s_q = reinterpret_cast<uint32_t *>(s_raw + size_t(kWarps) * kDQueue * sizeof(unsigned long long)) +
                    warp * kDQueue; // point rows
    const uint64_t keep = policy_evict_last();
    // walk queued points [k0, k0 + m), m <= 32, one per lane
    auto walk = [&](uint32_t k0, uint32_t m) {
        if ((uint32_t)lane < m) {
            const uint32_t pid = s_q[k0 + lane];
            unsigned long long o = s_o[k0 + lane];
            const int2 p = a.pts[pid];
            uint32_t f = 0, t = 0;
            disk_walk(a.dv, p.x, p.y, f, t, keep, [&](uint32_t q) {
                if (o < a.cap)
                    __stcs(a.pairs + o, make_uint2(pid, q));
                ++o;
            });
        }
    };
    uint32_t qn = 0; // queued points, < 32 between chunks
    const uint32_t nw = gridDim.x * kWarps;
    const uint32_t r0 = 8u * (uint32_t)lane; // this lane's first row in a chunk
    uint32_t nres[8];
    unsigned long long noff = 0;
    auto fetch = [&](uint32_t ch) {
        const uint64_t base = (uint64_t)ch * kWChunk;
        const uint32_t npts = ch < nchunks ? (uint32_t)min((uint64_t)kWChunk, a.n - base) : 0u;
        if (r0 + 8 <= npts) {
            const uint4 u = __ldcs(reinterpret_cast<const uint4 *>(res_in + base + r0));
            const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(res_in + base + r0 + 4));
            nres[0] = u.x, nres[1] = u.y, nres[2] = u.z, nres[3] = u.w;
            nres[4] = v.x, nres[5] = v.y, nres[6] = v.z, nres[7] = v.w;
        } else { // the table's ragged end
#pragma unroll
            for (int k = 0; k < 8; ++k)
                nres[k] = r0 + k < npts ? __ldcs(res_in + base + r0 + k) : kResNone;
        }
        noff = ch < nchunks ? chunk_off[ch] : 0ull;
    };
    fetch(blockIdx.x * kWarps + warp);
    for (uint32_t ch = blockIdx.x * kWarps + warp; ch < nchunks; ch += nw) {
        const uint32_t pid0 = (uint32_t)((uint64_t)ch * kWChunk) + r0;
        const unsigned long long run = noff;
        uint32_t res[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            res[k] = nres[k];
        fetch(ch + nw);
        // pairs (low 32 bits) and multi-disk points (high 32 bits) of this
        // lane's rows, for one scan; a multi-disk row keeps kResMulti | count
        unsigned long long mine = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t r = res[k];
            if (r == kResNone)
                continue;
            uint32_t c = 1;
            if (r & kResMulti) {
                if (r & kResCount) {
                    c = (r >> 20) & 0x3ffu;
                } else { // count not stored: count again
                    const int2 p = a.pts[pid0 + k];
                    uint32_t f = 0, t = 0;
                    c = disk_walk(a.dv, p.x, p.y, f, t, keep, [](uint32_t) {});
                }
                res[k] = kResMulti | c;
                mine += 1ull << 32;
            }
            mine += c;
        }
        unsigned long long inc = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(kFull, inc, o);
            if (lane >= o)
                inc += v;
        }
        const unsigned long long tot = __shfl_sync(kFull, inc, 31), before = inc - mine;
        if (mine) {
            unsigned long long o = run + (uint32_t)before;
            uint32_t slot = qn + (uint32_t)(before >> 32);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t r = res[k];
                if (r == kResNone)
                    continue;
                if (r & kResMulti) {
                    s_q[slot] = pid0 + k;
                    s_o[slot] = o;
                    ++slot;
                    o += r & ~kResMulti;
                } else {
                    if (o < a.cap)
                        __stcs(a.pairs + o, make_uint2(pid0 + k, r));
                    ++o;
                }
            }
        }
        qn += (uint32_t)(tot >> 32);
        __syncwarp();
        if (qn >= 32) {
            uint32_t k0 = 0;
            for (; qn - k0 >= 32; k0 += 32)
                walk(k0, 32);
            // move the partial round (< 32, from k0 >= 32) to the front
            const uint32_t rem = qn - k0;
            uint32_t q = 0;
            unsigned long long oo = 0;
            if ((uint32_t)lane < rem) {
                q = s_q[k0 + lane];
                oo = s_o[k0 + lane];
            }
            __syncwarp();
            if ((uint32_t)lane < rem) {
                s_q[lane] = q;
                s_o[lane] = oo;
            }
            qn = rem;
            __syncwarp();
        }
    }
    __syncwarp();
    walk(0, qn);
}

// ------------------------------------------------------ disk index, built on the device
// The same arrays as the host build (build_disk_index): for every disk, every
// cell of its clipped bounding box is classified exactly in int64 (the cell's
// integer point nearest the centre beyond r: no entry; its farthest corner
// within r: INSIDE; else BOUNDARY); the (cell, disk) records are bucketed by
// cell; a cell with one INSIDE record gets a kind-1 word, any other non-empty
// cell a list (n, then the records in disk order), lists laid out in cell
// order after a reserved word 0.  No kernel here waits on another.
struct DiskBox {
    uint32_t i0, j0, w, h; // first cell column / row and the box's size in cells (w = 0: no cell)
};

__device__ __forceinline__ DiskBox disk_box(const int4 &d, int sh)
{
    const long long last = (long long)kBox - 1;
    const long long xlo = max(0ll, (long long)d.x - d.z), xhi = min(last, (long long)d.x + d.z);
    const long long ylo = max(0ll, (long long)d.y - d.z), yhi = min(last, (long long)d.y + d.z);
    if (xlo > xhi || ylo > yhi)
        return {0u, 0u, 0u, 0u};
    const uint32_t i0 = (uint32_t)(xlo >> sh), j0 = (uint32_t)(ylo >> sh);
    return {i0, j0, (uint32_t)(xhi >> sh) - i0 + 1, (uint32_t)(yhi >> sh) - j0 + 1};
}

// Does disk d reach cell (i, j) of side 2^sh, and does it hold the whole cell?
__device__ __forceinline__ bool disk_cell(const int4 &d, uint32_t i, uint32_t j, int sh, bool &inside)
{
    const long long S = 1ll << sh, x0 = (long long)i << sh, y0 = (long long)j << sh, x1 = x0 + S - 1,
                    y1 = y0 + S - 1;
    const long long cx = d.x, cy = d.y, rr = (long long)d.z * d.z;
    const long long nx = min(max(cx, x0), x1) - cx, ny = min(max(cy, y0), y1) - cy;
    if (nx * nx + ny * ny > rr)
        return false;
    const long long fx = max(cx - x0, x1 - cx), fy = max(cy - y0, y1 - cy);
    inside = fx * fx + fy * fy <= rr;
    return true;
}

// Records per disk (a block per disk, its threads over the box's cells) and
// the number of BOUNDARY records.
__global__ void __launch_bounds__(256) k_dbuild_count(const int4 *disk, uint32_t Q, int g,
                                                      unsigned long long *rec_cnt, unsigned long long *n_bnd)
{
    __shared__ unsigned long long s_c, s_b;
    const int sh = kBoxLog2 - g;
    for (uint32_t q = blockIdx.x; q < Q; q += gridDim.x) {
        if (threadIdx.x == 0)
            s_c = s_b = 0;
        __syncthreads();
        const int4 d = disk[q];
        const DiskBox b = disk_box(d, sh);
        const uint64_t n = (uint64_t)b.w * b.h;
        unsigned long long c = 0, bn = 0;
        for (uint64_t t = threadIdx.x; t < n; t += blockDim.x) {
            bool in = false;
            if (disk_cell(d, b.i0 + (uint32_t)(t % b.w), b.j0 + (uint32_t)(t / b.w), sh, in)) {
                ++c;
                bn += in ? 0u : 1u;
            }
        }
        c = warp_sum64(c);
        bn = warp_sum64(bn);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&s_c, c);
            atomicAdd(&s_b, bn);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            rec_cnt[q] = s_c;
            if (s_b)
                atomicAdd(n_bnd, s_b);
        }
        __syncthreads();
    }
}

// Records (cell, disk << 1 | boundary) at each disk's offset; per-cell record
// counts and an OR of their boundary flags.
__global__ void __launch_bounds__(256) k_dbuild_write(const int4 *disk, uint32_t Q, int g,
                                                      const unsigned long long *rec_off, uint2 *rec,
                                                      uint32_t *cell_cnt, uint32_t *cell_bnd)
{
    __shared__ unsigned long long s_pos;
    const int sh = kBoxLog2 - g;
    for (uint32_t q = blockIdx.x; q < Q; q += gridDim.x) {
        if (threadIdx.x == 0)
            s_pos = 0;
        __syncthreads();
        const int4 d = disk[q];
        const DiskBox b = disk_box(d, sh);
        const uint64_t n = (uint64_t)b.w * b.h;
        const unsigned long long base = rec_off[q];
        for (uint64_t t = threadIdx.x; t < n; t += blockDim.x) {
            const uint32_t i = b.i0 + (uint32_t)(t % b.w), j = b.j0 + (uint32_t)(t / b.w);
            bool in = false;
            if (disk_cell(d, i, j, sh, in)) {
                const uint32_t c = (j << g) | i;
                rec[base + atomicAdd(&s_pos, 1ull)] = make_uint2(c, (q << 1) | (in ? 0u : 1u));
                atomicAdd(cell_cnt + c, 1u);
                if (!in)
                    atomicOr(cell_bnd + c, 1u);
            }
        }
        __syncthreads();
    }
}

// Words of the entry list of every cell that needs one (0 for the others).
__global__ void k_dbuild_words(uint32_t ncell, const uint32_t *cell_cnt, const uint32_t *cell_bnd,
                               unsigned long long *list_words)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        const uint32_t n = cell_cnt[c];
        list_words[c] = (n >= 2 || (n == 1 && cell_bnd[c])) ? n + 1ull : 0ull;
    }
}

// List cells: their word and list length (after the reserved word 0).
__global__ void k_dbuild_cells(uint32_t ncell, const uint32_t *cell_cnt, const uint32_t *cell_bnd,
                               const unsigned long long *list_off, uint32_t *cell_word, uint32_t *ent)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        const uint32_t n = cell_cnt[c];
        if (n >= 2 || (n == 1 && cell_bnd[c])) {
            const uint32_t off = 1u + (uint32_t)list_off[c];
            cell_word[c] = (kCellList << 30) | off;
            ent[off] = n;
        }
    }
}

// Every record to its cell: the word of a one-INSIDE cell, else the next slot
// of the cell's list (sorted afterwards).
__global__ void k_dbuild_scatter(uint64_t R, const uint2 *rec, const uint32_t *cell_cnt, const uint32_t *cell_bnd,
                                 const unsigned long long *list_off, uint32_t *cursor, uint32_t *cell_word,
                                 uint32_t *ent)
{
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < R; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 r = rec[k];
        if (cell_cnt[r.x] == 1 && !cell_bnd[r.x])
            cell_word[r.x] = (kCellInsideOne << 30) | (r.y >> 1);
        else
            ent[2u + (uint32_t)list_off[r.x] + atomicAdd(cursor + r.x, 1u)] = r.y;
    }
}

// Each list in disk order (insertion sort: lists are short).
__global__ void k_dbuild_sort(uint32_t ncell, const uint32_t *cell_word, uint32_t *ent)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        const uint32_t w = cell_word[c];
        if ((w >> 30) != kCellList)
            continue;
        uint32_t *l = ent + (w & kPayloadMask) + 1;
        const uint32_t n = l[-1];
        for (uint32_t a = 1; a < n; ++a) {
            const uint32_t v = l[a];
            uint32_t b = a;
            for (; b > 0 && l[b - 1] > v; --b)
                l[b] = l[b - 1];
            l[b] = v;
        }
    }
}

// Cover bitmap: a bit per block of cells that holds a non-empty cell.
__global__ void k_dbuild_cover(uint32_t ncell, int g, int cg, const uint32_t *cell_word, uint32_t *cover)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        if (!cell_word[c])
            continue;
        const uint32_t cx = c & ((1u << g) - 1), cy = c >> g;
        const uint32_t b = ((cy >> (g - cg)) << cg) | (cx >> (g - cg));
        atomicOr(cover + (b >> 5), 1u << (b & 31));
    }
}

int build_disk_index_device(const int4 *disks_host, uint32_t Q, int g, DiskIndexDev &out, cudaError_t &cerr)
{
    out = DiskIndexDev{};
    cerr = cudaSuccess;
    const uint32_t ncell = 1u << (2 * g);
    const int cg = g < kCoverLog2 ? g : kCoverLog2;
    const size_t cover_words = ((size_t(1) << (2 * cg)) / 32) > 0 ? ((size_t(1) << (2 * cg)) / 32) : 1;
    const size_t nd = Q ? Q : 1;
    const uint64_t nparts = scan_partials(ncell > nd ? ncell : nd) + 2;
    // temporaries: disks | per-disk record counts | totals | scan partials |
    // per-cell counts, flags, cursors | per-cell list words
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t t_disk = up(nd * sizeof(int4)), t_cnt = up((nd + 1) * 8), t_tot = up(3 * 8), t_part = up(nparts * 8),
                 t_cell = up(size_t(ncell) * 4), t_words = up(size_t(ncell) * 8);
    char *tmp = nullptr, *recm = nullptr;
    auto done = [&](int status, cudaError_t e) {
        cerr = e;
        if (recm)
            cudaFree(recm);
        if (tmp)
            cudaFree(tmp);
        if (status && out.mem) {
            cudaFree(out.mem);
            out.mem = nullptr;
        }
        return status;
    };
    cudaError_t e = cudaMalloc(&tmp, t_disk + t_cnt + t_tot + t_part + 3 * t_cell + t_words);
    if (e != cudaSuccess)
        return done(2, e);
    int4 *d_disk = reinterpret_cast<int4 *>(tmp);
    auto *rec_cnt = reinterpret_cast<unsigned long long *>(tmp + t_disk);
    auto *tot = reinterpret_cast<unsigned long long *>(tmp + t_disk + t_cnt); // records, list words, boundary
    auto *part = reinterpret_cast<unsigned long long *>(tmp + t_disk + t_cnt + t_tot);
    auto *cell_cnt = reinterpret_cast<uint32_t *>(tmp + t_disk + t_cnt + t_tot + t_part);
    auto *cell_bnd = reinterpret_cast<uint32_t *>(tmp + t_disk + t_cnt + t_tot + t_part + t_cell);
    auto *cursor = reinterpret_cast<uint32_t *>(tmp + t_disk + t_cnt + t_tot + t_part + 2 * t_cell);
    auto *words = reinterpret_cast<unsigned long long *>(tmp + t_disk + t_cnt + t_tot + t_part + 3 * t_cell);
    if ((e = cudaMemcpy(d_disk, disks_host, nd * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(tot, 0, 3 * 8)) != cudaSuccess || (e = cudaMemset(cell_cnt, 0, 3 * t_cell)) != cudaSuccess)
        return done(2, e);
    const int sms = device_sm_count();
    const unsigned dblocks = Q ? (Q < unsigned(sms * 8) ? Q : unsigned(sms * 8)) : 1u;
    const unsigned cblocks = unsigned((ncell + 255) / 256 < uint32_t(sms * 16) ? (ncell + 255) / 256 : sms * 16);
    unsigned long long R = 0, T = 0, nb = 0;
    if (Q) {
        k_dbuild_count<<<dblocks, 256>>>(d_disk, Q, g, rec_cnt, tot + 2);
        if ((e = cudaGetLastError()) != cudaSuccess || (e = launch_scan(rec_cnt, Q, tot, part, 0)) != cudaSuccess ||
            (e = cudaMemcpy(&R, tot, 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return done(2, e);
    }
    if (R) {
        if ((e = cudaMalloc(&recm, R * sizeof(uint2))) != cudaSuccess)
            return done(2, e);
        k_dbuild_write<<<dblocks, 256>>>(d_disk, Q, g, rec_cnt, reinterpret_cast<uint2 *>(recm), cell_cnt, cell_bnd);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return done(2, e);
    }
    k_dbuild_words<<<cblocks, 256>>>(ncell, cell_cnt, cell_bnd, words);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = launch_scan(words, ncell, tot + 1, part, 0)) != cudaSuccess ||
        (e = cudaMemcpy(&T, tot + 1, 8, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(&nb, tot + 2, 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return done(2, e);
    const uint64_t E = 1 + T;
    if (E > kPayloadMask)
        return done(1, cudaSuccess);
    // the index's own allocation: cells | entries | disks | cover, as the host path lays it out
    const size_t b_cell = size_t(ncell) * 4, b_ent = size_t(E) * 4, b_disk = nd * sizeof(int4), b_cover = cover_words * 4;
    out.bytes = up(b_cell) + up(b_ent) + up(b_disk) + up(b_cover);
    if ((e = cudaMalloc(&out.mem, out.bytes)) != cudaSuccess) {
        out.mem = nullptr;
        return done(2, e);
    }
    char *m = static_cast<char *>(out.mem);
    out.cell = reinterpret_cast<uint32_t *>(m);
    out.ent = reinterpret_cast<uint32_t *>(m + up(b_cell));
    out.disk = reinterpret_cast<int4 *>(m + up(b_cell) + up(b_ent));
    out.cover = reinterpret_cast<uint32_t *>(m + up(b_cell) + up(b_ent) + up(b_disk));
    if ((e = cudaMemset(out.cell, 0, b_cell)) != cudaSuccess || (e = cudaMemset(out.ent, 0, b_ent)) != cudaSuccess ||
        (e = cudaMemset(out.cover, 0, b_cover)) != cudaSuccess ||
        (e = cudaMemcpy(out.disk, d_disk, b_disk, cudaMemcpyDeviceToDevice)) != cudaSuccess)
        return done(2, e);
    k_dbuild_cells<<<cblocks, 256>>>(ncell, cell_cnt, cell_bnd, words, out.cell, out.ent);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return done(2, e);
    if (R) {
        const unsigned rblocks = unsigned((R + 255) / 256 < uint64_t(sms * 16) ? (R + 255) / 256 : sms * 16);
        k_dbuild_scatter<<<rblocks, 256>>>(R, reinterpret_cast<const uint2 *>(recm), cell_cnt, cell_bnd, words, cursor,
                                           out.cell, out.ent);
        k_dbuild_sort<<<cblocks, 256>>>(ncell, out.cell, out.ent);
    }
    k_dbuild_cover<<<cblocks, 256>>>(ncell, g, cg, out.cell, out.cover);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess)
        return done(2, e);
    out.n_ent = E;
    out.n_boundary = nb;
    out.n_inside = R - nb;
    return done(0, cudaSuccess);
}

// ------------------------------------------------------ clustered point table
// Counting sort of a point table by grid cell (row-major cells of a 2^c x 2^c
// grid; points outside the box go to one last bin).  Lanes of a warp with the
// same key share one atomic.
__device__ __forceinline__ uint32_t cell_key(int2 p, int c)
{
    if ((unsigned)p.x >= kBox || (unsigned)p.y >= kBox)
        return 1u << (2 * c);
    const int sh = kBoxLog2 - c;
    return (((uint32_t)p.y >> sh) << c) | ((uint32_t)p.x >> sh);
}

__global__ void __launch_bounds__(256) k_cell_hist(const int2 *__restrict__ pts, uint64_t n, int c,
                                                 unsigned long long *cnt)
{
    const uint64_t stride = (uint64_t)gridDim.x * 256;
    for (uint64_t i0 = (uint64_t)blockIdx.x * 256 + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
        const uint64_t i = i0 + (threadIdx.x & 31);
        const bool has = i < n;
        const uint32_t key = has ? cell_key(__ldcs(pts + i), c) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(kFull, key);
        if (has && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
            atomicAdd(cnt + key, (unsigned long long)__popc(peers));
    }
}

__global__ void __launch_bounds__(256) k_cell_scatter(const int2 *__restrict__ pts, uint64_t n, int c,
                                                    unsigned long long *cursor, int2 *__restrict__ out)
{
    const uint64_t stride = (uint64_t)gridDim.x * 256;
    const int lane = threadIdx.x & 31;
    for (uint64_t i0 = (uint64_t)blockIdx.x * 256 + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
        const uint64_t i = i0 + lane;
        const bool has = i < n;
        const int2 p = has ? __ldcs(pts + i) : make_int2(-1, -1);
        const uint32_t key = has ? cell_key(p, c) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(kFull, key);
        const int leader = __ffs(peers) - 1;
        unsigned long long base = 0;
        if (has && lane == leader)
            base = atomicAdd(cursor + key, (unsigned long long)__popc(peers));
        base = __shfl_sync(kFull, base, leader);
        if (has)
            out[base + __popc(peers & lanemask_lt())] = p;
    }
}

size_t cluster_scratch_bytes(int c)
{
    const uint64_t bins = (uint64_t(1) << (2 * c)) + 1;
    return size_t(bins + scan_partials(bins) + 2) * 8 + 64;
}

cudaError_t launch_cluster(const int2 *pts, uint64_t n, int c, void *scratch, int2 *out, cudaStream_t s)
{
    if (c < 1 || c > 13)
        return cudaErrorInvalidValue;
    if (n == 0)
        return cudaSuccess;
    const uint64_t bins = (uint64_t(1) << (2 * c)) + 1;
    unsigned long long *cnt = static_cast<unsigned long long *>(scratch);
    unsigned long long *part = cnt + bins;
    cudaError_t e = cudaMemsetAsync(cnt, 0, bins * 8, s);
    if (e != cudaSuccess)
        return e;
    const unsigned grid = unsigned(std::min<uint64_t>((n + 255) / 256, uint64_t(device_sm_count()) * 16));
    k_cell_hist<<<grid, 256, 0, s>>>(pts, n, c, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    if ((e = launch_scan(cnt, bins, nullptr, part, s)) != cudaSuccess) // cnt: cell starts (cursors)
        return e;
    k_cell_scatter<<<grid, 256, 0, s>>>(pts, n, c, cnt, out);
    return cudaGetLastError();
}

uint32_t join_chunk_points() { return kWChunk; }
// part: the bitmap of pass 1 (8 words per chunk = 4 u64), then the scan's partials
uint64_t join_part_words(uint64_t n)
{
    const uint64_t nchunks = (n + kWChunk - 1) / kWChunk;
    return nchunks * (kWItems / 2) + scan_partials(nchunks) + 2;
}

// Passes 1 and 2.  ev (or null): events recorded after pass 1a, after pass 1b
// and after the scan.
static cudaError_t join_resolve_scan(const JoinLaunch &a, unsigned long long *part, cudaStream_t s, cudaEvent_t *ev)
{
    const uint64_t nchunks = (a.n + kWChunk - 1) / kWChunk;
    if (nchunks >= (1ull << 31))
        return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(a.pts) & 15)
        return cudaErrorMisalignedAddress;
    if (nchunks == 0)
        return a.total ? cudaMemsetAsync(a.total, 0, sizeof(unsigned long long), s) : cudaSuccess;
    uint32_t *pend = reinterpret_cast<uint32_t *>(part);
    cudaError_t e = a.fp32 ? launch_pass1<true>(a, pend, s, ev ? ev[0] : nullptr)
                           : launch_pass1<false>(a, pend, s, ev ? ev[0] : nullptr);
    if (e != cudaSuccess)
        return e;
    if (ev)
        cudaEventRecord(ev[1], s);
    e = launch_scan(a.tile_tot, nchunks, a.total, part + nchunks * (kWItems / 2), s);
    if (ev)
        cudaEventRecord(ev[2], s);
    return e;
}

cudaError_t launch_join_resolve(const JoinLaunch &a, unsigned long long *part, cudaStream_t s)
{
    return join_resolve_scan(a, part, s, nullptr);
}

cudaError_t launch_join_emit(const JoinLaunch &a, cudaStream_t s, const uint32_t *pend)
{
    const uint32_t nchunks = uint32_t((a.n + kWChunk - 1) / kWChunk);
    if (nchunks == 0 || a.cap == 0)
        return cudaSuccess;
    if (a.narrow && !pend)
        return cudaErrorInvalidValue;
    const uint32_t nblk = (nchunks + kWarps - 1) / kWarps;
    static bool done[4][64] = {};
    auto emit = [&](auto kr, bool(&d)[64]) -> cudaError_t {
        cudaError_t e = smem_opt_in(kr, kEmitSmem, d);
        if (e != cudaSuccess)
            return e;
        kr<<<persistent_grid(kr, kThreads, kEmitSmem, nblk), kThreads, kEmitSmem, s>>>(a, a.tile_tot, nchunks, pend);
        return cudaGetLastError();
    };
    if (a.narrow)
        return a.fp32 ? emit(k_wemit<true, true>, done[2]) : emit(k_wemit<false, true>, done[3]);
    return a.fp32 ? emit(k_wemit<true, false>, done[0]) : emit(k_wemit<false, false>, done[1]);
}

__global__ void k_sum_u64(unsigned long long *dst, const unsigned long long *x, const unsigned long long *y)
{
    *dst = *x + *y;
}

cudaError_t launch_sum_u64(unsigned long long *dst, const unsigned long long *x, const unsigned long long *y,
                           cudaStream_t s)
{
    k_sum_u64<<<1, 1, 0, s>>>(dst, x, y);
    return cudaGetLastError();
}

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
    // per-point results | per-chunk totals (then offsets) | scan partials
    const uint64_t nchunks = (n + kWChunk - 1) / kWChunk;
    return size_t(((n * 4 + 15) & ~uint64_t(15)) + (nchunks + join_part_words(n)) * 8 + 16);
}

size_t plain_scratch_bytes(uint64_t n)
{
    const uint64_t nb = (n + kPlainThreads - 1) / kPlainThreads;
    return size_t(nb * 8 + 16);
}

// The join's scratch: per-point results | per-chunk totals (then offsets) |
// row bitmap and scan partials.  Fills b's result and total pointers and the
// result width.
static unsigned long long *join_layout(JoinLaunch &b, void *scratch)
{
    char *sc = static_cast<char *>(scratch);
    b.res = reinterpret_cast<uint32_t *>(sc);
    b.tile_tot = reinterpret_cast<unsigned long long *>(sc + ((b.n * 4 + 15) & ~uint64_t(15)));
    // 16-bit results when every polygon id and every point's polygon count
    // fit (the row bitmap in part stays in place until pass 3)
    b.narrow = b.ix.P <= kRes16MaxP ? 1 : 0;
    return b.tile_tot + (b.n + kWChunk - 1) / kWChunk;
}

cudaError_t launch_join_count(const JoinLaunch &a, void *scratch, cudaStream_t s, cudaEvent_t *ev)
{
    if ((a.n + kWChunk - 1) / kWChunk >= (1ull << 31))
        return cudaErrorInvalidValue;
    JoinLaunch b = a;
    unsigned long long *part = join_layout(b, scratch);
    cudaError_t e;
    if (a.counts && a.ix.P && !a.keep_counts)
        if ((e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * a.ix.P, s)) != cudaSuccess)
            return e;
    if (a.n == 0)
        return a.total ? cudaMemsetAsync(a.total, 0, sizeof(unsigned long long), s) : cudaSuccess;
    // passes 1 and 2: resolve every point (counts per polygon, per-point
    // results, per-chunk totals), then the offsets and the total
    if (ev)
        cudaEventRecord(ev[0], s);
    return join_resolve_scan(b, part, s, ev ? ev + 1 : nullptr);
}

cudaError_t launch_join_write(const JoinLaunch &a, void *scratch, cudaStream_t s)
{
    if (a.n == 0)
        return cudaSuccess;
    JoinLaunch b = a;
    unsigned long long *part = join_layout(b, scratch);
    // pass 3: pairs in point order
    return launch_join_emit(b, s, reinterpret_cast<const uint32_t *>(part));
}

cudaError_t launch_join(const JoinLaunch &a, void *scratch, cudaStream_t s, cudaEvent_t *ev)
{
    cudaError_t e = launch_join_count(a, scratch, s, ev);
    if (e != cudaSuccess || a.n == 0)
        return e;
    if ((e = launch_join_write(a, scratch, s)) != cudaSuccess)
        return e;
    if (ev)
        cudaEventRecord(ev[4], s);
    return cudaSuccess;
}

static bool use_directory(const JoinLaunch &a)
{
    return a.clustered && a.cell_end && a.cluster_log2 >= a.ix.gc && a.cluster_log2 <= 13;
}

size_t aggregate_scratch_bytes(const JoinLaunch &a)
{
    const uint64_t nchunks = (a.n + kWChunk - 1) / kWChunk;
    return use_directory(a) ? size_t((nchunks + 31) / 32) * 4 + 16 : 16;
}

cudaError_t launch_aggregate(const JoinLaunch &a, void *scratch, cudaStream_t s, cudaEvent_t *ev)
{
    cudaError_t e = cudaSuccess;
    if (!a.keep_counts)
        e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * (a.ix.P ? a.ix.P : 1), s);
    if (e != cudaSuccess || a.n == 0)
        return e;
    if (reinterpret_cast<uintptr_t>(a.pts) & 15)
        return cudaErrorMisalignedAddress;
    const int use_hist = a.ix.P <= (uint32_t)kHistMax ? 1 : 0;
    if (ev)
        cudaEventRecord(ev[0], s);
    if (use_directory(a)) {
        // cells INSIDE one polygon counted from the directory, then the chunks of mixed cells
        uint32_t *mask = static_cast<uint32_t *>(scratch);
        const uint64_t nchunks = (a.n + kWChunk - 1) / kWChunk;
        if ((e = cudaMemsetAsync(mask, 0, size_t((nchunks + 31) / 32) * 4, s)) != cudaSuccess)
            return e;
        const uint64_t ncell = uint64_t(1) << (2 * a.cluster_log2);
        const unsigned grid = unsigned(std::min<uint64_t>((ncell + 255) / 256, uint64_t(device_sm_count()) * 16));
        k_agg_cells<<<grid, 256, 0, s>>>(a.cell_end, a.cluster_log2, a.ix, a.counts, mask, a.stats);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        e = a.fp32 ? launch_warp_kernel<true, true, true>(a, use_hist, s, mask)
                   : launch_warp_kernel<false, true, true>(a, use_hist, s, mask);
    } else if (a.clustered)
        e = a.fp32 ? launch_warp_kernel<true, true>(a, use_hist, s) : launch_warp_kernel<false, true>(a, use_hist, s);
    else
        e = a.fp32 ? launch_warp_kernel<true, false>(a, use_hist, s) : launch_warp_kernel<false, false>(a, use_hist, s);
    if (ev)
        cudaEventRecord(ev[1], s);
    return e;
}

size_t select_scratch_bytes(uint64_t n, uint32_t P, uint64_t cap)
{
    return ((join_scratch_bytes(n) + 15) & ~size_t(15)) + n * 8 + 16 + cap * 8 + partition_scratch_bytes(cap, P);
}

size_t partition_scratch_bytes(uint64_t cap, uint32_t P)
{
    const uint64_t n_super = (cap + kSuperTile - 1) / kSuperTile;
    const uint64_t tab = uint64_t(P) * (n_super ? n_super : 1);
    return size_t(tab * 8 + (scan_partials(tab) + 2) * 8 + 64);
}

cudaError_t launch_partition(const uint2 *pairs, const unsigned long long *total, uint64_t cap, uint32_t P,
                             uint32_t *ids, unsigned long long *offsets, void *scratch, cudaStream_t s)
{
    if (P > (uint32_t)kSelMaxQ)
        return cudaErrorInvalidValue;
    const uint64_t n_super64 = (cap + kSuperTile - 1) / kSuperTile;
    if (n_super64 >= (1ull << 31))
        return cudaErrorInvalidValue;
    if (P == 0)
        return cudaMemsetAsync(offsets, 0, sizeof(unsigned long long), s);
    const uint32_t n_super = uint32_t(n_super64 ? n_super64 : 1);
    unsigned long long *table = static_cast<unsigned long long *>(scratch);
    unsigned long long *part = table + uint64_t(P) * n_super;
    unsigned long long *tab_total = part + scan_partials(uint64_t(P) * n_super) + 1;
    // per (query, super-tile) counts of the pairs, scanned in query-major order
    k_part_count<<<n_super, kThreads, sizeof(uint32_t) * P, s>>>(pairs, total, cap, P, table, n_super);
    cudaError_t e = launch_scan(table, uint64_t(P) * n_super, tab_total, part, s);
    if (e != cudaSuccess)
        return e;
    k_sel_offsets<<<(P + 256) / 256, 256, 0, s>>>(table, n_super, P, total, offsets);
    // point ids, ascending per query
    static bool done[64] = {};
    if ((e = smem_opt_in(k_part_emit, (sizeof(unsigned long long) + 4) * kWarps * kSelMaxQ, done)) != cudaSuccess)
        return e;
    if (cap)
        k_part_emit<<<n_super, kThreads, (sizeof(unsigned long long) + 4) * size_t(kWarps) * P, s>>>(
            pairs, total, P, table, n_super, ids, cap);
    return cudaGetLastError();
}

cudaError_t launch_select(const JoinLaunch &a, uint32_t *ids, uint64_t cap, unsigned long long *offsets,
                          void *scratch, cudaStream_t s)
{
    if (a.ix.P > (uint32_t)kSelMaxQ)
        return cudaErrorInvalidValue;
    char *sc = static_cast<char *>(scratch);
    void *join_scratch = sc;
    sc += (join_scratch_bytes(a.n) + 15) & ~size_t(15);
    // overlapping queries put many points in several polygons: pass 1b packs
    // their ids so that pass 3 does not walk them again
    uint64_t *aux = reinterpret_cast<uint64_t *>(sc);
    sc += a.n * 8;
    unsigned long long *total = reinterpret_cast<unsigned long long *>(sc);
    sc += 16;
    uint2 *pairs = reinterpret_cast<uint2 *>(sc);
    sc += cap * 8;
    // 1. the join: (point, query) pairs in point order, and their total
    JoinLaunch b = a;
    b.pairs = pairs;
    b.cap = cap;
    b.counts = nullptr;
    b.total = total;
    b.aux = aux;
    cudaError_t e = launch_join(b, join_scratch, s);
    if (e != cudaSuccess)
        return e;
    // 2. stable partition by query
    return launch_partition(pairs, total, cap, a.ix.P, ids, offsets, sc, s);
}

cudaError_t launch_join_plain(const JoinLaunch &a, void *scratch, cudaStream_t s)
{
    const uint64_t nb = (a.n + kPlainThreads - 1) / kPlainThreads;
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
    k_plain_count<<<(unsigned)nb, kPlainThreads, 0, s>>>(a, block);
    k_scan<<<1, 1024, 0, s>>>(block, nb, a.total);
    k_plain_write<<<(unsigned)nb, kPlainThreads, 0, s>>>(a, block);
    return cudaGetLastError();
}

// ------------------------------------------------------ multi-request launchers
namespace {
uint64_t multi_ntiles(uint64_t n) { return (n + kMChunk - 1) / kMChunk; }
uint64_t multi_part_words(uint64_t ntiles) { return scan_partials(ntiles) + 2; }
} // namespace

size_t multi_scratch_bytes(uint64_t n, int K)
{
    const uint64_t nt = multi_ntiles(n);
    return size_t(K) * size_t(nt + multi_part_words(nt)) * 8 + 256;
}

static cudaError_t multi_check(const MultiLaunch &m)
{
    if (m.K < 1 || m.K > kMaxBatch)
        return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(m.pts) & 7)
        return cudaErrorMisalignedAddress;
    if (multi_ntiles(m.n) >= (1ull << 31))
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t launch_multi_count(const MultiLaunch &m, void *scratch, cudaStream_t s)
{
    cudaError_t e = multi_check(m);
    if (e != cudaSuccess)
        return e;
    for (int r = 0; r < m.K; ++r)
        if (m.counts[r] && m.ix[r].P)
            if ((e = cudaMemsetAsync(m.counts[r], 0, sizeof(unsigned long long) * m.ix[r].P, s)) != cudaSuccess)
                return e;
    const uint64_t nt = multi_ntiles(m.n);
    if (nt == 0)
        return cudaMemsetAsync(m.totals, 0, sizeof(unsigned long long) * m.K, s);
    unsigned long long *tile_tot = static_cast<unsigned long long *>(scratch);
    unsigned long long *part = tile_tot + uint64_t(m.K) * nt;
    const int use_hist = m.qbase[m.K] <= kMultiHistMax ? 1 : 0;
    const size_t smem = kMultiSmem + (use_hist ? sizeof(uint32_t) * m.qbase[m.K] : 0);
    static bool done[2][64] = {};
    if (m.fp32) {
        if ((e = smem_opt_in(k_multi<true, false>, kMultiSmem + 4 * kMultiHistMax, done[0])) != cudaSuccess)
            return e;
        k_multi<true, false><<<persistent_grid(k_multi<true, false>, kThreads, smem, uint32_t((nt + kWarps - 1) / kWarps)), kThreads, smem,
                               s>>>(m, tile_tot, uint32_t(nt), use_hist);
    } else {
        if ((e = smem_opt_in(k_multi<false, false>, kMultiSmem + 4 * kMultiHistMax, done[1])) != cudaSuccess)
            return e;
        k_multi<false, false><<<persistent_grid(k_multi<false, false>, kThreads, smem, uint32_t((nt + kWarps - 1) / kWarps)), kThreads,
                                smem, s>>>(m, tile_tot, uint32_t(nt), use_hist);
    }
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    for (int r = 0; r < m.K; ++r)
        if ((e = launch_scan(tile_tot + uint64_t(r) * nt, nt, m.totals + r, part + uint64_t(r) * multi_part_words(nt),
                             s)) != cudaSuccess)
            return e;
    return cudaSuccess;
}

cudaError_t launch_multi_emit(const MultiLaunch &m, void *scratch, cudaStream_t s)
{
    cudaError_t e = multi_check(m);
    if (e != cudaSuccess)
        return e;
    const uint64_t nt = multi_ntiles(m.n);
    if (nt == 0)
        return cudaSuccess;
    unsigned long long *tile_tot = static_cast<unsigned long long *>(scratch);
    const size_t smem = kMultiSmem;
    static bool done[2][64] = {};
    const size_t smem_max = kMultiSmem;
    if (m.fp32) {
        if ((e = smem_opt_in(k_multi<true, true>, smem_max, done[0])) != cudaSuccess)
            return e;
        k_multi<true, true><<<persistent_grid(k_multi<true, true>, kThreads, smem, uint32_t((nt + kWarps - 1) / kWarps)), kThreads, smem,
                              s>>>(m, tile_tot, uint32_t(nt), 0);
    } else {
        if ((e = smem_opt_in(k_multi<false, true>, smem_max, done[1])) != cudaSuccess)
            return e;
        k_multi<false, true><<<persistent_grid(k_multi<false, true>, kThreads, smem, uint32_t((nt + kWarps - 1) / kWarps)), kThreads, smem,
                               s>>>(m, tile_tot, uint32_t(nt), 0);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------ plain path in two halves (serving comparison)
size_t plain_split_scratch_bytes(uint64_t n)
{
    const uint64_t nb = (n + kPlainThreads - 1) / kPlainThreads;
    return size_t(nb + scan_partials(nb) + 2) * 8 + 64;
}

cudaError_t launch_plain_count(const JoinLaunch &a, void *scratch, cudaStream_t s)
{
    const uint64_t nb = (a.n + kPlainThreads - 1) / kPlainThreads;
    if (nb >= (1ull << 31))
        return cudaErrorInvalidValue;
    cudaError_t e;
    if (a.counts && a.ix.P)
        if ((e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * a.ix.P, s)) != cudaSuccess)
            return e;
    if (nb == 0)
        return cudaMemsetAsync(a.total, 0, sizeof(unsigned long long), s);
    unsigned long long *block = static_cast<unsigned long long *>(scratch);
    k_plain_count<<<(unsigned)nb, kPlainThreads, 0, s>>>(a, block);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    return launch_scan(block, nb, a.total, block + nb, s);
}

cudaError_t launch_plain_write(const JoinLaunch &a, void *scratch, cudaStream_t s)
{
    const uint64_t nb = (a.n + kPlainThreads - 1) / kPlainThreads;
    if (nb == 0)
        return cudaSuccess;
    k_plain_write<<<(unsigned)nb, kPlainThreads, 0, s>>>(a, static_cast<const unsigned long long *>(scratch));
    return cudaGetLastError();
}

// ------------------------------------------------------ distance-query launchers
template <bool RESOLVE>
cudaError_t launch_dwarp(const DiskLaunch &a, unsigned long long *tot, uint32_t *res, uint32_t nchunks,
                         cudaStream_t s)
{
    static bool done[64] = {};
    const int use_hist = a.counts && a.dv.Q <= (uint32_t)kHistMax;
    const size_t fixed = kDWarpSmem + sizeof(uint32_t) * kDiskCoverWords;
    const size_t smem = fixed + (use_hist ? sizeof(uint32_t) * a.dv.Q : 0);
    auto kern = k_dwarp<RESOLVE>;
    cudaError_t e = smem_opt_in(kern, fixed + sizeof(uint32_t) * kHistMax, done);
    if (e != cudaSuccess)
        return e;
    const uint32_t nblk = (nchunks + kWarps - 1) / kWarps;
    kern<<<persistent_grid(kern, kThreads, smem, nblk), kThreads, smem, s>>>(a, tot, res, nchunks, use_hist);
    return cudaGetLastError();
}

// The polygon join's scratch layout: per-point results | per-chunk totals
// (then offsets) | scan partials.
size_t disk_scratch_bytes(uint64_t n) { return join_scratch_bytes(n); }

cudaError_t launch_disk_join(const DiskLaunch &a, void *scratch, cudaStream_t s, cudaEvent_t *ev)
{
    const uint64_t nchunks = (a.n + kWChunk - 1) / kWChunk;
    if (nchunks >= (1ull << 31))
        return cudaErrorInvalidValue;
    cudaError_t e;
    if (a.counts && a.dv.Q)
        if ((e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * a.dv.Q, s)) != cudaSuccess)
            return e;
    if (nchunks == 0)
        return a.total ? cudaMemsetAsync(a.total, 0, sizeof(unsigned long long), s) : cudaSuccess;
    char *sc = static_cast<char *>(scratch);
    uint32_t *res = reinterpret_cast<uint32_t *>(sc);
    unsigned long long *tot = reinterpret_cast<unsigned long long *>(sc + ((a.n * 4 + 15) & ~uint64_t(15)));
    unsigned long long *part = tot + nchunks;
    const uint32_t nblk = uint32_t((nchunks + kWarps - 1) / kWarps);
    if (ev)
        cudaEventRecord(ev[0], s);
    if ((e = launch_dwarp<true>(a, tot, res, uint32_t(nchunks), s)) != cudaSuccess)
        return e;
    if (ev)
        cudaEventRecord(ev[1], s);
    if ((e = launch_scan(tot, nchunks, a.total, part, s)) != cudaSuccess)
        return e;
    if (ev)
        cudaEventRecord(ev[2], s);
    if (a.cap) {
        static bool done[64] = {};
        if ((e = smem_opt_in(k_dwemit, kDEmitSmem, done)) != cudaSuccess)
            return e;
        k_dwemit<<<persistent_grid(k_dwemit, kThreads, kDEmitSmem, nblk), kThreads, kDEmitSmem, s>>>(
            a, tot, res, uint32_t(nchunks));
    }
    if (ev)
        cudaEventRecord(ev[3], s);
    return cudaGetLastError();
}

cudaError_t launch_disk_aggregate(const DiskLaunch &a, cudaStream_t s)
{
    const uint64_t nchunks = (a.n + kWChunk - 1) / kWChunk;
    if (nchunks >= (1ull << 31))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * (a.dv.Q ? a.dv.Q : 1), s);
    if (e != cudaSuccess || nchunks == 0)
        return e;
    return launch_dwarp<false>(a, nullptr, nullptr, uint32_t(nchunks), s);
}

size_t disk_select_scratch_bytes(uint64_t n, uint32_t Q, uint64_t cap)
{
    return ((disk_scratch_bytes(n) + 15) & ~size_t(15)) + 16 + cap * 8 + partition_scratch_bytes(cap, Q);
}

cudaError_t launch_disk_select(const DiskLaunch &a, uint32_t *ids, uint64_t cap, unsigned long long *offsets,
                               void *scratch, cudaStream_t s)
{
    if (a.dv.Q > (uint32_t)kSelMaxQ)
        return cudaErrorInvalidValue;
    char *sc = static_cast<char *>(scratch);
    void *join_scratch = sc;
    sc += (disk_scratch_bytes(a.n) + 15) & ~size_t(15);
    unsigned long long *total = reinterpret_cast<unsigned long long *>(sc);
    sc += 16;
    uint2 *pairs = reinterpret_cast<uint2 *>(sc);
    sc += cap * 8;
    DiskLaunch b = a;
    b.pairs = pairs;
    b.cap = cap;
    b.counts = nullptr;
    b.total = total;
    cudaError_t e = launch_disk_join(b, join_scratch, s, nullptr);
    if (e != cudaSuccess)
        return e;
    return launch_partition(pairs, total, cap, a.dv.Q, ids, offsets, sc, s);
}

// ------------------------------------------------ buffered polygons: launchers
__global__ void k_buf_mask(const uint32_t *cell, int gp, uint32_t *mask, int g)
{
    const uint64_t n = uint64_t(1) << (2 * gp);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (!cell[i])
            continue;
        const uint32_t cx = uint32_t(i & ((1u << gp) - 1)), cy = uint32_t(i >> gp);
        if (g <= gp) { // one mask cell holds 2^(gp - g) x 2^(gp - g) coarse cells
            const uint32_t m = ((cy >> (gp - g)) << g) | (cx >> (gp - g));
            atomicOr(mask + (m >> 5), 1u << (m & 31));
        } else { // the coarse cell spans 2^(g - gp) x 2^(g - gp) mask cells
            const uint32_t k = 1u << (g - gp);
            for (uint32_t y = cy * k; y < (cy + 1) * k; ++y)
                for (uint32_t x = cx * k; x < (cx + 1) * k; ++x) {
                    const uint32_t m = (y << g) | x;
                    atomicOr(mask + (m >> 5), 1u << (m & 31));
                }
        }
    }
}

cudaError_t launch_buffer_mask(const IndexView &ix, uint32_t *mask, int g, cudaStream_t s)
{
    const uint64_t n = uint64_t(1) << (2 * ix.gc);
    const unsigned grid = unsigned(std::min<uint64_t>((n + 255) / 256, uint64_t(device_sm_count()) * 32));
    k_buf_mask<<<grid, 256, 0, s>>>(ix.cell, ix.gc, mask, g);
    return cudaGetLastError();
}


size_t buffer_scratch_bytes(uint64_t n)
{
    const uint64_t nb = (n + kPlainThreads - 1) / kPlainThreads;
    return size_t(((n * 4 + 15) & ~uint64_t(15)) + (nb + scan_partials(nb) + 2) * 8 + 16);
}

cudaError_t launch_buffer_join(const BufferLaunch &a, void *scratch, cudaStream_t s)
{
    if (a.n >= (1ull << 32))
        return cudaErrorInvalidValue; // point ids are 32-bit
    cudaError_t e = cudaSuccess;
    if (a.counts && a.bv.P)
        e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * a.bv.P, s);
    if (e != cudaSuccess)
        return e;
    if (a.n == 0)
        return a.total ? cudaMemsetAsync(a.total, 0, sizeof(unsigned long long), s) : cudaSuccess;
    const uint64_t nb = (a.n + kPlainThreads - 1) / kPlainThreads;
    char *sc = static_cast<char *>(scratch);
    uint32_t *pt_cnt = reinterpret_cast<uint32_t *>(sc);
    unsigned long long *block = reinterpret_cast<unsigned long long *>(sc + ((a.n * 4 + 15) & ~uint64_t(15)));
    unsigned long long *part = block + nb;
    if (a.fp32)
        k_buf_count<true><<<(unsigned)nb, kPlainThreads, 0, s>>>(a, pt_cnt, block);
    else
        k_buf_count<false><<<(unsigned)nb, kPlainThreads, 0, s>>>(a, pt_cnt, block);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    if ((e = launch_scan(block, nb, a.total, part, s)) != cudaSuccess)
        return e;
    if (!a.cap)
        return cudaSuccess;
    if (a.fp32)
        k_buf_write<true><<<(unsigned)nb, kPlainThreads, 0, s>>>(a, pt_cnt, block);
    else
        k_buf_write<false><<<(unsigned)nb, kPlainThreads, 0, s>>>(a, pt_cnt, block);
    return cudaGetLastError();
}

cudaError_t launch_buffer_aggregate(const BufferLaunch &a, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * (a.bv.P ? a.bv.P : 1), s);
    if (e != cudaSuccess || a.n == 0)
        return e;
    const uint64_t nb = (a.n + kPlainThreads - 1) / kPlainThreads;
    if (nb >= (1ull << 31))
        return cudaErrorInvalidValue;
    if (a.fp32)
        k_buf_count<true><<<(unsigned)nb, kPlainThreads, 0, s>>>(a, nullptr, nullptr);
    else
        k_buf_count<false><<<(unsigned)nb, kPlainThreads, 0, s>>>(a, nullptr, nullptr);
    return cudaGetLastError();
}

size_t buffer_select_scratch_bytes(uint64_t n, uint32_t P, uint64_t cap)
{
    return ((buffer_scratch_bytes(n) + 15) & ~size_t(15)) + 16 + cap * 8 + partition_scratch_bytes(cap, P);
}

cudaError_t launch_buffer_select(const BufferLaunch &a, uint32_t *ids, uint64_t cap, unsigned long long *offsets,
                                 void *scratch, cudaStream_t s)
{
    if (a.bv.P > (uint32_t)kSelMaxQ)
        return cudaErrorInvalidValue;
    char *sc = static_cast<char *>(scratch);
    void *join_scratch = sc;
    sc += (buffer_scratch_bytes(a.n) + 15) & ~size_t(15);
    unsigned long long *total = reinterpret_cast<unsigned long long *>(sc);
    sc += 16;
    uint2 *pairs = reinterpret_cast<uint2 *>(sc);
    sc += cap * 8;
    BufferLaunch b = a;
    b.pairs = pairs;
    b.cap = cap;
    b.counts = nullptr;
    b.total = total;
    cudaError_t e = launch_buffer_join(b, join_scratch, s);
    if (e != cudaSuccess)
        return e;
    return launch_partition(pairs, total, cap, a.bv.P, ids, offsets, sc, s);
}

} // namespace spx
