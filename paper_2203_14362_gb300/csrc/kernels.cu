// sm_103a kernels of libspx: the point-in-polygon join, count aggregate and
// the plain comparison join (SPADE §5.2 selection / join / aggregation; the
// per-point work of the paper's fragment shader: mask with exact boundary
// tests, additive blend for counts, Map with scan compaction, §5.1).
//
// Per point (one thread):
//   cell   = (y >> shift) << g | (x >> shift)               -- geometric transform
//   word   = cell word: empty / one INSIDE polygon / entry list
//   entry  INSIDE   -> the point is in the polygon          -- mask, inside pixel
//          BOUNDARY -> crossing parity over the row's edges -- mask, boundary pixel
// The crossing rule is exact: an edge a->b counts iff it straddles y
// ((a.y > y) != (b.y > y)) and the orientation d = (b.x-a.x)(y-a.y) -
// (b.y-a.y)(x-a.x) is nonzero with the sign of b.y - a.y.  d is taken from
// FP32 when |d_f| > 2^-21 (|t1| + |t2|) (forward error bound of the FP32
// evaluation, factor 2 margin), else recomputed exactly in int64.
#include "kernels.h"
#include "spx_internal.h"

#include <cuda_runtime.h>

namespace spx {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;                    // points per thread per tile
constexpr int kTile = kThreads * kItems;     // 2048 points per tile
constexpr uint32_t kFull = 0xffffffffu;
constexpr int kHistMax = 11776;              // polygons counted in shared memory (46 KB, under the 48 KB default)

constexpr unsigned long long kFlagAgg = 1ull << 62;   // tile total published
constexpr unsigned long long kFlagPre = 2ull << 62;   // inclusive prefix published
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr unsigned kSpinLimit = 1u << 22;             // ~ seconds with the back-off below

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

// Parity of the crossings of the rightward ray from (px, py) with a row edge
// list sorted by max x descending.
template <bool FP32>
__device__ __forceinline__ uint32_t row_parity(const int4 *__restrict__ e, uint32_t n, int px, int py,
                                               uint32_t &tests, uint32_t &esc)
{
    uint32_t par = 0;
    for (uint32_t k = 0; k < n; ++k) {
        const int4 v = __ldg(e + k);
        if (max(v.x, v.z) <= px)
            break; // this and every later edge ends left of p: no crossing right of p
        if ((v.y > py) == (v.w > py))
            continue; // does not straddle
        if (min(v.x, v.z) > px) {
            par ^= 1u; // the crossing lies right of p
            continue;
        }
        ++tests;
        const int s = orient_sign<FP32>(v.x, v.y, v.z, v.w, px, py, esc);
        par ^= uint32_t((s != 0) & ((s > 0) == (v.w > v.y)));
    }
    return par;
}

// Number of polygons containing (px, py) and the smallest such polygon id.
template <bool FP32>
__device__ __forceinline__ uint32_t point_count(const IndexView &ix, int px, int py, uint32_t &first,
                                                uint32_t &tests, uint32_t &esc)
{
    if ((unsigned)px >= kBox || (unsigned)py >= kBox)
        return 0;
    const uint32_t w =
        __ldg(ix.cell + ((((unsigned)py >> ix.shift) << ix.glog2) | ((unsigned)px >> ix.shift)));
    const uint32_t kind = w >> 30;
    if (kind == kCellEmpty)
        return 0;
    if (kind == kCellInsideOne) {
        first = w & kPayloadMask;
        return 1;
    }
    const uint4 *e = ix.ent + (w & kPayloadMask);
    uint32_t c = 0;
    for (;;) {
        const uint4 en = __ldg(e++);
        const uint32_t in =
            (en.w & kEntBoundary) ? row_parity<FP32>(ix.edge + en.y, en.z, px, py, tests, esc) : 1u;
        if (in) {
            if (c == 0)
                first = en.x;
            ++c;
        }
        if (en.w & kEntLast)
            break;
    }
    return c;
}

// Calls f(polygon) for every polygon containing (px, py), ascending.
template <bool FP32, class F>
__device__ __forceinline__ void point_emit(const IndexView &ix, int px, int py, F f)
{
    uint32_t t = 0, s = 0;
    const uint32_t w =
        __ldg(ix.cell + ((((unsigned)py >> ix.shift) << ix.glog2) | ((unsigned)px >> ix.shift)));
    if ((w >> 30) != kCellList)
        return; // only lists hold more than one polygon
    const uint4 *e = ix.ent + (w & kPayloadMask);
    for (;;) {
        const uint4 en = __ldg(e++);
        if (!(en.w & kEntBoundary) || row_parity<FP32>(ix.edge + en.y, en.z, px, py, t, s))
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
    unsigned long long a = warp_sum64(pts), b = warp_sum64(tests), c = warp_sum64(esc), d = warp_sum64(pairs);
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(stats + kStatPoints, a);
        if (b) atomicAdd(stats + kStatTests, b);
        if (c) atomicAdd(stats + kStatEscalations, c);
        if (d) atomicAdd(stats + kStatPairs, d);
    }
}

// Decoupled look-back (single-pass chained scan): publish this tile's total,
// then walk back over predecessor tiles, 32 at a time, until one has published
// its inclusive prefix.  Tiles are claimed in order from an atomic counter, so
// every tile waited on belongs to a CTA that is already running and has
// published (or will publish without waiting on us): the wait always ends.
// The wait is still bounded; on expiry the error word gets kErrTimeout.
__device__ unsigned long long lookback(unsigned long long *status, uint32_t tile, uint32_t total, unsigned *err)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0)
            st_relaxed(status, kFlagPre | total);
        return 0;
    }
    if (lane == 0)
        st_relaxed(status + tile, kFlagAgg | total);
    unsigned long long excl = 0;
    long long top = (long long)tile - 1;
    unsigned spins = 0;
    for (;;) {
        const long long k = top - lane;
        const unsigned long long s = (k >= 0) ? ld_relaxed(status + k) : kFlagPre;
        if (__any_sync(kFull, (s >> 62) == 0)) {
            if (++spins > kSpinLimit) {
                if (lane == 0)
                    atomicOr(err, kErrTimeout);
                break;
            }
            __nanosleep(64);
            continue;
        }
        const uint32_t pm = __ballot_sync(kFull, (s >> 62) == 2);
        if (pm) {
            const int fp = __ffs(pm) - 1;
            excl += warp_sum64(lane <= fp ? (s & kValMask) : 0ull);
            break;
        }
        excl += warp_sum64(s & kValMask);
        top -= 32;
    }
    if (lane == 0)
        st_relaxed(status + tile, kFlagPre | (excl + total));
    return excl;
}

// ---------------------------------------------------------------- fused join
// Persistent: each CTA claims 2048-point tiles in order; per tile it evaluates
// its points, scans the per-point match counts (warp ballots, one warp for the
// 64 warp-row totals), obtains the tile's global offset by look-back and
// writes the pairs, so the output is sorted by point id (and polygon id within
// a point, entries being sorted) in one pass over the points.
template <bool FP32>
__global__ void __launch_bounds__(kThreads) k_join(JoinLaunch a, uint32_t ntiles, int use_hist)
{
    extern __shared__ uint32_t s_hist[];
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_off[kItems * kWarps];
    __shared__ unsigned long long s_excl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (use_hist)
        for (uint32_t i = tid; i < a.ix.P; i += kThreads)
            s_hist[i] = 0;
    uint32_t n_tests = 0, n_esc = 0, n_pts = 0, n_pairs = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0)
            s_tile = atomicAdd(a.tile_counter, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles)
            break;
        const uint64_t base = (uint64_t)tile * kTile;
        uint32_t cnt[kItems], first[kItems], pre[kItems];
        bool multi = false;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const uint64_t idx = base + (uint64_t)(i * kThreads + tid);
            cnt[i] = 0;
            first[i] = 0;
            if (idx < a.n) {
                const int2 p = __ldcs(a.pts + idx);
                cnt[i] = point_count<FP32>(a.ix, p.x, p.y, first[i], n_tests, n_esc);
                ++n_pts;
                multi |= cnt[i] > 1;
            }
        }
        multi = __any_sync(kFull, multi);
        if (!multi) {
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                const uint32_t b = __ballot_sync(kFull, cnt[i] != 0);
                pre[i] = __popc(b & lanemask_lt());
                if (lane == 0)
                    s_off[i * kWarps + warp] = __popc(b);
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
            const unsigned long long excl = lookback(a.tile_status, tile, tile_total, a.err);
            if (lane == 0) {
                s_excl = excl;
                if (tile == ntiles - 1 && a.total)
                    *a.total = excl + tile_total;
            }
        }
        __syncthreads();
        const unsigned long long tbase = s_excl;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if (!cnt[i])
                continue;
            const uint64_t idx = base + (uint64_t)(i * kThreads + tid);
            unsigned long long o = tbase + s_off[i * kWarps + warp] + pre[i];
            n_pairs += cnt[i];
            if (cnt[i] == 1) {
                if (o < a.cap)
                    __stcs(a.pairs + o, make_uint2((uint32_t)idx, first[i]));
                if (use_hist)
                    atomicAdd(&s_hist[first[i]], 1u);
                else if (a.counts)
                    atomicAdd(a.counts + first[i], 1ull);
            } else {
                const int2 p = __ldg(a.pts + idx);
                point_emit<FP32>(a.ix, p.x, p.y, [&](uint32_t q) {
                    if (o < a.cap)
                        __stcs(a.pairs + o, make_uint2((uint32_t)idx, q));
                    ++o;
                    if (use_hist)
                        atomicAdd(&s_hist[q], 1u);
                    else if (a.counts)
                        atomicAdd(a.counts + q, 1ull);
                });
            }
        }
    }
    add_stats(a.stats, n_pts, n_tests, n_esc, n_pairs);
    if (use_hist && a.counts) {
        __syncthreads();
        for (uint32_t i = tid; i < a.ix.P; i += kThreads)
            if (s_hist[i])
                atomicAdd(a.counts + i, (unsigned long long)s_hist[i]);
    }
}

// ---------------------------------------------------------- count aggregate
// No materialisation (§5.2, the aggregation plan for points): counts only,
// grid-stride over point pairs with 16-byte loads.
template <bool FP32>
__global__ void __launch_bounds__(kThreads) k_count(JoinLaunch a, int use_hist)
{
    extern __shared__ uint32_t s_hist[];
    const int tid = threadIdx.x;
    if (use_hist) {
        for (uint32_t i = tid; i < a.ix.P; i += kThreads)
            s_hist[i] = 0;
        __syncthreads();
    }
    uint32_t n_tests = 0, n_esc = 0, n_pts = 0, n_pairs = 0;
    auto add = [&](uint32_t q) {
        ++n_pairs;
        if (use_hist)
            atomicAdd(&s_hist[q], 1u);
        else
            atomicAdd(a.counts + q, 1ull);
    };
    auto one = [&](int px, int py) {
        uint32_t first = 0;
        const uint32_t c = point_count<FP32>(a.ix, px, py, first, n_tests, n_esc);
        ++n_pts;
        if (c == 1)
            add(first);
        else if (c > 1)
            point_emit<FP32>(a.ix, px, py, add);
    };
    const uint64_t npairs = a.n / 2;
    const int4 *p4 = reinterpret_cast<const int4 *>(a.pts);
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    for (uint64_t i = (uint64_t)blockIdx.x * kThreads + tid; i < npairs; i += stride) {
        const int4 v = __ldcs(p4 + i);
        one(v.x, v.y);
        one(v.z, v.w);
    }
    if ((a.n & 1) && blockIdx.x == 0 && tid == 0) {
        const int2 v = a.pts[a.n - 1];
        one(v.x, v.y);
    }
    add_stats(a.stats, n_pts, n_tests, n_esc, n_pairs);
    if (use_hist) {
        __syncthreads();
        for (uint32_t i = tid; i < a.ix.P; i += kThreads)
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
        c = point_count<false>(a.ix, p.x, p.y, first, t, e);
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
    // exclusive scan of n values by one block: chunks of 1024, carried total
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
            unsigned long long w = s_w[lane], wi = w;
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
    if (idx < a.n) {
        p = a.pts[idx];
        c = point_count<false>(a.ix, p.x, p.y, first, t, e);
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
        point_emit<false>(a.ix, p.x, p.y, [&](uint32_t q) {
            if (o < a.cap)
                a.pairs[o] = make_uint2((uint32_t)idx, q);
            ++o;
            if (a.counts)
                atomicAdd(a.counts + q, 1ull);
        });
    }
}

int g_sm_count = 0;

} // namespace

int device_sm_count()
{
    int dev = 0;
    cudaGetDevice(&dev);
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_sm_count = n;
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

template <class K>
static int persistent_grid(K kernel, size_t smem)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
    if (per_sm < 1)
        per_sm = 1;
    return per_sm * device_sm_count();
}

cudaError_t launch_join(const JoinLaunch &a, void *scratch, cudaStream_t s)
{
    const uint64_t ntiles64 = (a.n + kTile - 1) / kTile;
    if (ntiles64 >= (1ull << 32))
        return cudaErrorInvalidValue;
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
    const size_t smem = use_hist ? sizeof(uint32_t) * a.ix.P : 0;
    if (a.fp32) {
        int grid = persistent_grid(k_join<true>, smem);
        if ((uint32_t)grid > ntiles) grid = (int)ntiles;
        k_join<true><<<grid, kThreads, smem, s>>>(b, ntiles, use_hist);
    } else {
        int grid = persistent_grid(k_join<false>, smem);
        if ((uint32_t)grid > ntiles) grid = (int)ntiles;
        k_join<false><<<grid, kThreads, smem, s>>>(b, ntiles, use_hist);
    }
    return cudaGetLastError();
}

cudaError_t launch_aggregate(const JoinLaunch &a, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * (a.ix.P ? a.ix.P : 1), s);
    if (e != cudaSuccess || a.n == 0)
        return e;
    const int use_hist = a.ix.P <= (uint32_t)kHistMax ? 1 : 0;
    const size_t smem = use_hist ? sizeof(uint32_t) * a.ix.P : 0;
    const uint64_t work = (a.n / 2 + kThreads - 1) / kThreads;
    if (a.fp32) {
        int grid = persistent_grid(k_count<true>, smem);
        if ((uint64_t)grid > work) grid = int(work ? work : 1);
        k_count<true><<<grid, kThreads, smem, s>>>(a, use_hist);
    } else {
        int grid = persistent_grid(k_count<false>, smem);
        if ((uint64_t)grid > work) grid = int(work ? work : 1);
        k_count<false><<<grid, kThreads, smem, s>>>(a, use_hist);
    }
    return cudaGetLastError();
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
