// Device build of the polygon grid index (SPADE §4.2 canvas creation by
// conservative rasterisation of the polygons' boundaries, §4.3 boundary
// index; §6.1 builds the index of query-time polygons on the fly and counts
// it in the query time).  It takes the same decisions as the host build
// (index_build.cpp), stage by stage, so the arrays are the same bytes:
//   1. per polygon, its box in coarse and fine cells (a warp per polygon);
//   2. per edge (a thread per edge): the conservative marks of the cells its
//      pieces can meet at both levels (mixed coarse cells, BOUNDARY fine
//      cells), the toggles of the corner thresholds of every coarse and fine
//      row corner it straddles, and the count of the fine rows it lies in;
//   3. per coarse row of a box, the suffix parity of the toggles classifies
//      every coarse cell no edge meets; per fine row, the same for the fine
//      cells of mixed coarse cells, and whether the row needs an edge list;
//   4. the fine rows' edge lists, each sorted by right end descending, then
//      ring order (the host's stable sort), laid out polygon by polygon;
//   5. the (coarse cell, polygon) records bucketed by cell and sorted by
//      polygon, then coarse words, fine blocks and entries in cell order, as
//      the host's merge writes them; then the cover bitmap and block summary.
// No kernel here waits on another; every limit of the index format is
// checked as the host build checks it.
#include "kernels.h"
#include "spx_internal.h"

#include <algorithm>
#include <cuda_runtime.h>
#include <vector>

namespace spx {
namespace {

struct PBox {
    int32_t cx0, cx1, cy0, cy1; // coarse columns and rows of the half-open box (cx1 < cx0: no cell)
    int32_t fx0, fx1, fy0, fy1; // fine columns and rows
};

__device__ __forceinline__ long long fdiv(long long a, long long b) // floor(a / b), b > 0
{
    const long long q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}
__device__ __forceinline__ long long cdiv(long long a, long long b) // ceil(a / b), b > 0
{
    const long long q = a / b;
    return (a % b != 0 && a > 0) ? q + 1 : q;
}
// x of the line through a -> b at height Y, as floor and ceil (exact rationals)
__device__ __forceinline__ void line_x(long long ax, long long ay, long long bx, long long by, long long Y,
                                       long long &fl, long long &ce)
{
    long long num = (bx - ax) * (Y - ay), den = by - ay;
    if (den < 0) {
        num = -num;
        den = -den;
    }
    fl = ax + fdiv(num, den);
    ce = ax + cdiv(num, den);
}
// The edge a -> b straddles the corner row at height y0: the corners (x0, y0)
// left of its crossing x* are those with x0 <= ceil(x*) - 1; the largest such
// cell column of side S.
__device__ __forceinline__ long long corner_col(long long ax, long long ay, long long bx, long long by, long long y0,
                                                long long S)
{
    long long num = (bx - ax) * (y0 - ay), den = by - ay;
    if (den < 0) {
        num = -num;
        den = -den;
    }
    return fdiv(ax + cdiv(num, den) - 1, S);
}

// the polygon owning vertex (and edge) i: the largest q with off[q] <= i
__device__ __forceinline__ uint32_t owner(const uint64_t *off, uint32_t P, uint64_t i)
{
    uint32_t lo = 0, hi = P; // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

constexpr int kT = 256;
constexpr uint32_t kFullMask = 0xffffffffu;

// 1. boxes; ncc / nfr / nfw: coarse cells, fine rows and fine toggle words of each box
__global__ void __launch_bounds__(kT) k_ib_box(const int2 *v, const uint64_t *off, uint32_t P, int g, int sb,
                                               PBox *box, unsigned long long *ncc, unsigned long long *nfr,
                                               unsigned long long *nfw)
{
    const int lane = threadIdx.x & 31;
    const uint32_t w0 = (blockIdx.x * kT + threadIdx.x) >> 5, nwarp = (gridDim.x * kT) >> 5;
    const int sc = kBoxLog2 - g, sf = kBoxLog2 - g - sb;
    const long long Gc = 1ll << g, Gf = 1ll << (g + sb);
    for (uint32_t q = w0; q < P; q += nwarp) {
        const uint64_t a = off[q], b = off[q + 1];
        int xmin = INT32_MAX, xmax = INT32_MIN, ymin = INT32_MAX, ymax = INT32_MIN;
        for (uint64_t k = a + lane; k < b; k += 32) {
            const int2 p = v[k];
            xmin = min(xmin, p.x);
            xmax = max(xmax, p.x);
            ymin = min(ymin, p.y);
            ymax = max(ymax, p.y);
        }
        xmin = __reduce_min_sync(kFullMask, xmin);
        xmax = __reduce_max_sync(kFullMask, xmax);
        ymin = __reduce_min_sync(kFullMask, ymin);
        ymax = __reduce_max_sync(kFullMask, ymax);
        PBox bx{0, -1, 0, -1, 0, -1, 0, -1};
        // fewer than 3 vertices, or an empty half-open box: no point is inside
        if (b - a >= 3 && xmax > xmin && ymax > ymin) {
            bx.cx0 = xmin >> sc;
            bx.cx1 = (int32_t)min((long long)((xmax - 1) >> sc), Gc - 1);
            bx.cy0 = ymin >> sc;
            bx.cy1 = (int32_t)min((long long)((ymax - 1) >> sc), Gc - 1);
            bx.fx0 = xmin >> sf;
            bx.fx1 = (int32_t)min((long long)((xmax - 1) >> sf), Gf - 1);
            bx.fy0 = ymin >> sf;
            bx.fy1 = (int32_t)min((long long)((ymax - 1) >> sf), Gf - 1);
        }
        if (lane == 0) {
            box[q] = bx;
            const unsigned long long wc = (unsigned long long)(bx.cx1 - bx.cx0 + 1),
                                     hc = (unsigned long long)(bx.cy1 - bx.cy0 + 1),
                                     wf = (unsigned long long)(bx.fx1 - bx.fx0 + 1),
                                     hf = (unsigned long long)(bx.fy1 - bx.fy0 + 1);
            ncc[q] = wc * hc;
            nfr[q] = hf;
            nfw[q] = hf * ((wf + 31) / 32);
        }
    }
}

// 2. per edge: marks, corner toggles, fine-row counts
__global__ void __launch_bounds__(kT) k_ib_mark(const int2 *v, const uint64_t *off, uint32_t P, uint64_t V, int g,
                                                int sb, const PBox *box, const unsigned long long *ccoff,
                                                const unsigned long long *froff, const unsigned long long *fwoff,
                                                uint32_t *cmix, uint32_t *cflip, unsigned long long *fbnd,
                                                uint32_t *fflip, uint32_t *rcnt)
{
    const int sc = kBoxLog2 - g, sf = kBoxLog2 - g - sb, F = 1 << sb;
    const long long Sc = 1ll << sc, Sf = 1ll << sf;
    for (uint64_t i = blockIdx.x * (uint64_t)kT + threadIdx.x; i < V; i += (uint64_t)gridDim.x * kT) {
        const uint32_t q = owner(off, P, i);
        const PBox b = box[q];
        if (b.cx1 < b.cx0)
            continue;
        const uint64_t j = (i + 1 == off[q + 1]) ? off[q] : i + 1;
        const int2 pa = v[i], pb = v[j];
        const long long ax = pa.x, ay = pa.y, bx = pb.x, by = pb.y;
        const long long wc = b.cx1 - b.cx0 + 1, wwords = (b.fx1 - b.fx0 + 1 + 31) / 32;
        const unsigned long long cbase = ccoff[q];
        // coarse cells [lo, hi] of row `row` are mixed
        auto mark_c = [&](long long row, long long lo, long long hi) {
            if (row < b.cy0 || row > b.cy1)
                return;
            lo = max(lo, (long long)b.cx0);
            hi = min(hi, (long long)b.cx1);
            for (long long c = lo; c <= hi; ++c)
                atomicOr(cmix + cbase + (row - b.cy0) * wc + (c - b.cx0), 1u);
        };
        // fine cells [lo, hi] of fine row `fr` are BOUNDARY: one OR per coarse cell
        auto mark_f = [&](long long fr, long long lo, long long hi) {
            if (fr < b.fy0 || fr > b.fy1)
                return;
            lo = max(lo, (long long)b.fx0);
            hi = min(hi, (long long)b.fx1);
            const long long crow = (fr >> sb) - b.cy0;
            const int bit0 = int(fr & (F - 1)) * F;
            for (long long fx = lo; fx <= hi;) {
                const long long ce = min(hi, (fx | (F - 1)));
                const int n = int(ce - fx + 1), s = int(fx & (F - 1)); // n <= F <= 8
                const unsigned long long m = ((1ull << n) - 1) << (bit0 + s);
                atomicOr(fbnd + cbase + crow * wc + ((fx >> sb) - b.cx0), m);
                fx = ce + 1;
            }
        };
        if (ay == by) {
            // a horizontal edge meets the open squares of its row unless it lies on a row border
            const long long lo = min(ax, bx), hi = max(ax, bx);
            if (ay % Sc != 0)
                mark_c(ay >> sc, fdiv(lo, Sc), cdiv(hi, Sc) - 1);
            if (ay % Sf != 0)
                mark_f(ay >> sf, fdiv(lo, Sf), cdiv(hi, Sf) - 1);
            continue; // never straddles a corner row, in no row list
        }
        const long long lo_y = min(ay, by), hi_y = max(ay, by);
        for (long long row = max(lo_y >> sc, (long long)b.cy0), r1 = min(cdiv(hi_y, Sc) - 1, (long long)b.cy1);
             row <= r1; ++row) {
            long long fa, ca, fb, cb;
            line_x(ax, ay, bx, by, max(lo_y, row * Sc), fa, ca);
            line_x(ax, ay, bx, by, min(hi_y, (row + 1) * Sc), fb, cb);
            mark_c(row, fdiv(min(fa, fb), Sc), cdiv(max(ca, cb), Sc) - 1);
        }
        // coarse corner rows y0 = cy Sc with lo_y <= y0 < hi_y
        for (long long cy = max(cdiv(lo_y, Sc), (long long)b.cy0), c1 = min(cdiv(hi_y, Sc) - 1, (long long)b.cy1);
             cy <= c1; ++cy) {
            const long long kx = corner_col(ax, ay, bx, by, cy * Sc, Sc);
            if (kx >= b.cx0)
                atomicXor(cflip + cbase + (cy - b.cy0) * wc + (min(kx, (long long)b.cx1) - b.cx0), 1u);
        }
        for (long long fr = max(lo_y >> sf, (long long)b.fy0), r1 = min(cdiv(hi_y, Sf) - 1, (long long)b.fy1);
             fr <= r1; ++fr) {
            atomicAdd(rcnt + froff[q] + (fr - b.fy0), 1u);
            long long fa, ca, fb, cb;
            line_x(ax, ay, bx, by, max(lo_y, fr * Sf), fa, ca);
            line_x(ax, ay, bx, by, min(hi_y, (fr + 1) * Sf), fb, cb);
            mark_f(fr, fdiv(min(fa, fb), Sf), cdiv(max(ca, cb), Sf) - 1);
        }
        // fine corner rows
        for (long long fy = max(cdiv(lo_y, Sf), (long long)b.fy0), f1 = min(cdiv(hi_y, Sf) - 1, (long long)b.fy1);
             fy <= f1; ++fy) {
            const long long kf = corner_col(ax, ay, bx, by, fy * Sf, Sf);
            if (kf >= b.fx0) {
                const long long col = min(kf, (long long)b.fx1) - b.fx0;
                atomicXor(fflip + fwoff[q] + (fy - b.fy0) * wwords + (col >> 5), 1u << (col & 31));
            }
        }
    }
}

// 3a. coarse rows: status of every box cell (0 none, 1 INSIDE, 2 mixed) and
// the records per grid cell.  A block per polygon, a thread per row.
__global__ void __launch_bounds__(kT) k_ib_coarse(uint32_t P, int g, const PBox *box,
                                                  const unsigned long long *ccoff, const uint32_t *cmix,
                                                  const uint32_t *cflip, uint8_t *cst, unsigned long long *cell_cnt,
                                                  unsigned long long *counters)
{
    unsigned long long n_in = 0, n_mx = 0;
    for (uint32_t q = blockIdx.x; q < P; q += gridDim.x) {
        const PBox b = box[q];
        if (b.cx1 < b.cx0)
            continue;
        const long long wc = b.cx1 - b.cx0 + 1, hc = b.cy1 - b.cy0 + 1;
        for (long long r = threadIdx.x; r < hc; r += kT) {
            uint32_t par = 0;
            for (long long c = wc - 1; c >= 0; --c) {
                const unsigned long long k = ccoff[q] + r * wc + c;
                par ^= cflip[k] & 1u; // parity of the toggles at columns >= c
                const uint8_t st = cmix[k] ? 2 : (par ? 1 : 0);
                cst[k] = st;
                if (st) {
                    atomicAdd(cell_cnt + ((uint64_t(b.cy0 + r) << g) | uint64_t(b.cx0 + c)), 1ull);
                    n_in += st == 1;
                    n_mx += st == 2;
                }
            }
        }
    }
    atomicAdd(counters + 0, n_in);
    atomicAdd(counters + 1, n_mx);
}

// suffix XOR within a word: bit i = XOR of bits i..31
__device__ __forceinline__ uint32_t suffix_xor(uint32_t x)
{
    x ^= x >> 1;
    x ^= x >> 2;
    x ^= x >> 4;
    x ^= x >> 8;
    x ^= x >> 16;
    return x;
}

// 3b. fine rows: the INSIDE fine cells of mixed coarse cells, whether the row
// needs an edge list (it holds a BOUNDARY fine cell of a mixed coarse cell),
// and its list length.  A block per polygon, a thread per fine row.
__global__ void __launch_bounds__(kT) k_ib_fine(uint32_t P, int sb, const PBox *box, const unsigned long long *ccoff,
                                                const unsigned long long *froff, const unsigned long long *fwoff,
                                                const uint8_t *cst, const unsigned long long *fbnd, uint32_t *fflip,
                                                const uint32_t *rcnt, unsigned long long *finside, uint32_t *rlen,
                                                unsigned long long *rsz, uint32_t *rpoly, unsigned long long *counters)
{
    const int F = 1 << sb;
    const unsigned long long row_bits = (F == 8) ? 0xFFull : ((1ull << F) - 1);
    unsigned long long n_b = 0;
    for (uint32_t q = blockIdx.x; q < P; q += gridDim.x) {
        const PBox b = box[q];
        if (b.cx1 < b.cx0)
            continue;
        const long long wc = b.cx1 - b.cx0 + 1, hf = b.fy1 - b.fy0 + 1, ww = (b.fx1 - b.fx0 + 1 + 31) / 32;
        for (long long r = threadIdx.x; r < hf; r += kT) {
            const long long fy = b.fy0 + r, crow = (fy >> sb) - b.cy0;
            const int rb = int(fy & (F - 1));
            const unsigned long long rmask = row_bits << (rb * F);
            bool any_m = false, any_b = false;
            for (long long c = 0; c < wc; ++c) {
                const unsigned long long k = ccoff[q] + crow * wc + c;
                if (cst[k] == 2) {
                    any_m = true;
                    const unsigned long long bm = fbnd[k] & rmask;
                    any_b |= bm != 0;
                    n_b += __popcll(bm);
                }
            }
            const uint64_t ri = froff[q] + r;
            const uint32_t len = (any_m && any_b) ? rcnt[ri] : 0u;
            rlen[ri] = len;
            rsz[ri] = len;
            rpoly[ri] = q;
            if (!any_m)
                continue;
            // parity of the toggles at columns >= each column, in place, from the right
            uint32_t *row = fflip + fwoff[q] + r * ww;
            uint32_t carry = 0;
            for (long long w = ww - 1; w >= 0; --w) {
                const uint32_t y = suffix_xor(row[w]) ^ (carry ? 0xFFFFFFFFu : 0u);
                carry = y & 1u;
                row[w] = y;
            }
            for (long long c = 0; c < wc; ++c) {
                const unsigned long long k = ccoff[q] + crow * wc + c;
                if (cst[k] != 2)
                    continue;
                const long long ccx = b.cx0 + c;
                unsigned long long m = 0;
                for (long long fx = max(ccx << sb, (long long)b.fx0), fe = min((ccx << sb) + F - 1, (long long)b.fx1);
                     fx <= fe; ++fx) {
                    const int bit = rb * F + int(fx & (F - 1));
                    const long long col = fx - b.fx0;
                    if (!((fbnd[k] >> bit) & 1ull) && ((row[col >> 5] >> (col & 31)) & 1u))
                        m |= 1ull << bit;
                }
                if (m)
                    atomicOr(finside + k, m);
            }
        }
    }
    atomicAdd(counters + 2, n_b);
}

// 4a. the edges of every listed fine row, as sort keys (right end descending,
// then ring order): a thread per edge
__global__ void __launch_bounds__(kT) k_ib_lists(const int2 *v, const uint64_t *off, uint32_t P, uint64_t V, int g,
                                                 int sb, const PBox *box, const unsigned long long *froff,
                                                 const uint32_t *rlen, const unsigned long long *rowoff,
                                                 uint32_t *rcur, unsigned long long *keys)
{
    const int sf = kBoxLog2 - g - sb;
    const long long Sf = 1ll << sf;
    for (uint64_t i = blockIdx.x * (uint64_t)kT + threadIdx.x; i < V; i += (uint64_t)gridDim.x * kT) {
        const uint32_t q = owner(off, P, i);
        const PBox b = box[q];
        if (b.cx1 < b.cx0)
            continue;
        const uint64_t j = (i + 1 == off[q + 1]) ? off[q] : i + 1;
        const int2 pa = v[i], pb = v[j];
        if (pa.y == pb.y)
            continue;
        const long long lo_y = min(pa.y, pb.y), hi_y = max(pa.y, pb.y);
        const unsigned long long key =
            ((unsigned long long)(0x7FFFFFFF - max(pa.x, pb.x)) << 32) | (unsigned long long)(i - off[q]);
        for (long long fr = max(lo_y >> sf, (long long)b.fy0), r1 = min(cdiv(hi_y, Sf) - 1, (long long)b.fy1);
             fr <= r1; ++fr) {
            const uint64_t ri = froff[q] + (fr - b.fy0);
            if (rlen[ri])
                keys[rowoff[ri] + atomicAdd(rcur + ri, 1u)] = key;
        }
    }
}

// 4b. each listed row sorted, its edges written: a thread per row
__global__ void __launch_bounds__(kT) k_ib_rows(uint64_t NR, const int2 *v, const uint64_t *off,
                                                const uint32_t *rlen, const uint32_t *rpoly,
                                                const unsigned long long *rowoff, unsigned long long *keys,
                                                int4 *edge)
{
    for (uint64_t ri = blockIdx.x * (uint64_t)kT + threadIdx.x; ri < NR; ri += (uint64_t)gridDim.x * kT) {
        const uint32_t n = rlen[ri];
        if (!n)
            continue;
        unsigned long long *k = keys + rowoff[ri];
        if (n <= 32) {
            for (uint32_t a = 1; a < n; ++a) {
                const unsigned long long x = k[a];
                uint32_t c = a;
                for (; c > 0 && k[c - 1] > x; --c)
                    k[c] = k[c - 1];
                k[c] = x;
            }
        } else { // heap sort
            auto sift = [&](uint32_t root, uint32_t end) {
                while (2 * root + 1 < end) {
                    uint32_t ch = 2 * root + 1;
                    if (ch + 1 < end && k[ch + 1] > k[ch])
                        ++ch;
                    if (k[root] >= k[ch])
                        return;
                    const unsigned long long t = k[root];
                    k[root] = k[ch];
                    k[ch] = t;
                    root = ch;
                }
            };
            for (uint32_t s = n / 2; s-- > 0;)
                sift(s, n);
            for (uint32_t e = n - 1; e > 0; --e) {
                const unsigned long long t = k[0];
                k[0] = k[e];
                k[e] = t;
                sift(0, e);
            }
        }
        const uint32_t q = rpoly[ri];
        const uint64_t a0 = off[q], nv = off[q + 1] - a0;
        for (uint32_t m = 0; m < n; ++m) {
            const uint64_t i = k[m] & 0xFFFFFFFFull, j = (i + 1 == nv) ? 0 : i + 1;
            const int2 pa = v[a0 + i], pb = v[a0 + j];
            edge[rowoff[ri] + m] = make_int4(pa.x, pa.y, pb.x, pb.y);
        }
    }
}

// 5a. records (polygon | mixed << 31, box cell) to their grid cell
__global__ void __launch_bounds__(kT) k_ib_scatter(uint32_t P, int g, const PBox *box,
                                                   const unsigned long long *ccoff, const uint8_t *cst,
                                                   const unsigned long long *cell_off, uint32_t *ccur, uint2 *rec)
{
    for (uint32_t q = blockIdx.x; q < P; q += gridDim.x) {
        const PBox b = box[q];
        if (b.cx1 < b.cx0)
            continue;
        const unsigned long long wc = b.cx1 - b.cx0 + 1, n = wc * (unsigned long long)(b.cy1 - b.cy0 + 1);
        for (unsigned long long t = threadIdx.x; t < n; t += kT) {
            const unsigned long long k = ccoff[q] + t;
            const uint8_t st = cst[k];
            if (!st)
                continue;
            const uint64_t cell = (uint64_t(b.cy0 + t / wc) << g) | uint64_t(b.cx0 + t % wc);
            rec[cell_off[cell] + atomicAdd(ccur + cell, 1u)] = make_uint2(q | (st == 2 ? 0x80000000u : 0u), uint32_t(k));
        }
    }
}

// 5b. every cell's records in polygon order (insertion sort: lists are short)
__global__ void __launch_bounds__(kT) k_ib_sortcells(uint64_t ncell, const unsigned long long *cell_off, uint2 *rec)
{
    for (uint64_t c = blockIdx.x * (uint64_t)kT + threadIdx.x; c < ncell; c += (uint64_t)gridDim.x * kT) {
        uint2 *l = rec + cell_off[c];
        const uint32_t n = uint32_t(cell_off[c + 1] - cell_off[c]);
        for (uint32_t a = 1; a < n; ++a) {
            const uint2 x = l[a];
            uint32_t b = a;
            for (; b > 0 && (l[b - 1].x & 0x7FFFFFFFu) > (x.x & 0x7FFFFFFFu); --b)
                l[b] = l[b - 1];
            l[b] = x;
        }
    }
}

// the entry list of fine cell f of a cell with records l[0 .. n): calls
// e(poly, boundary) per entry, in polygon order
template <class E>
__device__ __forceinline__ void fine_entries(const uint2 *l, uint32_t n, int f, const unsigned long long *fbnd,
                                             const unsigned long long *finside, E e)
{
    for (uint32_t m = 0; m < n; ++m) {
        const uint32_t q = l[m].x & 0x7FFFFFFFu;
        if (!(l[m].x & 0x80000000u)) {
            e(q, false);
        } else if ((fbnd[l[m].y] >> f) & 1ull) {
            e(q, true);
        } else if ((finside[l[m].y] >> f) & 1ull) {
            e(q, false);
        }
    }
}

// 5c. per cell: a fine block or not, and its entries
__global__ void __launch_bounds__(kT) k_ib_count(uint64_t ncell, int sb, const unsigned long long *cell_off,
                                                 const uint2 *rec, const unsigned long long *fbnd,
                                                 const unsigned long long *finside, unsigned long long *blk,
                                                 unsigned long long *entc)
{
    const int FF = 1 << (2 * sb);
    for (uint64_t c = blockIdx.x * (uint64_t)kT + threadIdx.x; c < ncell; c += (uint64_t)gridDim.x * kT) {
        const uint2 *l = rec + cell_off[c];
        const uint32_t n = uint32_t(cell_off[c + 1] - cell_off[c]);
        if (n == 0 || (n == 1 && !(l[0].x & 0x80000000u))) {
            blk[c] = 0;
            entc[c] = 0;
            continue;
        }
        unsigned long long ne = 0;
        for (int f = 0; f < FF; ++f) {
            uint32_t k = 0;
            bool bnd = false;
            fine_entries(l, n, f, fbnd, finside, [&](uint32_t, bool b) {
                ++k;
                bnd |= b;
            });
            if (k > 1 || (k == 1 && bnd)) // not empty and not one INSIDE polygon
                ne += k;
        }
        blk[c] = 1;
        entc[c] = ne;
    }
}

// 5d. coarse words, fine blocks, entries
__global__ void __launch_bounds__(kT) k_ib_write(uint64_t ncell, int g, int sb, const PBox *box,
                                                 const unsigned long long *froff, const unsigned long long *cell_off,
                                                 const uint2 *rec, const unsigned long long *fbnd,
                                                 const unsigned long long *finside, const unsigned long long *rowoff,
                                                 const uint32_t *rlen, const int4 *edge,
                                                 const unsigned long long *blk_of, const unsigned long long *ent_of,
                                                 uint32_t *cell_w, uint32_t *fine_w, uint4 *ent, uint32_t *err)
{
    const int F = 1 << sb, FF = F * F, sf = kBoxLog2 - g - sb;
    for (uint64_t c = blockIdx.x * (uint64_t)kT + threadIdx.x; c < ncell; c += (uint64_t)gridDim.x * kT) {
        const uint2 *l = rec + cell_off[c];
        const uint32_t n = uint32_t(cell_off[c + 1] - cell_off[c]);
        if (n == 0) {
            cell_w[c] = 0u;
            continue;
        }
        if (n == 1 && !(l[0].x & 0x80000000u)) {
            cell_w[c] = (kCellInsideOne << 30) | l[0].x;
            continue;
        }
        const uint64_t b = blk_of[c];
        cell_w[c] = (kCellSub << 30) | uint32_t(b);
        uint64_t e0 = ent_of[c];
        const long long cx = (long long)(c & ((1ull << g) - 1)), cy = (long long)(c >> g);
        for (int f = 0; f < FF; ++f) {
            uint32_t k = 0, one = 0;
            bool bnd = false;
            fine_entries(l, n, f, fbnd, finside, [&](uint32_t q, bool bd) {
                ++k;
                bnd |= bd;
                one = q;
            });
            uint32_t w = 0;
            if (k == 1 && !bnd) {
                w = (kCellInsideOne << 30) | one;
            } else if (k > 0) {
                const long long fy = (cy << sb) + f / F, fx = (cx << sb) + f % F, x0 = fx << sf;
                uint32_t m = 0;
                fine_entries(l, n, f, fbnd, finside, [&](uint32_t q, bool bd) {
                    uint32_t eb = 0, ec = 0;
                    if (bd) {
                        const uint64_t ri = froff[q] + (fy - box[q].fy0);
                        eb = uint32_t(rowoff[ri]);
                        // the prefix of the row's list with max x > x0 (sorted by max x descending)
                        uint32_t lo = 0, hi = rlen[ri];
                        while (lo < hi) {
                            const uint32_t mid = (lo + hi) >> 1;
                            const int4 ev = edge[rowoff[ri] + mid];
                            if ((long long)max(ev.x, ev.z) > x0)
                                lo = mid + 1;
                            else
                                hi = mid;
                        }
                        if (lo > 0xFFFFu)
                            atomicOr(err, 1u);
                        ec = lo;
                    }
                    ent[e0 + m] = make_uint4(q, eb, ec, (bd ? kEntBoundary : 0u) | (m + 1 == k ? kEntLast : 0u));
                    ++m;
                });
                w = (kCellList << 30) | uint32_t(e0);
                e0 += k;
            }
            fine_w[b * FF + f] = w;
        }
    }
}

// cover bitmap: a bit per block of cells that holds a non-empty cell
__global__ void __launch_bounds__(kT) k_ib_cover(uint64_t ncell, int g, int cg, const uint32_t *cell_w, uint32_t *cover)
{
    for (uint64_t c = blockIdx.x * (uint64_t)kT + threadIdx.x; c < ncell; c += (uint64_t)gridDim.x * kT) {
        if (!cell_w[c])
            continue;
        const uint32_t cx = uint32_t(c & ((1ull << g) - 1)), cy = uint32_t(c >> g);
        const uint32_t b = ((cy >> (g - cg)) << cg) | (cx >> (g - cg));
        atomicOr(cover + (b >> 5), 1u << (b & 31));
    }
}

// block summary: a 16-bit word per block of 2^(g - sg) x 2^(g - sg) cells
__global__ void __launch_bounds__(kT) k_ib_summary(int g, int sg, const uint32_t *cell_w, uint16_t *sum,
                                                   unsigned long long *resolved)
{
    const uint32_t nb = 1u << sg, sh = uint32_t(g - sg);
    unsigned long long r = 0;
    for (uint32_t t = blockIdx.x * kT + threadIdx.x; t < nb * nb; t += gridDim.x * kT) {
        const uint32_t by = t / nb, bx = t % nb;
        const uint32_t w0 = cell_w[(uint64_t(by << sh) << g) | (bx << sh)];
        bool same = (w0 >> 30) == kCellEmpty || ((w0 >> 30) == kCellInsideOne && (w0 & kPayloadMask) < kSumEmpty);
        for (uint32_t cy = by << sh; same && cy < ((by + 1) << sh); ++cy)
            for (uint32_t cx = bx << sh; same && cx < ((bx + 1) << sh); ++cx)
                same = cell_w[(uint64_t(cy) << g) | cx] == w0;
        sum[t] = !same ? uint16_t(kSumMixed) : (w0 >> 30) == kCellEmpty ? uint16_t(kSumEmpty)
                                                                      : uint16_t(w0 & kPayloadMask);
        r += same ? 1 : 0;
    }
    if (r)
        atomicAdd(resolved, r);
}

__global__ void k_ib_sentinels(uint4 *ent, uint64_t n_ent, int4 *edge, uint64_t n_edge, uint32_t *fine, int fine_pad)
{
    if (threadIdx.x < 4)
        ent[n_ent + threadIdx.x] = make_uint4(0u, 0u, 0u, kEntLast);
    if (threadIdx.x == 0) {
        edge[n_edge] = make_int4(0, 0, 0, 0);
        if (fine_pad)
            fine[0] = 0u;
    }
}

} // namespace

int build_grid_index_device(const int32_t *xy, const uint64_t *ring_off, uint32_t P, int g, int sb,
                            GridIndexDev &out, const char *&err, cudaError_t &cerr, cudaStream_t s,
                            cudaMemPool_t pool)
{
    out = GridIndexDev{};
    err = nullptr;
    cerr = cudaSuccess;
    const uint64_t V = P ? ring_off[P] : 0;
    const uint64_t ncell = uint64_t(1) << (2 * g);
    const int F = 1 << sb, FF = F * F;
    std::vector<void *> owned;
    // with a stream: stream-ordered memory (from `pool` when given), copies
    // and kernels on that stream, and the host waits on that stream alone
    auto dmalloc = [&](void **p, size_t bytes) {
        return !s ? cudaMalloc(p, bytes) : pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
    };
    auto dfree = [&](void *p) { return s ? cudaFreeAsync(p, s) : cudaFree(p); };
    auto copy = [&](void *dst, const void *src, size_t n, cudaMemcpyKind kind) {
        if (!s)
            return cudaMemcpy(dst, src, n, kind);
        const cudaError_t x = cudaMemcpyAsync(dst, src, n, kind, s);
        return x != cudaSuccess || kind != cudaMemcpyDeviceToHost ? x : cudaStreamSynchronize(s);
    };
    auto dset = [&](void *p, int v, size_t n) { return s ? cudaMemsetAsync(p, v, n, s) : cudaMemset(p, v, n); };
    auto finish = [&](int status, cudaError_t e) {
        cerr = e;
        for (void *p : owned)
            dfree(p);
        if (status && out.mem) {
            dfree(out.mem);
            out.mem = nullptr;
        }
        return status;
    };
    auto alloc = [&](void **p, size_t bytes) {
        *p = nullptr;
        const cudaError_t e = dmalloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess)
            owned.push_back(*p);
        return e;
    };
    cudaError_t e;
    auto ok = [&](cudaError_t x) { return (e = x) == cudaSuccess; };
    const uint64_t np = uint64_t(P) + 1;
    int2 *v = nullptr;
    uint64_t *off = nullptr;
    PBox *box = nullptr;
    unsigned long long *ncc = nullptr, *nfr = nullptr, *nfw = nullptr, *tot = nullptr, *part = nullptr;
    uint64_t part_cap = 0; // words of `part`, the scans' partial sums
    if (!ok(alloc((void **)&v, V * sizeof(int2))) || !ok(alloc((void **)&off, np * 8)) ||
        !ok(alloc((void **)&box, np * sizeof(PBox))) || !ok(alloc((void **)&ncc, np * 8)) ||
        !ok(alloc((void **)&nfr, np * 8)) || !ok(alloc((void **)&nfw, np * 8)) || !ok(alloc((void **)&tot, 16 * 8)))
        return finish(2, e);
    if (!ok(copy(v, xy, V * sizeof(int2), cudaMemcpyHostToDevice)) ||
        !ok(copy(off, ring_off, np * 8, cudaMemcpyHostToDevice)) || !ok(dset(tot, 0, 16 * 8)) ||
        !ok(dset(ncc, 0, np * 8)) || !ok(dset(nfr, 0, np * 8)) || !ok(dset(nfw, 0, np * 8)))
        return finish(2, e);
    const int sms = device_sm_count();
    auto grid = [&](uint64_t items) {
        const uint64_t b = (items + kT - 1) / kT;
        return unsigned(std::max<uint64_t>(1, std::min<uint64_t>(b, uint64_t(sms) * 16)));
    };
    const unsigned pblocks = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(P, uint64_t(sms) * 16)));
    // 1. boxes and their sizes; exclusive scans give each polygon its offsets
    if (P)
        k_ib_box<<<grid(uint64_t(P) * 32), kT, 0, s>>>(v, off, P, g, sb, box, ncc, nfr, nfw);
    auto scan = [&](unsigned long long *a, uint64_t n, unsigned long long *total) -> cudaError_t {
        const uint64_t need = scan_part_words(n);
        if (need > part_cap) { // grown for a longer scan (the old one is freed at the end)
            part_cap = std::max<uint64_t>(need, scan_part_words(ncell + 1));
            if (!ok(alloc((void **)&part, part_cap * 8)))
                return e;
        }
        return launch_exclusive_scan(a, n, total, part, s);
    };
    unsigned long long h[16] = {};
    if (!ok(cudaGetLastError()) || !ok(scan(ncc, np, tot + 0)) || !ok(scan(nfr, np, tot + 1)) ||
        !ok(scan(nfw, np, tot + 2)) || !ok(copy(h, tot, 3 * 8, cudaMemcpyDeviceToHost)))
        return finish(2, e);
    const uint64_t NCC = h[0], NR = h[1], NW = h[2];
    if (NCC >= (uint64_t(1) << 32)) {
        err = "index too large (polygon boxes of more than 2^32 coarse cells)";
        return finish(1, cudaSuccess);
    }
    // box cells: mixed marks, corner toggles, status, fine BOUNDARY and INSIDE bits
    uint32_t *cmix = nullptr, *cflip = nullptr, *fflip = nullptr, *rcnt = nullptr, *rlen = nullptr, *rcur = nullptr,
             *rpoly = nullptr, *ccur = nullptr, *errw = nullptr;
    uint8_t *cst = nullptr;
    unsigned long long *fbnd = nullptr, *finside = nullptr, *rsz = nullptr, *cell_cnt = nullptr, *blk = nullptr,
                       *entc = nullptr, *keys = nullptr;
    if (!ok(alloc((void **)&cmix, NCC * 4)) || !ok(alloc((void **)&cflip, NCC * 4)) ||
        !ok(alloc((void **)&cst, NCC)) || !ok(alloc((void **)&fbnd, NCC * 8)) ||
        !ok(alloc((void **)&finside, NCC * 8)) || !ok(alloc((void **)&fflip, NW * 4)) ||
        !ok(alloc((void **)&rcnt, NR * 4)) || !ok(alloc((void **)&rlen, NR * 4)) || !ok(alloc((void **)&rcur, NR * 4)) ||
        !ok(alloc((void **)&rpoly, NR * 4)) || !ok(alloc((void **)&rsz, (NR + 1) * 8)) ||
        !ok(alloc((void **)&cell_cnt, (ncell + 1) * 8)) || !ok(alloc((void **)&ccur, ncell * 4)) ||
        !ok(alloc((void **)&errw, 4)))
        return finish(2, e);
    if (!ok(dset(cmix, 0, NCC * 4)) || !ok(dset(cflip, 0, NCC * 4)) || !ok(dset(cst, 0, NCC)) ||
        !ok(dset(fbnd, 0, NCC * 8)) || !ok(dset(finside, 0, NCC * 8)) ||
        !ok(dset(fflip, 0, NW * 4)) || !ok(dset(rcnt, 0, NR * 4)) || !ok(dset(rcur, 0, NR * 4)) ||
        !ok(dset(rsz, 0, (NR + 1) * 8)) || !ok(dset(cell_cnt, 0, (ncell + 1) * 8)) ||
        !ok(dset(ccur, 0, ncell * 4)) || !ok(dset(errw, 0, 4)))
        return finish(2, e);
    // 2. per edge; 3. per row
    if (V)
        k_ib_mark<<<grid(V), kT, 0, s>>>(v, off, P, V, g, sb, box, ncc, nfr, nfw, cmix, cflip, fbnd, fflip, rcnt);
    if (P) {
        k_ib_coarse<<<pblocks, kT, 0, s>>>(P, g, box, ncc, cmix, cflip, cst, cell_cnt, tot + 4);
        k_ib_fine<<<pblocks, kT, 0, s>>>(P, sb, box, ncc, nfr, nfw, cst, fbnd, fflip, rcnt, finside, rlen, rsz, rpoly,
                                   tot + 4);
    }
    // 4. row lists: offsets (polygon by polygon, row by row), sort keys, sorted edges
    if (!ok(cudaGetLastError()) || !ok(scan(rsz, NR + 1, tot + 3)) ||
        !ok(copy(h + 3, tot + 3, 4 * 8, cudaMemcpyDeviceToHost)))
        return finish(2, e);
    const uint64_t E = h[3];
    out.n_inside = h[4];
    out.n_mixed = h[5];
    out.n_boundary = h[6];
    if (E >= (uint64_t(1) << 32)) {
        err = "index too large (edge list limit 2^32)";
        return finish(1, cudaSuccess);
    }
    if (!ok(alloc((void **)&keys, E * 8)))
        return finish(2, e);
    // the index's own allocation: cells | fine | entries | edges | cover | summary (sizes known
    // once the blocks and entries are counted; the edges are sorted straight into place)
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    if (V)
        k_ib_lists<<<grid(V), kT, 0, s>>>(v, off, P, V, g, sb, box, nfr, rlen, rsz, rcur, keys);
    int4 *edge_tmp = nullptr;
    if (!ok(cudaGetLastError()) || !ok(alloc((void **)&edge_tmp, (E + 1) * sizeof(int4))))
        return finish(2, e);
    if (NR)
        k_ib_rows<<<grid(NR), kT, 0, s>>>(NR, v, off, rlen, rpoly, rsz, keys, edge_tmp);
    // 5. records by cell, sorted by polygon; blocks and entries per cell
    if (!ok(cudaGetLastError()) || !ok(scan(cell_cnt, ncell + 1, tot + 7)) ||
        !ok(copy(h + 7, tot + 7, 8, cudaMemcpyDeviceToHost)))
        return finish(2, e);
    const uint64_t R = h[7];
    uint2 *rec = nullptr;
    if (!ok(alloc((void **)&rec, R * sizeof(uint2))) || !ok(alloc((void **)&blk, (ncell + 1) * 8)) ||
        !ok(alloc((void **)&entc, (ncell + 1) * 8)))
        return finish(2, e);
    if (P)
        k_ib_scatter<<<pblocks, kT, 0, s>>>(P, g, box, ncc, cst, cell_cnt, ccur, rec);
    k_ib_sortcells<<<grid(ncell), kT, 0, s>>>(ncell, cell_cnt, rec);
    k_ib_count<<<grid(ncell), kT, 0, s>>>(ncell, sb, cell_cnt, rec, fbnd, finside, blk, entc);
    if (!ok(cudaGetLastError()) || !ok(dset(blk + ncell, 0, 8)) || !ok(dset(entc + ncell, 0, 8)) ||
        !ok(scan(blk, ncell + 1, tot + 8)) || !ok(scan(entc, ncell + 1, tot + 9)) ||
        !ok(copy(h + 8, tot + 8, 2 * 8, cudaMemcpyDeviceToHost)))
        return finish(2, e);
    const uint64_t NB = h[8], NE = h[9];
    if (NB * uint64_t(FF) >= (uint64_t(1) << 32) || (NB && NB - 1 >= (uint64_t(1) << 30))) {
        err = "index too large (fine block limit)";
        return finish(1, cudaSuccess);
    }
    if (NE >= (uint64_t(1) << 30)) {
        err = "index too large (entry limit 2^30)";
        return finish(1, cudaSuccess);
    }
    const int cg = std::min(g, kCoverLog2), sg = std::min(g, kSumLog2);
    const uint64_t n_fine = std::max<uint64_t>(NB * FF, 1);
    const size_t cover_words = std::max<size_t>((size_t(1) << (2 * cg)) / 32, 1);
    const size_t b_cell = ncell * 4, b_fine = n_fine * 4, b_ent = (NE + 4) * 16, b_edge = (E + 1) * 16,
                 b_cover = cover_words * 4, b_sum = std::max<size_t>((size_t(2) << (2 * sg)), 16);
    out.bytes = up(b_cell) + up(b_fine) + up(b_ent) + up(b_edge) + up(b_cover) + up(b_sum) + 256;
    if (!ok(dmalloc(&out.mem, out.bytes))) {
        out.mem = nullptr;
        return finish(2, e);
    }
    char *m = static_cast<char *>(out.mem);
    out.cell = reinterpret_cast<uint32_t *>(m);
    out.fine = reinterpret_cast<uint32_t *>(m + up(b_cell));
    out.ent = reinterpret_cast<uint32_t *>(m + up(b_cell) + up(b_fine));
    out.edge = reinterpret_cast<int4 *>(m + up(b_cell) + up(b_fine) + up(b_ent));
    out.cover = reinterpret_cast<uint32_t *>(m + up(b_cell) + up(b_fine) + up(b_ent) + up(b_edge));
    out.sum = reinterpret_cast<uint16_t *>(m + up(b_cell) + up(b_fine) + up(b_ent) + up(b_edge) + up(b_cover));
    if (!ok(dset(out.cover, 0, b_cover)) ||
        !ok(copy(out.edge, edge_tmp, E * sizeof(int4), cudaMemcpyDeviceToDevice)))
        return finish(2, e);
    k_ib_write<<<grid(ncell), kT, 0, s>>>(ncell, g, sb, box, nfr, cell_cnt, rec, fbnd, finside, rsz, rlen, out.edge, blk,
                                    entc, out.cell, out.fine, reinterpret_cast<uint4 *>(out.ent), errw);
    k_ib_sentinels<<<1, 32, 0, s>>>(reinterpret_cast<uint4 *>(out.ent), NE, out.edge, E, out.fine, NB == 0 ? 1 : 0);
    k_ib_cover<<<grid(ncell), kT, 0, s>>>(ncell, g, cg, out.cell, out.cover);
    k_ib_summary<<<grid(uint64_t(1) << (2 * sg)), kT, 0, s>>>(g, sg, out.cell, out.sum, tot + 10);
    uint32_t herr = 0;
    if (!ok(cudaGetLastError()) || !ok(s ? cudaStreamSynchronize(s) : cudaDeviceSynchronize()) ||
        !ok(copy(&herr, errw, 4, cudaMemcpyDeviceToHost)) ||
        !ok(copy(h + 10, tot + 10, 8, cudaMemcpyDeviceToHost)))
        return finish(2, e);
    if (herr) {
        err = "a fine row edge list exceeds 65535 edges; use a finer grid";
        return finish(1, cudaSuccess);
    }
    out.n_cell = ncell;
    out.n_fine = n_fine;
    out.n_ent = NE + 4;
    out.n_edge = E + 1;
    out.n_blocks = NB;
    out.sum_resolved = double(h[10]) / double(uint64_t(1) << (2 * sg));
    return finish(0, cudaSuccess);
}

} // namespace spx
