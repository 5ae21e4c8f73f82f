// Host build of the grid index (SPADE §4.2 canvas creation, §4.3 boundary
// index; the paper rasterises polygons into a texture, here they are
// rasterised into the cells of a 2^g x 2^g grid over the coordinate box).
//
// Per polygon:
//  1. Conservative rasterisation of the boundary (the paper's conservative
//     rasterisation of polygon edges): for every row strip an edge meets,
//     the edge's piece inside the closed strip is clipped with exact rational
//     arithmetic and every cell whose OPEN square it can meet is marked
//     BOUNDARY.
//  2. Every other cell of the polygon's bounding box holds points of one status
//     only: its perturbed points p + (eps, eps^2) all lie in the open square,
//     which no edge meets.  The status of the cell's lower-left corner is
//     decided for a whole row at once by a scanline: each edge straddling the
//     row's bottom line counts for exactly the cells whose corner x is left of
//     the edge's crossing, i.e. cx <= floor((a.x + ceil(num/den) - 1) / S).
//  3. For every row with a BOUNDARY cell, the edges meeting the row's open
//     strip are stored once, sorted by max x descending; a BOUNDARY entry
//     points at the prefix with max x > the cell's x0.
// Then the (cell, polygon) records of all polygons are bucketed by cell in
// polygon order, so every cell's list is sorted by polygon id.
#include "spx_internal.h"

#include <algorithm>
#include <cmath>
#include <thread>

namespace spx {
namespace {

inline int64_t floor_div(int64_t a, int64_t b) // b > 0
{
    int64_t q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}
inline int64_t ceil_div(int64_t a, int64_t b) // b > 0
{
    int64_t q = a / b;
    return (a % b != 0 && a > 0) ? q + 1 : q;
}

struct Rec {
    uint32_t cell, poly, flags, edge_begin, edge_cnt;
};

struct Part {
    std::vector<Rec> recs;
    std::vector<int32_t> edges; // 4 per edge
    uint64_t n_boundary = 0, n_inside = 0;
    bool overflow = false;
};

struct RowEdge {
    int64_t xmax;
    uint32_t idx;
};

void build_polygon(const int32_t *r, uint64_t nv, uint32_t q, int g, Part &out)
{
    if (nv < 3)
        return; // fewer than 3 vertices: no point is inside (the crossings cancel)
    const int shift = kBoxLog2 - g;
    const int64_t S = int64_t(1) << shift;
    const int64_t G = int64_t(1) << g;
    int64_t xmin = INT64_MAX, xmax = INT64_MIN, ymin = INT64_MAX, ymax = INT64_MIN;
    for (uint64_t k = 0; k < nv; ++k) {
        xmin = std::min<int64_t>(xmin, r[2 * k]);
        xmax = std::max<int64_t>(xmax, r[2 * k]);
        ymin = std::min<int64_t>(ymin, r[2 * k + 1]);
        ymax = std::max<int64_t>(ymax, r[2 * k + 1]);
    }
    if (xmax <= xmin || ymax <= ymin)
        return; // inside implies xmin <= px < xmax and ymin <= py < ymax: empty
    const int64_t cx0 = xmin >> shift, cx1 = std::min((xmax - 1) >> shift, G - 1);
    const int64_t cy0 = ymin >> shift, cy1 = std::min((ymax - 1) >> shift, G - 1);
    const int64_t W = cx1 - cx0 + 1, H = cy1 - cy0 + 1;
    std::vector<uint8_t> bnd(size_t(W * H), 0);
    std::vector<std::pair<uint32_t, uint32_t>> row_edge; // (row - cy0, edge index)

    auto mark = [&](int64_t row, int64_t clo, int64_t chi) {
        if (row < cy0 || row > cy1)
            return;
        clo = std::max(clo, cx0);
        chi = std::min(chi, cx1);
        uint8_t *b = &bnd[size_t((row - cy0) * W)];
        for (int64_t c = clo; c <= chi; ++c)
            b[c - cx0] = 1;
    };
    // x of the edge at height Y as floor and ceil (exact rational arithmetic)
    auto x_at = [](int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t Y, int64_t &fl, int64_t &ce) {
        int64_t num = (bx - ax) * (Y - ay), den = by - ay;
        if (den < 0) {
            num = -num;
            den = -den;
        }
        fl = ax + floor_div(num, den);
        ce = ax + ceil_div(num, den);
    };

    for (uint64_t i = 0; i < nv; ++i) {
        uint64_t j = (i + 1 == nv) ? 0 : i + 1;
        const int64_t ax = r[2 * i], ay = r[2 * i + 1], bx = r[2 * j], by = r[2 * j + 1];
        if (ay == by) {
            if (ay % S == 0)
                continue; // on a row border: meets no open cell square
            const int64_t lo = std::min(ax, bx), hi = std::max(ax, bx);
            mark(ay >> shift, floor_div(lo, S), ceil_div(hi, S) - 1);
            continue; // horizontal edges never straddle: not in any row list
        }
        const int64_t lo_y = std::min(ay, by), hi_y = std::max(ay, by);
        const int64_t r0 = std::max(lo_y >> shift, cy0);
        const int64_t r1 = std::min(ceil_div(hi_y, S) - 1, cy1);
        for (int64_t row = r0; row <= r1; ++row) {
            row_edge.emplace_back(uint32_t(row - cy0), uint32_t(i));
            const int64_t Ya = std::max(lo_y, row * S), Yb = std::min(hi_y, (row + 1) * S);
            int64_t fa, ca, fb, cb;
            x_at(ax, ay, bx, by, Ya, fa, ca);
            x_at(ax, ay, bx, by, Yb, fb, cb);
            const int64_t xlo = std::min(fa, fb), xhi = std::max(ca, cb);
            mark(row, floor_div(xlo, S), ceil_div(xhi, S) - 1);
        }
    }
    // bucket the row list by row (stable: edges keep ring order within a row)
    std::vector<uint32_t> row_off(size_t(H + 1), 0);
    for (auto &p : row_edge)
        row_off[p.first + 1]++;
    for (int64_t k = 0; k < H; ++k)
        row_off[k + 1] += row_off[k];
    std::vector<uint32_t> row_list(row_edge.size());
    {
        std::vector<uint32_t> cur(row_off.begin(), row_off.end() - 1);
        for (auto &p : row_edge)
            row_list[cur[p.first]++] = p.second;
    }

    std::vector<uint8_t> flip(size_t(W), 0);
    std::vector<RowEdge> sorted;
    for (int64_t row = cy0; row <= cy1; ++row) {
        const int64_t y0 = row * S;
        const uint32_t *le = row_list.data() + row_off[row - cy0];
        const uint32_t ne = row_off[row - cy0 + 1] - row_off[row - cy0];
        // scanline status of the cell corners (x0, y0) of this row
        std::fill(flip.begin(), flip.end(), 0);
        uint8_t all = 0; // parity of edges that count for every cell of the row
        for (uint32_t k = 0; k < ne; ++k) {
            uint64_t i = le[k], j = (i + 1 == nv) ? 0 : i + 1;
            const int64_t ax = r[2 * i], ay = r[2 * i + 1], bx = r[2 * j], by = r[2 * j + 1];
            if ((ay > y0) == (by > y0))
                continue;
            int64_t num = (bx - ax) * (y0 - ay), den = by - ay;
            if (den < 0) {
                num = -num;
                den = -den;
            }
            // corner x counts iff x < a.x + num/den  <=>  x <= a.x + ceil(num/den) - 1
            const int64_t kx = floor_div(ax + ceil_div(num, den) - 1, S);
            if (kx >= cx1)
                all ^= 1;
            else if (kx >= cx0)
                flip[size_t(kx - cx0)] ^= 1;
        }
        const uint8_t *b = &bnd[size_t((row - cy0) * W)];
        bool any_b = false;
        for (int64_t c = 0; c < W; ++c)
            any_b |= b[c] != 0;
        uint32_t list_begin = 0;
        if (any_b) {
            sorted.clear();
            for (uint32_t k = 0; k < ne; ++k) {
                uint64_t i = le[k], j = (i + 1 == nv) ? 0 : i + 1;
                sorted.push_back({std::max<int64_t>(r[2 * i], r[2 * j]), le[k]});
            }
            std::stable_sort(sorted.begin(), sorted.end(),
                             [](const RowEdge &u, const RowEdge &v) { return u.xmax > v.xmax; });
            if (out.edges.size() / 4 + sorted.size() >= (uint64_t(1) << 32)) {
                out.overflow = true;
                return;
            }
            list_begin = uint32_t(out.edges.size() / 4);
            for (auto &e : sorted) {
                uint64_t i = e.idx, j = (i + 1 == nv) ? 0 : i + 1;
                out.edges.push_back(r[2 * i]);
                out.edges.push_back(r[2 * i + 1]);
                out.edges.push_back(r[2 * j]);
                out.edges.push_back(r[2 * j + 1]);
            }
        }
        uint8_t par = all;
        uint32_t n_right = 0; // edges of `sorted` with xmax > x0, tracked from the right
        for (int64_t c = W - 1; c >= 0; --c) {
            const int64_t cx = cx0 + c;
            if (c < W - 1)
                par ^= flip[size_t(c)];
            else
                par ^= flip[size_t(c)]; // kx == cx1 was folded into `all`; flip[W-1] is always 0
            const uint32_t cell = uint32_t((row << g) | cx);
            if (b[c]) {
                const int64_t x0 = cx * S;
                while (n_right < sorted.size() && sorted[n_right].xmax > x0)
                    ++n_right;
                out.recs.push_back({cell, q, kEntBoundary, list_begin, n_right});
                out.n_boundary++;
            } else if (par) {
                out.recs.push_back({cell, q, 0u, 0u, 0u});
                out.n_inside++;
            }
        }
    }
}

} // namespace

int default_grid_log2(const int32_t *xy, const uint64_t *ring_off, uint32_t P)
{
    if (P == 0)
        return 6;
    std::vector<double> side;
    side.reserve(P);
    for (uint32_t q = 0; q < P; ++q) {
        int64_t xmin = INT64_MAX, xmax = INT64_MIN, ymin = INT64_MAX, ymax = INT64_MIN;
        for (uint64_t k = ring_off[q]; k < ring_off[q + 1]; ++k) {
            xmin = std::min<int64_t>(xmin, xy[2 * k]);
            xmax = std::max<int64_t>(xmax, xy[2 * k]);
            ymin = std::min<int64_t>(ymin, xy[2 * k + 1]);
            ymax = std::max<int64_t>(ymax, xy[2 * k + 1]);
        }
        if (xmax > xmin && ymax > ymin)
            side.push_back(std::sqrt(double(xmax - xmin) * double(ymax - ymin)) / double(kBox));
    }
    if (side.empty())
        return 6;
    std::nth_element(side.begin(), side.begin() + side.size() / 2, side.end());
    const double med = side[side.size() / 2];
    // about 16 cells across a typical polygon
    int g = int(std::lround(std::log2(16.0 / std::max(med, 1e-9))));
    return std::min(std::max(g, 6), 12);
}

bool build_grid_index(const int32_t *xy, const uint64_t *ring_off, uint32_t P, int g, int threads, HostIndex &out,
                      std::string &err)
{
    if (g < 1 || g > kMaxGridLog2) {
        err = "grid_log2 out of range [1, 13]";
        return false;
    }
    if (P >= (1u << 30)) {
        err = "too many polygons (limit 2^30 - 1)";
        return false;
    }
    threads = std::max(1, std::min(threads, int(P ? P : 1)));
    std::vector<Part> parts(static_cast<size_t>(threads));
    // polygons are split by vertex count so the threads get similar work
    std::vector<uint32_t> split(static_cast<size_t>(threads + 1), P);
    split[0] = 0;
    {
        const uint64_t V = ring_off[P];
        int t = 1;
        for (uint32_t q = 0; q < P && t < threads; ++q)
            if (ring_off[q] >= V * uint64_t(t) / uint64_t(threads))
                split[size_t(t++)] = q;
        for (; t < threads; ++t)
            split[size_t(t)] = P;
    }
    auto work = [&](int t) {
        for (uint32_t q = split[size_t(t)]; q < split[size_t(t + 1)] && !parts[size_t(t)].overflow; ++q)
            build_polygon(xy + 2 * ring_off[q], ring_off[q + 1] - ring_off[q], q, g, parts[size_t(t)]);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t)
        pool.emplace_back(work, t);
    work(0);
    for (auto &th : pool)
        th.join();

    out = HostIndex();
    out.grid_log2 = g;
    out.n_polys = P;
    const uint64_t n_cells = uint64_t(1) << (2 * g);
    uint64_t n_recs = 0, n_edges = 0;
    for (auto &p : parts) {
        if (p.overflow) {
            err = "index too large (edge list limit 2^32)";
            return false;
        }
        n_recs += p.recs.size();
        n_edges += p.edges.size() / 4;
        out.n_boundary += p.n_boundary;
        out.n_inside += p.n_inside;
    }
    if (n_edges >= (uint64_t(1) << 32)) {
        err = "index too large (edge list limit 2^32)";
        return false;
    }
    // bucket records by cell; parts and records within a part are in polygon order
    std::vector<uint32_t> cnt(size_t(n_cells) + 1, 0);
    for (auto &p : parts)
        for (auto &rc : p.recs)
            cnt[rc.cell + 1]++;
    out.cell.assign(size_t(n_cells), 0);
    uint64_t n_entries = 0;
    std::vector<uint32_t> ent_off(size_t(n_cells), 0);
    for (uint64_t c = 0; c < n_cells; ++c) {
        ent_off[c] = uint32_t(n_entries);
        const uint32_t k = cnt[c + 1];
        if (k >= 2 || k == 1) {
            // a single INSIDE polygon is stored in the cell word itself (decided below)
            n_entries += k;
        }
        if (n_entries >= (uint64_t(1) << 30)) {
            err = "index too large (entry limit 2^30)";
            return false;
        }
    }
    out.entries.assign(size_t(n_entries) * 4, 0);
    out.edges.resize(size_t(n_edges) * 4);
    std::vector<uint32_t> fill(ent_off);
    uint64_t edge_base = 0;
    for (auto &p : parts) {
        for (auto &rc : p.recs) {
            uint32_t *e = &out.entries[size_t(fill[rc.cell]++) * 4];
            e[0] = rc.poly;
            e[1] = uint32_t(rc.edge_begin + edge_base);
            e[2] = rc.edge_cnt;
            e[3] = rc.flags;
        }
        std::copy(p.edges.begin(), p.edges.end(), out.edges.begin() + ptrdiff_t(edge_base * 4));
        edge_base += p.edges.size() / 4;
        std::vector<Rec>().swap(p.recs);
        std::vector<int32_t>().swap(p.edges);
    }
    // cell words; drop the entry of cells whose only polygon is INSIDE
    std::vector<uint32_t> keep(size_t(n_entries) * 4);
    uint64_t kept = 0;
    for (uint64_t c = 0; c < n_cells; ++c) {
        const uint32_t k = cnt[c + 1];
        if (k == 0)
            continue;
        const uint32_t *e = &out.entries[size_t(ent_off[c]) * 4];
        if (k == 1 && (e[3] & kEntBoundary) == 0) {
            out.cell[c] = (kCellInsideOne << 30) | e[0];
            continue;
        }
        out.cell[c] = (kCellList << 30) | uint32_t(kept);
        for (uint32_t m = 0; m < k; ++m) {
            uint32_t *d = &keep[size_t(kept + m) * 4];
            d[0] = e[4 * m];
            d[1] = e[4 * m + 1];
            d[2] = e[4 * m + 2];
            d[3] = e[4 * m + 3] | (m + 1 == k ? kEntLast : 0u);
        }
        kept += k;
    }
    keep.resize(size_t(kept) * 4);
    out.entries.swap(keep);
    return true;
}

} // namespace spx
