// Host build of the edge grid of a set of buffered polygons (SPADE §4.2
// "Canvases for Distance-Based Queries": the distance constraint of radius r
// around a polygon is the polygon plus a rounded rectangle of radius r around
// every edge; §5.2 "Distance-Based Queries").
//
// Grid of 2^g x 2^g cells of side S = 2^(30-g); a cell holds the integer
// points [x0, x0 + S - 1] x [y0, y0 + S - 1].  Edge i of polygon q runs from
// vertex i to vertex i + 1 of its ring (the last back to the first; a ring of
// one vertex has one edge of length 0).  The edge is listed in every cell of
// its bounding box grown by r[q] whose centre lies within r[q] + h + 2 of the
// segment, h being the half-diagonal of the cell's points: a point of the cell
// within r[q] of the segment is within h of the centre, so no cell that holds
// such a point is left out (the margin of 2 covers the rounding of the
// distance in double precision, below 1e-6 at these magnitudes).  Each cell's
// list is sorted by (polygon, edge), so a point's candidate polygons come in
// ascending order, each polygon's edges together; a polygon whose r-region
// holds the whole cell keeps one item, flagged, instead of its edges.
#include "spx_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

namespace spx {

int default_buffer_grid_log2(const int32_t *xy, const uint64_t *ring_off, uint32_t P, const int32_t *r)
{
    // cells of about a quarter of the median radius: most cells near an edge
    // then lie wholly within r of it (one flagged item, no test); with no
    // radius, cells of about the median edge length
    std::vector<double> w, len;
    for (uint32_t q = 0; q < P; ++q) {
        w.push_back(r[q]);
        const uint64_t b = ring_off[q], n = ring_off[q + 1] - b;
        for (uint64_t i = 0; i < n; i += std::max<uint64_t>(1, n / 16)) {
            const uint64_t j = i + 1 == n ? 0 : i + 1;
            const double dx = double(xy[2 * (b + j)]) - xy[2 * (b + i)], dy = double(xy[2 * (b + j) + 1]) - xy[2 * (b + i) + 1];
            len.push_back(std::sqrt(dx * dx + dy * dy));
        }
    }
    if (w.empty())
        return 8;
    std::nth_element(w.begin(), w.begin() + w.size() / 2, w.end());
    double side = 0.25 * w[w.size() / 2];
    if (side < 1.0 && !len.empty()) {
        std::nth_element(len.begin(), len.begin() + len.size() / 2, len.end());
        side = len[len.size() / 2];
    }
    const int g = int(std::lround(std::log2(double(int64_t(1) << kBoxLog2) / std::max(side, 1.0))));
    return std::min(std::max(g, 5), 12);
}

// Is (px, py) within distance r of the closed segment (ax, ay)-(bx, by)?
// Exact: products of coordinate differences stay below 2^62 in int64; the
// distance to the segment's interior compares (d x w)^2 with r^2 |d|^2 in
// unsigned 128-bit arithmetic.
static bool near_segment(int64_t px, int64_t py, int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t r)
{
    const int64_t dx = bx - ax, dy = by - ay, wx = px - ax, wy = py - ay, rr = r * r;
    const int64_t t = wx * dx + wy * dy;
    if (t <= 0)
        return wx * wx + wy * wy <= rr;
    const int64_t dd = dx * dx + dy * dy;
    if (t >= dd)
        return (px - bx) * (px - bx) + (py - by) * (py - by) <= rr;
    const int64_t c = dx * wy - dy * wx;
    const unsigned __int128 ca = (unsigned __int128)(uint64_t)(c < 0 ? -c : c);
    return ca * ca <= (unsigned __int128)(uint64_t)rr * (unsigned __int128)(uint64_t)dd;
}

bool build_buffer_edges(const int32_t *xy, const uint64_t *ring_off, uint32_t P, const int32_t *r, int g,
                        HostBufferEdges &out, std::string &err)
{
    if (g < 1 || g > 12) {
        err = "edge grid_log2 must be in [1, 12]";
        return false;
    }
    const int sh = kBoxLog2 - g;
    const int64_t S = int64_t(1) << sh, ncs = int64_t(1) << g;
    const double h = (S - 1) * std::sqrt(0.5);
    struct Rec {
        uint32_t cell, q;
        uint64_t edge;
    };
    std::vector<Rec> recs;
    std::vector<int32_t> seg; // 4 per global edge
    for (uint32_t q = 0; q < P; ++q) {
        const uint64_t b = ring_off[q], n = ring_off[q + 1] - b;
        for (uint64_t i = 0; i < n; ++i) {
            const uint64_t j = i + 1 == n ? 0 : i + 1;
            const int64_t ax = xy[2 * (b + i)], ay = xy[2 * (b + i) + 1], bx = xy[2 * (b + j)], by = xy[2 * (b + j) + 1];
            const uint64_t e = seg.size() / 4;
            seg.insert(seg.end(), {int32_t(ax), int32_t(ay), int32_t(bx), int32_t(by)});
            const int64_t rq = r[q];
            auto cell_of = [&](int64_t v) { return std::min(std::max<int64_t>(v, 0), (int64_t(1) << kBoxLog2) - 1) >> sh; };
            const int64_t cx0 = cell_of(std::min(ax, bx) - rq), cx1 = cell_of(std::max(ax, bx) + rq);
            const int64_t cy0 = cell_of(std::min(ay, by) - rq), cy1 = cell_of(std::max(ay, by) + rq);
            const double dx = double(bx - ax), dy = double(by - ay), dd = dx * dx + dy * dy;
            for (int64_t cy = cy0; cy <= cy1; ++cy)
                for (int64_t cx = cx0; cx <= cx1; ++cx) {
                    const double px = double(cx * S) + 0.5 * (S - 1), py = double(cy * S) + 0.5 * (S - 1);
                    double t = dd > 0 ? ((px - ax) * dx + (py - ay) * dy) / dd : 0.0;
                    t = std::min(1.0, std::max(0.0, t));
                    const double ex = px - (ax + t * dx), ey = py - (ay + t * dy);
                    if (std::sqrt(ex * ex + ey * ey) <= double(rq) + h + 2.0)
                        recs.push_back({uint32_t(cy * ncs + cx), q, e});
                }
        }
    }
    if (recs.size() >= (uint64_t(1) << 32)) {
        err = "too many (cell, edge) entries for 32-bit offsets; use a coarser edge grid";
        return false;
    }
    std::sort(recs.begin(), recs.end(), [](const Rec &x, const Rec &y) {
        return x.cell != y.cell ? x.cell < y.cell : x.q != y.q ? x.q < y.q : x.edge < y.edge;
    });
    const uint64_t ncell = uint64_t(1) << (2 * g);
    out.g = g;
    out.cell_off.assign(ncell + 1, 0);
    out.item_q.clear();
    out.item_seg.clear();
    out.n_full = 0;
    // per (cell, polygon) group: when the four extreme points of the cell lie
    // within r of one of the group's edges, every point of the cell does (the
    // set of points within r of a segment is convex): the group becomes one
    // item flagged kBufferFull and the points of the cell need no test
    for (size_t k = 0; k < recs.size();) {
        size_t e = k;
        while (e < recs.size() && recs[e].cell == recs[k].cell && recs[e].q == recs[k].q)
            ++e;
        const uint32_t q = recs[k].q, cell = recs[k].cell;
        const int64_t x0 = int64_t(cell % ncs) * S, y0 = int64_t(cell / ncs) * S, x1 = x0 + S - 1, y1 = y0 + S - 1;
        bool full = false;
        for (size_t m = k; m < e && !full; ++m) {
            const int32_t *v = &seg[4 * recs[m].edge];
            full = near_segment(x0, y0, v[0], v[1], v[2], v[3], r[q]) && near_segment(x1, y0, v[0], v[1], v[2], v[3], r[q]) &&
                   near_segment(x0, y1, v[0], v[1], v[2], v[3], r[q]) && near_segment(x1, y1, v[0], v[1], v[2], v[3], r[q]);
        }
        out.cell_off[cell + 1] += full ? 1 : uint32_t(e - k);
        for (size_t m = k; m < (full ? k + 1 : e); ++m) {
            out.item_q.push_back(full ? (q | kBufferFull) : q);
            for (int c = 0; c < 4; ++c)
                out.item_seg.push_back(full ? 0 : seg[4 * recs[m].edge + c]);
        }
        out.n_full += full ? 1 : 0;
        k = e;
    }
    for (uint64_t c = 0; c < ncell; ++c)
        out.cell_off[c + 1] += out.cell_off[c];
    return true;
}

} // namespace spx
