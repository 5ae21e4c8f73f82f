// Host build of the grid index of a set of disks (SPADE §4.2 "Canvases for
// Distance-Based Queries": a distance constraint around a point is a disk of
// radius r; §5.2 "Distance-Based Queries": a point is selected iff its
// distance to the centre is <= r).
//
// Grid of 2^g x 2^g cells of side S = 2^(30-g); a cell holds the integer
// points [x0, x0 + S - 1] x [y0, y0 + S - 1].  For every disk, every cell of
// its bounding box is classified exactly in int64:
//   - the cell's point nearest to the centre is farther than r: no entry;
//   - the cell's farthest corner is within r: INSIDE (the disk is convex, so
//     every point of the cell is within r);
//   - otherwise BOUNDARY: the kernel tests each point.
// Cells keep their disks in disk order.  Cell word: 0 empty; kind 1 with the
// disk id when the cell is INSIDE exactly one disk and no other; kind 2 with
// the offset of its list (entries[off] = n, then n words disk << 1 | boundary).
#include "spx_internal.h"

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

namespace spx {

bool build_disk_index(const int32_t *cxy, const int32_t *r, uint32_t Q, int g, HostDiskIndex &out, std::string &err)
{
    if (g < 1 || g > kMaxGridLog2) {
        err = "grid_log2 must be in [1, 13]";
        return false;
    }
    const int sh = kBoxLog2 - g;
    const int64_t S = int64_t(1) << sh, last = (int64_t(1) << kBoxLog2) - 1;
    const uint64_t ncell = uint64_t(1) << (2 * g);
    // pass 1: (cell, disk, flag) records, disk by disk
    std::vector<uint64_t> recs; // cell << 32 | disk << 1 | boundary
    uint64_t n_inside = 0, n_boundary = 0;
    for (uint32_t q = 0; q < Q; ++q) {
        const int64_t cx = cxy[2 * q], cy = cxy[2 * q + 1], rr = int64_t(r[q]) * r[q];
        const int64_t xlo = std::max<int64_t>(0, cx - r[q]), xhi = std::min<int64_t>(last, cx + r[q]);
        const int64_t ylo = std::max<int64_t>(0, cy - r[q]), yhi = std::min<int64_t>(last, cy + r[q]);
        if (xlo > xhi || ylo > yhi)
            continue;
        for (int64_t j = ylo >> sh; j <= yhi >> sh; ++j)
            for (int64_t i = xlo >> sh; i <= xhi >> sh; ++i) {
                const int64_t x0 = i * S, x1 = x0 + S - 1, y0 = j * S, y1 = y0 + S - 1;
                const int64_t nx = std::min(std::max(cx, x0), x1) - cx, ny = std::min(std::max(cy, y0), y1) - cy;
                if (nx * nx + ny * ny > rr)
                    continue;
                const int64_t fx = std::max(cx - x0, x1 - cx), fy = std::max(cy - y0, y1 - cy);
                const bool inside = fx * fx + fy * fy <= rr;
                (inside ? n_inside : n_boundary)++;
                recs.push_back((uint64_t((j << g) | i) << 32) | (uint64_t(q) << 1) | (inside ? 0u : 1u));
            }
    }
    // pass 2: bucket by cell, keeping disk order (stable sort by cell)
    std::stable_sort(recs.begin(), recs.end(), [](uint64_t a, uint64_t b) { return (a >> 32) < (b >> 32); });
    out = HostDiskIndex{};
    out.grid_log2 = g;
    out.n_disks = Q;
    out.cell.assign(ncell, 0u);
    out.entries.push_back(0); // offset 0 is never a list
    for (size_t a = 0; a < recs.size();) {
        size_t b = a;
        while (b < recs.size() && (recs[b] >> 32) == (recs[a] >> 32))
            ++b;
        const uint64_t c = recs[a] >> 32;
        const uint32_t w0 = uint32_t(recs[a]);
        if (b - a == 1 && !(w0 & 1u)) {
            out.cell[c] = (kCellInsideOne << 30) | (w0 >> 1);
        } else {
            if (out.entries.size() + (b - a) + 1 > kPayloadMask) {
                err = "too many disk entries for one index; use a smaller grid";
                return false;
            }
            out.cell[c] = (kCellList << 30) | uint32_t(out.entries.size());
            out.entries.push_back(uint32_t(b - a));
            for (size_t k = a; k < b; ++k)
                out.entries.push_back(uint32_t(recs[k]));
        }
        a = b;
    }
    out.n_inside = n_inside;
    out.n_boundary = n_boundary;
    return true;
}

int default_disk_grid_log2(const int32_t *r, uint32_t Q)
{
    // about eight cells across the median diameter, clamped to [5, 12]
    if (!Q)
        return 5;
    std::vector<int32_t> v(r, r + Q);
    std::nth_element(v.begin(), v.begin() + Q / 2, v.end());
    const double d = 2.0 * std::max<int32_t>(v[Q / 2], 1);
    int g = 5;
    while (g < 12 && double(int64_t(1) << (kBoxLog2 - g)) > d / 8.0)
        ++g;
    return g;
}

} // namespace spx
