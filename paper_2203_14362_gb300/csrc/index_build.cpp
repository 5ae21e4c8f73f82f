// Host build of the two-level grid index (SPADE §4.2 canvas creation with
// conservative rasterisation of polygon boundaries, §4.3 boundary index; the
// paper rasterises polygons into a texture, here into the cells of a grid
// over the coordinate box, refined once where a cell is cut by a boundary).
//
// Per polygon, with coarse cells of side Sc = 2^(30-g) and fine cells of side
// Sf = Sc / F, F = 2^sub:
//  1. Conservative rasterisation of the boundary at both levels: for every row
//     strip an edge meets, the edge's piece inside the closed strip is clipped
//     with exact rational arithmetic and every cell whose OPEN square it can
//     meet is marked.  Coarse marks make a coarse cell "mixed"; fine marks make
//     a fine cell BOUNDARY.
//  2. A cell no edge meets holds points of one status only: its perturbed
//     points p + (eps, eps^2) all lie in its open square.  The status of the
//     lower-left corner (x0, y0) is decided for a whole row by a scanline: an
//     edge straddling y0 counts for exactly the corners left of its crossing,
//     x0 <= a.x + ceil(num/den) - 1 with num/den the crossing's offset from a.x.
//     Coarse rows classify coarse cells that are not mixed; fine rows classify
//     the fine cells of mixed coarse cells.
//  3. For every fine row with a BOUNDARY fine cell, the edges meeting the row's
//     open strip are stored once, sorted by max x descending; a BOUNDARY entry
//     points at the prefix with max x > the fine cell's x0.
// Then the records of all polygons are bucketed by coarse cell in polygon
// order, so every list is sorted by polygon id.
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

// (coarse cell, polygon): wholly inside, or mixed with its fine detail
struct Rec {
    uint32_t cell, poly, mixed, fine_idx;
};

// fine detail of one mixed (coarse cell, polygon)
struct FineRec {
    uint64_t inside = 0, bnd = 0;        // bit (fy mod F) * F + (fx mod F)
    uint32_t row_begin[1 << kMaxSubLog2] = {}; // first edge of each fine row's list
    uint16_t cnt[1 << (2 * kMaxSubLog2)] = {};  // edges listed for each BOUNDARY fine cell
};

struct Part {
    std::vector<Rec> recs;
    std::vector<FineRec> fine;
    std::vector<int32_t> edges; // 4 per edge
    uint64_t n_inside = 0, n_mixed = 0, n_boundary = 0;
    std::string err;
};

struct RowEdge {
    int64_t xmax;
    uint32_t idx;
};

// x of edge a->b at height Y, as floor and ceil (exact)
inline void x_at(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t Y, int64_t &fl, int64_t &ce)
{
    int64_t num = (bx - ax) * (Y - ay), den = by - ay;
    if (den < 0) {
        num = -num;
        den = -den;
    }
    fl = ax + floor_div(num, den);
    ce = ax + ceil_div(num, den);
}

// largest corner x (in cells of side S) that edge a->b counts for at height y0,
// where the edge straddles y0: x0 counts iff x0 < crossing
inline int64_t corner_threshold(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t y0, int64_t S)
{
    int64_t num = (bx - ax) * (y0 - ay), den = by - ay;
    if (den < 0) {
        num = -num;
        den = -den;
    }
    return floor_div(ax + ceil_div(num, den) - 1, S);
}

void build_polygon(const int32_t *r, uint64_t nv, uint32_t q, int gc, int sb, Part &out)
{
    if (nv < 3)
        return; // fewer than 3 vertices: no point is inside (the crossings cancel)
    const int gf = gc + sb, sc = kBoxLog2 - gc, sf = kBoxLog2 - gf, F = 1 << sb;
    const int64_t Sc = int64_t(1) << sc, Sf = int64_t(1) << sf;
    const int64_t Gc = int64_t(1) << gc, Gf = int64_t(1) << gf;
    int64_t xmin = INT64_MAX, xmax = INT64_MIN, ymin = INT64_MAX, ymax = INT64_MIN;
    for (uint64_t k = 0; k < nv; ++k) {
        xmin = std::min<int64_t>(xmin, r[2 * k]);
        xmax = std::max<int64_t>(xmax, r[2 * k]);
        ymin = std::min<int64_t>(ymin, r[2 * k + 1]);
        ymax = std::max<int64_t>(ymax, r[2 * k + 1]);
    }
    if (xmax <= xmin || ymax <= ymin)
        return; // inside implies xmin <= px < xmax and ymin <= py < ymax: empty
    const int64_t cx0 = xmin >> sc, cx1 = std::min((xmax - 1) >> sc, Gc - 1);
    const int64_t cy0 = ymin >> sc, cy1 = std::min((ymax - 1) >> sc, Gc - 1);
    const int64_t fx0 = xmin >> sf, fx1 = std::min((xmax - 1) >> sf, Gf - 1);
    const int64_t fy0 = ymin >> sf, fy1 = std::min((ymax - 1) >> sf, Gf - 1);
    const int64_t Wc = cx1 - cx0 + 1, Hc = cy1 - cy0 + 1, Hf = fy1 - fy0 + 1;
    std::vector<uint8_t> cb(size_t(Wc * Hc), 0);   // coarse cell is mixed
    std::vector<uint64_t> fm(size_t(Wc * Hc), 0);  // fine BOUNDARY bits per coarse cell
    std::vector<std::pair<uint32_t, uint32_t>> row_edge; // (fine row - fy0, edge index)

    auto mark_c = [&](int64_t row, int64_t lo, int64_t hi) {
        if (row < cy0 || row > cy1)
            return;
        lo = std::max(lo, cx0);
        hi = std::min(hi, cx1);
        uint8_t *b = &cb[size_t((row - cy0) * Wc)];
        for (int64_t c = lo; c <= hi; ++c)
            b[c - cx0] = 1;
    };
    auto mark_f = [&](int64_t frow, int64_t lo, int64_t hi) {
        if (frow < fy0 || frow > fy1)
            return;
        lo = std::max(lo, fx0);
        hi = std::min(hi, fx1);
        const int64_t crow = (frow >> sb) - cy0;
        const int bit0 = int(frow & (F - 1)) * F;
        for (int64_t fx = lo; fx <= hi; ++fx)
            fm[size_t(crow * Wc + ((fx >> sb) - cx0))] |= uint64_t(1) << (bit0 + int(fx & (F - 1)));
    };

    for (uint64_t i = 0; i < nv; ++i) {
        const uint64_t j = (i + 1 == nv) ? 0 : i + 1;
        const int64_t ax = r[2 * i], ay = r[2 * i + 1], bx = r[2 * j], by = r[2 * j + 1];
        if (ay == by) {
            // a horizontal edge meets the open squares of its row unless it lies on a row border
            const int64_t lo = std::min(ax, bx), hi = std::max(ax, bx);
            if (ay % Sc != 0)
                mark_c(ay >> sc, floor_div(lo, Sc), ceil_div(hi, Sc) - 1);
            if (ay % Sf != 0)
                mark_f(ay >> sf, floor_div(lo, Sf), ceil_div(hi, Sf) - 1);
            continue; // never straddles: in no row list
        }
        const int64_t lo_y = std::min(ay, by), hi_y = std::max(ay, by);
        for (int64_t row = std::max(lo_y >> sc, cy0), r1 = std::min(ceil_div(hi_y, Sc) - 1, cy1); row <= r1; ++row) {
            int64_t fa, ca, fb, cb2;
            x_at(ax, ay, bx, by, std::max(lo_y, row * Sc), fa, ca);
            x_at(ax, ay, bx, by, std::min(hi_y, (row + 1) * Sc), fb, cb2);
            mark_c(row, floor_div(std::min(fa, fb), Sc), ceil_div(std::max(ca, cb2), Sc) - 1);
        }
        for (int64_t fr = std::max(lo_y >> sf, fy0), r1 = std::min(ceil_div(hi_y, Sf) - 1, fy1); fr <= r1; ++fr) {
            row_edge.emplace_back(uint32_t(fr - fy0), uint32_t(i));
            int64_t fa, ca, fb, cb2;
            x_at(ax, ay, bx, by, std::max(lo_y, fr * Sf), fa, ca);
            x_at(ax, ay, bx, by, std::min(hi_y, (fr + 1) * Sf), fb, cb2);
            mark_f(fr, floor_div(std::min(fa, fb), Sf), ceil_div(std::max(ca, cb2), Sf) - 1);
        }
    }
    // fine row lists (bucketed, ring order kept within a row)
    std::vector<uint32_t> row_off(size_t(Hf + 1), 0);
    for (auto &p : row_edge)
        row_off[p.first + 1]++;
    for (int64_t k = 0; k < Hf; ++k)
        row_off[k + 1] += row_off[k];
    std::vector<uint32_t> row_list(row_edge.size());
    {
        std::vector<uint32_t> cur(row_off.begin(), row_off.end() - 1);
        for (auto &p : row_edge)
            row_list[cur[p.first]++] = p.second;
    }
    auto edge_of = [&](uint32_t i, int64_t &ax, int64_t &ay, int64_t &bx, int64_t &by) {
        const uint64_t j = (uint64_t(i) + 1 == nv) ? 0 : uint64_t(i) + 1;
        ax = r[2 * uint64_t(i)];
        ay = r[2 * uint64_t(i) + 1];
        bx = r[2 * j];
        by = r[2 * j + 1];
    };

    // one FineRec per mixed coarse cell
    std::vector<int64_t> fr_idx(size_t(Wc * Hc), -1);
    for (size_t k = 0; k < cb.size(); ++k)
        if (cb[k]) {
            fr_idx[k] = int64_t(out.fine.size());
            out.fine.emplace_back();
            out.fine.back().bnd = fm[k];
        }

    // coarse scanline: status of the corners of the coarse cells that are not mixed
    std::vector<uint8_t> flip(size_t(Wc), 0);
    for (int64_t cy = cy0; cy <= cy1; ++cy) {
        const int64_t y0 = cy * Sc;
        const int64_t fr = cy << sb; // the fine row whose strip starts at y0
        std::fill(flip.begin(), flip.end(), 0);
        uint8_t all = 0;
        if (fr >= fy0 && fr <= fy1) {
            for (uint32_t k = row_off[fr - fy0]; k < row_off[fr - fy0 + 1]; ++k) {
                int64_t ax, ay, bx, by;
                edge_of(row_list[k], ax, ay, bx, by);
                if ((ay > y0) == (by > y0))
                    continue;
                const int64_t kx = corner_threshold(ax, ay, bx, by, y0, Sc);
                if (kx >= cx1)
                    all ^= 1;
                else if (kx >= cx0)
                    flip[size_t(kx - cx0)] ^= 1;
            }
        } // else every vertex lies above y0: nothing straddles it
        uint8_t par = all;
        for (int64_t c = Wc - 1; c >= 0; --c) {
            par ^= flip[size_t(c)]; // parity of thresholds >= cx0 + c
            const size_t k = size_t((cy - cy0) * Wc + c);
            const uint32_t cell = uint32_t((cy << gc) | (cx0 + c));
            if (cb[k]) {
                out.recs.push_back({cell, q, 1u, uint32_t(fr_idx[k])});
                out.n_mixed++;
            } else if (par) {
                out.recs.push_back({cell, q, 0u, 0u});
                out.n_inside++;
            }
        }
    }

    // fine rows: classify the fine cells of mixed coarse cells, store edge lists
    std::vector<int64_t> thr;
    std::vector<RowEdge> sorted;
    const uint64_t row_bits = (F == 8) ? 0xFFull : ((uint64_t(1) << F) - 1);
    for (int64_t fy = fy0; fy <= fy1; ++fy) {
        const int64_t y0 = fy * Sf;
        const uint32_t *le = row_list.data() + row_off[fy - fy0];
        const uint32_t ne = row_off[fy - fy0 + 1] - row_off[fy - fy0];
        const int64_t crow = (fy >> sb) - cy0;
        const int rb = int(fy & (F - 1));
        const uint64_t rmask = row_bits << (rb * F);
        bool any_b = false, any_m = false;
        for (int64_t c = 0; c < Wc; ++c) {
            const size_t k = size_t(crow * Wc + c);
            if (cb[k]) {
                any_m = true;
                any_b |= (fm[k] & rmask) != 0;
            }
        }
        if (!any_m)
            continue;
        thr.clear();
        for (uint32_t k = 0; k < ne; ++k) {
            int64_t ax, ay, bx, by;
            edge_of(le[k], ax, ay, bx, by);
            if ((ay > y0) != (by > y0))
                thr.push_back(corner_threshold(ax, ay, bx, by, y0, Sf));
        }
        std::sort(thr.begin(), thr.end());
        uint32_t list_begin = 0;
        sorted.clear();
        if (any_b) {
            for (uint32_t k = 0; k < ne; ++k) {
                int64_t ax, ay, bx, by;
                edge_of(le[k], ax, ay, bx, by);
                sorted.push_back({std::max(ax, bx), le[k]});
            }
            std::stable_sort(sorted.begin(), sorted.end(),
                             [](const RowEdge &u, const RowEdge &v) { return u.xmax > v.xmax; });
            if (out.edges.size() / 4 + sorted.size() >= (uint64_t(1) << 32)) {
                out.err = "index too large (edge list limit 2^32)";
                return;
            }
            list_begin = uint32_t(out.edges.size() / 4);
            for (auto &e : sorted) {
                int64_t ax, ay, bx, by;
                edge_of(e.idx, ax, ay, bx, by);
                out.edges.push_back(int32_t(ax));
                out.edges.push_back(int32_t(ay));
                out.edges.push_back(int32_t(bx));
                out.edges.push_back(int32_t(by));
            }
        }
        for (int64_t c = 0; c < Wc; ++c) {
            const size_t k = size_t(crow * Wc + c);
            if (!cb[k])
                continue;
            FineRec &fr = out.fine[size_t(fr_idx[k])];
            fr.row_begin[rb] = list_begin;
            const int64_t ccx = cx0 + c;
            for (int64_t fx = std::max(ccx << sb, fx0), fe = std::min((ccx << sb) + F - 1, fx1); fx <= fe; ++fx) {
                const int bit = rb * F + int(fx & (F - 1));
                if ((fr.bnd >> bit) & 1) {
                    const int64_t x0 = fx * Sf;
                    // edges with max x > x0: a prefix of the descending list
                    const auto it = std::partition_point(sorted.begin(), sorted.end(),
                                                         [x0](const RowEdge &e) { return e.xmax > x0; });
                    const size_t n = size_t(it - sorted.begin());
                    if (n > 0xFFFF) {
                        out.err = "a fine row edge list exceeds 65535 edges; use a finer grid";
                        return;
                    }
                    fr.cnt[bit] = uint16_t(n);
                    out.n_boundary++;
                } else {
                    // corners right of fx count no threshold below fx
                    const size_t n_ge = size_t(thr.end() - std::lower_bound(thr.begin(), thr.end(), fx));
                    if (n_ge & 1)
                        fr.inside |= uint64_t(1) << bit;
                }
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
    // about 80 coarse cells across a typical polygon: then a point meets a
    // boundary-cut coarse cell rarely and a listed fine cell more rarely still
    // (the join's streaming pass reads most coarse words from the block
    // summary in shared memory, so a larger coarse level costs little, while
    // shorter fine-row edge lists shorten the exact tests)
    int g = int(std::lround(std::log2(80.0 / std::max(med, 1e-9))));
    return std::min(std::max(g, 5), kMaxGridLog2);
}

bool build_grid_index(const int32_t *xy, const uint64_t *ring_off, uint32_t P, int g, int sb, int threads,
                      HostIndex &out, std::string &err)
{
    if (g < 1 || g > kMaxGridLog2) {
        err = "grid_log2 out of range [1, 13]";
        return false;
    }
    if (sb < 0 || sb > kMaxSubLog2 || g + sb > kMaxFineLog2) {
        err = "sub_log2 out of range [0, 3] (and grid_log2 + sub_log2 <= 16)";
        return false;
    }
    if (P >= (1u << 30)) {
        err = "too many polygons (limit 2^30 - 1)";
        return false;
    }
    threads = std::max(1, std::min(threads, int(P ? P : 1)));
    std::vector<Part> parts(static_cast<size_t>(threads));
    // polygons split by vertex count, so the threads get similar work
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
        Part &pt = parts[size_t(t)];
        for (uint32_t q = split[size_t(t)]; q < split[size_t(t + 1)] && pt.err.empty(); ++q)
            build_polygon(xy + 2 * ring_off[q], ring_off[q + 1] - ring_off[q], q, g, sb, pt);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t)
        pool.emplace_back(work, t);
    work(0);
    for (auto &th : pool)
        th.join();

    out = HostIndex();
    out.grid_log2 = g;
    out.sub_log2 = sb;
    out.n_polys = P;
    const int F = 1 << sb, FF = F * F;
    const uint64_t n_cells = uint64_t(1) << (2 * g);
    // parts in order: global fine-record and edge offsets
    std::vector<uint64_t> fine_base(parts.size() + 1, 0), edge_base(parts.size() + 1, 0);
    for (size_t k = 0; k < parts.size(); ++k) {
        const Part &p = parts[k];
        if (!p.err.empty()) {
            err = p.err;
            return false;
        }
        fine_base[k + 1] = fine_base[k] + p.fine.size();
        edge_base[k + 1] = edge_base[k] + p.edges.size() / 4;
        out.n_inside += p.n_inside;
        out.n_mixed += p.n_mixed;
        out.n_boundary += p.n_boundary;
    }
    const uint64_t n_edges = edge_base.back(), n_fine = fine_base.back();
    if (n_edges >= (uint64_t(1) << 32)) {
        err = "index too large (edge list limit 2^32)";
        return false;
    }
    // every part, in parallel: its edges into place, its fine records' edge
    // offsets made global (records stay in their part; fine_ptr finds them)
    out.edges.resize(size_t(n_edges) * 4);
    std::vector<const FineRec *> fine_ptr(static_cast<size_t>(n_fine));
    {
        auto move_part = [&](size_t k) {
            Part &p = parts[k];
            for (size_t m = 0; m < p.fine.size(); ++m) {
                for (int r = 0; r < F; ++r)
                    p.fine[m].row_begin[r] += uint32_t(edge_base[k]);
                fine_ptr[size_t(fine_base[k] + m)] = &p.fine[m];
            }
            std::copy(p.edges.begin(), p.edges.end(), out.edges.begin() + ptrdiff_t(edge_base[k] * 4));
            std::vector<int32_t>().swap(p.edges);
        };
        std::vector<std::thread> pool;
        for (size_t k = 1; k < parts.size(); ++k)
            pool.emplace_back(move_part, k);
        move_part(0);
        for (auto &th : pool)
            th.join();
    }
    // records bucketed by coarse cell, parts in order (so polygon order within a cell)
    std::vector<uint32_t> cnt(size_t(n_cells) + 1, 0);
    for (size_t k = 0; k < parts.size(); ++k)
        for (auto &rc : parts[k].recs) {
            rc.fine_idx += uint32_t(fine_base[k]);
            cnt[rc.cell + 1]++;
        }
    for (uint64_t c = 0; c < n_cells; ++c)
        cnt[c + 1] += cnt[c];
    std::vector<Rec> recs(cnt[n_cells]);
    {
        std::vector<uint32_t> cur(cnt.begin(), cnt.end() - 1);
        for (auto &p : parts) {
            for (auto &rc : p.recs)
                recs[cur[rc.cell]++] = rc;
            std::vector<Rec>().swap(p.recs);
        }
    }
    // the entry list of fine cell f of the mixed coarse cell with records
    // [b0, b1): (poly, flags, edge_begin, edge_cnt) per entry
    auto fine_list = [&](uint32_t b0, uint32_t b1, int f, std::vector<uint32_t> &list) {
        list.clear();
        for (uint32_t m = b0; m < b1; ++m) {
            const Rec &rc = recs[m];
            if (!rc.mixed) {
                list.insert(list.end(), {rc.poly, 0u, 0u, 0u});
                continue;
            }
            const FineRec &fr = *fine_ptr[rc.fine_idx];
            if ((fr.bnd >> f) & 1)
                list.insert(list.end(), {rc.poly, kEntBoundary, fr.row_begin[f / F], uint32_t(fr.cnt[f])});
            else if ((fr.inside >> f) & 1)
                list.insert(list.end(), {rc.poly, 0u, 0u, 0u});
        }
    };
    auto is_one = [](const std::vector<uint32_t> &list) { return list.size() == 4 && list[1] == 0u; };
    // cells in parallel ranges, twice: first the fine blocks and entries each
    // cell needs, then (after a prefix sum, so the layout is the cell order)
    // the words themselves
    const int nt = threads;
    std::vector<uint64_t> c_lo(size_t(nt) + 1);
    for (int t = 0; t <= nt; ++t)
        c_lo[size_t(t)] = n_cells * uint64_t(t) / uint64_t(nt);
    std::vector<uint32_t> blk_of(size_t(n_cells) + 1, 0); // 1 per mixed cell, then exclusive prefix
    std::vector<uint64_t> ent_of(size_t(n_cells) + 1, 0); // entries per cell, then exclusive prefix
    auto count_cells = [&](int t) {
        std::vector<uint32_t> list;
        for (uint64_t c = c_lo[size_t(t)]; c < c_lo[size_t(t) + 1]; ++c) {
            const uint32_t b0 = cnt[c], b1 = cnt[c + 1];
            if (b0 == b1 || (b1 - b0 == 1 && !recs[b0].mixed))
                continue;
            blk_of[c] = 1;
            uint64_t n = 0;
            for (int f = 0; f < FF; ++f) {
                fine_list(b0, b1, f, list);
                if (!list.empty() && !is_one(list))
                    n += list.size() / 4;
            }
            ent_of[c] = n;
        }
    };
    {
        std::vector<std::thread> pool;
        for (int t = 1; t < nt; ++t)
            pool.emplace_back(count_cells, t);
        count_cells(0);
        for (auto &th : pool)
            th.join();
    }
    uint64_t n_blocks = 0, n_entries = 0;
    for (uint64_t c = 0; c <= n_cells; ++c) {
        const uint64_t b = blk_of[c], e = ent_of[c];
        blk_of[c] = uint32_t(std::min<uint64_t>(n_blocks, UINT32_MAX));
        ent_of[c] = n_entries;
        n_blocks += b;
        n_entries += e;
    }
    if (n_blocks * uint64_t(FF) >= (uint64_t(1) << 32) || (n_blocks && n_blocks - 1 >= (uint64_t(1) << 30))) {
        err = "index too large (fine block limit)";
        return false;
    }
    if (n_entries >= (uint64_t(1) << 30)) {
        err = "index too large (entry limit 2^30)";
        return false;
    }
    out.n_blocks = n_blocks;
    // every word of these is written below (empty cells included)
    out.cell.resize(size_t(n_cells));
    out.fine.resize(size_t(n_blocks * FF));
    out.entries.resize(size_t(n_entries) * 4);
    auto fill_cells = [&](int t) {
        std::vector<uint32_t> list;
        for (uint64_t c = c_lo[size_t(t)]; c < c_lo[size_t(t) + 1]; ++c) {
            const uint32_t b0 = cnt[c], b1 = cnt[c + 1];
            if (b0 == b1) {
                out.cell[c] = 0;
                continue;
            }
            if (b1 - b0 == 1 && !recs[b0].mixed) {
                out.cell[c] = (kCellInsideOne << 30) | recs[b0].poly;
                continue;
            }
            const uint64_t blk = blk_of[c];
            out.cell[c] = (kCellSub << 30) | uint32_t(blk);
            uint64_t e0 = ent_of[c];
            for (int f = 0; f < FF; ++f) {
                fine_list(b0, b1, f, list);
                uint32_t w = 0;
                if (is_one(list)) {
                    w = (kCellInsideOne << 30) | list[0];
                } else if (!list.empty()) {
                    const size_t n = list.size() / 4;
                    uint32_t *dst = out.entries.data() + e0 * 4;
                    for (size_t m = 0; m < n; ++m) {
                        // entry = (poly, edge_begin, edge_cnt, flags)
                        dst[4 * m] = list[4 * m];
                        dst[4 * m + 1] = list[4 * m + 2];
                        dst[4 * m + 2] = list[4 * m + 3];
                        dst[4 * m + 3] = list[4 * m + 1] | (m + 1 == n ? kEntLast : 0u);
                    }
                    w = (kCellList << 30) | uint32_t(e0);
                    e0 += n;
                }
                out.fine[size_t(blk * FF + uint64_t(f))] = w;
            }
        }
    };
    {
        std::vector<std::thread> pool;
        for (int t = 1; t < nt; ++t)
            pool.emplace_back(fill_cells, t);
        fill_cells(0);
        for (auto &th : pool)
            th.join();
    }
    // sentinels: the kernels read entries up to four at a time, and load fine word 0
    // and edge 0 in place of a missing one
    for (int k = 0; k < 4; ++k)
        out.entries.insert(out.entries.end(), {0u, 0u, 0u, kEntLast});
    if (out.fine.empty())
        out.fine.push_back(0u);
    out.edges.insert(out.edges.end(), {0, 0, 0, 0});
    return true;
}

bool validate_grid_index(const uint32_t *cell, uint64_t n_cell, const uint32_t *fine, uint64_t n_fine,
                         const uint32_t *ent, uint64_t n_ent, const int32_t *edges, uint64_t n_edge, int g, int sb,
                         uint32_t P, std::string &err)
{
    auto bad = [&](const std::string &m) {
        err = m;
        return false;
    };
    if (g < 1 || g > kMaxGridLog2 || sb < 1 || sb > kMaxSubLog2)
        return bad("grid_log2 / sub_log2 out of range");
    const uint64_t FF = uint64_t(1) << (2 * sb);
    if (n_cell != (uint64_t(1) << (2 * g)))
        return bad("coarse level is not 4^grid_log2 words");
    if (n_fine == 0 || (n_fine != 1 && n_fine % FF != 0))
        return bad("fine level is not a whole number of blocks");
    if (n_ent < 4)
        return bad("entry sentinels missing");
    for (uint64_t k = n_ent - 4; k < n_ent; ++k)
        if (ent[4 * k] != 0 || ent[4 * k + 1] != 0 || ent[4 * k + 2] != 0 || ent[4 * k + 3] != kEntLast)
            return bad("entry sentinels missing");
    if (n_edge < 1 || edges[4 * (n_edge - 1)] || edges[4 * (n_edge - 1) + 1] || edges[4 * (n_edge - 1) + 2] ||
        edges[4 * (n_edge - 1) + 3])
        return bad("edge sentinel missing");
    const uint64_t n_blocks = n_fine / FF, lists_end = n_ent - 4;
    // every entry list a fine word points at: inside the entries, ending with
    // its last entry before the sentinels, polygon ids below P, edge ranges
    // inside the edges (sentinel excluded)
    auto check_list = [&](uint64_t e0) {
        for (uint64_t k = e0;; ++k) {
            if (k >= lists_end)
                return bad("entry list " + std::to_string(e0) + " runs past the entries");
            const uint32_t q = ent[4 * k], eb = ent[4 * k + 1], ec = ent[4 * k + 2], fl = ent[4 * k + 3];
            if (q >= P)
                return bad("entry " + std::to_string(k) + " names polygon " + std::to_string(q));
            if (fl & ~(kEntBoundary | kEntLast))
                return bad("entry " + std::to_string(k) + " has unknown flags");
            if ((fl & kEntBoundary) && uint64_t(eb) + ec > n_edge - 1)
                return bad("entry " + std::to_string(k) + " lists edges past the edge array");
            if (fl & kEntLast)
                return true;
        }
    };
    for (uint64_t c = 0; c < n_cell; ++c) {
        const uint32_t kind = cell[c] >> 30, pay = cell[c] & kPayloadMask;
        if (kind == 3)
            return bad("coarse word " + std::to_string(c) + " of unknown kind");
        if (kind == kCellInsideOne && pay >= P)
            return bad("coarse word " + std::to_string(c) + " names polygon " + std::to_string(pay));
        if (kind == kCellSub && pay >= n_blocks)
            return bad("coarse word " + std::to_string(c) + " names fine block " + std::to_string(pay));
    }
    for (uint64_t f = 0; f < n_blocks * FF; ++f) {
        const uint32_t kind = fine[f] >> 30, pay = fine[f] & kPayloadMask;
        if (kind == 3)
            return bad("fine word " + std::to_string(f) + " of unknown kind");
        if (kind == kCellInsideOne && pay >= P)
            return bad("fine word " + std::to_string(f) + " names polygon " + std::to_string(pay));
        if (kind == kCellList && !check_list(pay))
            return false;
    }
    return true;
}

} // namespace spx
