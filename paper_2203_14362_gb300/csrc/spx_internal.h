// Internal layout of libspx: the grid index as the kernels read it, and the
// host-side build that produces it.  Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

namespace spx {

// An allocator whose value-less construct leaves trivial elements
// uninitialised: resize() of a large array then costs no zero fill, and its
// pages are first touched by the (parallel) code that writes every element.
template <class T>
struct DefaultInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = DefaultInitAlloc<U>;
    };
    DefaultInitAlloc() = default;
    template <class U>
    DefaultInitAlloc(const DefaultInitAlloc<U> &) noexcept {}
    template <class U>
    void construct(U *p) noexcept(std::is_nothrow_default_constructible<U>::value)
    {
        ::new (static_cast<void *>(p)) U;
    }
    template <class U, class... A>
    void construct(U *p, A &&...a)
    {
        ::new (static_cast<void *>(p)) U(std::forward<A>(a)...);
    }
};
template <class T>
using BigVec = std::vector<T, DefaultInitAlloc<T>>;

constexpr int kBoxLog2 = 30;            // points in [0, 2^30)^2, vertices in [0, 2^30]^2
constexpr uint32_t kBox = 1u << kBoxLog2;
constexpr int kMaxGridLog2 = 13;       // coarse grid: at most 2^13 cells per side
constexpr int kMaxSubLog2 = 3;         // a mixed coarse cell splits into at most 8 x 8 fine cells
constexpr int kMaxFineLog2 = 16;       // fine cells at least 2^14 units wide

// Two-level grid.  Coarse cell word (uint32, row-major, cell = (cy << g) | cx):
//   bits 31..30 = kind, bits 29..0 = payload
//   kind 0: no polygon can contain a point of this cell
//   kind 1: exactly one polygon, and the whole cell is INSIDE it: payload = polygon id
//   kind 2: mixed: payload = block b; the cell's F x F fine cells (F = 2^sub)
//           have words fine[b * F*F + (fy mod F) * F + (fx mod F)]
// Fine cell word: kind 0 none, kind 1 one INSIDE polygon (payload = id),
//   kind 2 list: payload = index of the fine cell's first entry in `entries`.
constexpr uint32_t kCellEmpty = 0u;
constexpr uint32_t kCellInsideOne = 1u;
constexpr uint32_t kCellSub = 2u;  // coarse words
constexpr uint32_t kCellList = 2u; // fine words
constexpr uint32_t kPayloadMask = (1u << 30) - 1;

// Entry (uint4): x = polygon id, y = first edge (index into `edges`),
// z = number of edges, w = flags.  A fine cell's entries are contiguous and
// sorted by polygon id; the last one carries kEntLast.
constexpr uint32_t kEntBoundary = 1u; // run the exact crossing test on the listed edges
constexpr uint32_t kEntLast = 2u;

// Edge (int4): (a.x, a.y, b.x, b.y), the directed edge a -> b of the ring.
// A BOUNDARY entry of fine cell (fx, fy) points at the polygon's edge list of
// fine row fy: every non-horizontal edge whose y-span meets the row's open
// strip, sorted by max(a.x, b.x) descending, cut to the edges with
// max(a.x, b.x) > x0 of the cell.  Every edge that a rightward ray from a
// point of the cell can cross is in that list, so the parity over it equals
// the parity over the whole ring.

struct HostIndex {
    int grid_log2 = 0;
    int sub_log2 = 0;
    uint32_t n_polys = 0;
    BigVec<uint32_t> cell;           // 4^g coarse words
    BigVec<uint32_t> fine;           // n_blocks * 4^sub fine words
    BigVec<uint32_t> entries;        // 4 words per entry
    BigVec<int32_t> edges;           // 4 ints per edge
    uint64_t n_blocks = 0;
    uint64_t n_inside = 0;           // (coarse cell, polygon) pairs wholly inside
    uint64_t n_mixed = 0;            // (coarse cell, polygon) pairs split into fine cells
    uint64_t n_boundary = 0;         // (fine cell, polygon) pairs that need the exact test
};

// Grid index of Q disks (centre, radius): cell words as in HostIndex's coarse
// level (empty / INSIDE one disk / list), lists in `entries`.
struct HostDiskIndex {
    int grid_log2 = 0;
    uint32_t n_disks = 0;
    std::vector<uint32_t> cell;     // 4^g words
    std::vector<uint32_t> entries;  // per list: n, then n words (disk << 1 | boundary)
    uint64_t n_inside = 0, n_boundary = 0;
};
bool build_disk_index(const int32_t *cxy, const int32_t *r, uint32_t Q, int g, HostDiskIndex &out, std::string &err);
int default_disk_grid_log2(const int32_t *r, uint32_t Q);

// Item flag of the edge grid: polygon q's r-region holds the whole cell (the
// item carries no edge; the cell's points meet q without a test).
constexpr uint32_t kBufferFull = 0x80000000u;

// Edge grid of P buffered polygons (ring q grown by r[q]): per cell of a
// 2^g grid, the edges whose r-neighbourhood may reach the cell, sorted by
// (polygon, edge), in CSR form.
struct HostBufferEdges {
    int g = 0;
    std::vector<uint32_t> cell_off; // 4^g + 1 item offsets
    std::vector<uint32_t> item_q;   // polygon of each item, | kBufferFull when the whole cell is within r
    std::vector<int32_t> item_seg;  // 4 per item: ax, ay, bx, by
    uint64_t n_full = 0;            // flagged items
};
bool build_buffer_edges(const int32_t *xy, const uint64_t *ring_off, uint32_t P, const int32_t *r, int g,
                        HostBufferEdges &out, std::string &err);
int default_buffer_grid_log2(const int32_t *xy, const uint64_t *ring_off, uint32_t P, const int32_t *r);

// Build the index of P rings (xy: interleaved int32 pairs, ring_off: P + 1
// offsets in vertices) with 2^grid_log2 coarse cells per side, each mixed
// cell split into 2^sub_log2 x 2^sub_log2 fine cells.  Returns false and sets
// err on bad input or if a limit is exceeded.
bool build_grid_index(const int32_t *xy, const uint64_t *ring_off, uint32_t P, int grid_log2, int sub_log2,
                      int threads, HostIndex &out, std::string &err);

// Bounds check of a polygon index's arrays (sizes in words / entries /
// edges, sentinels included): every coarse word names a polygon below P or a
// fine block that exists, every fine word a polygon below P or an entry list
// that ends with its last entry before the sentinels, every entry a polygon
// below P and an edge range inside the edges.  The same predicate the
// kernels apply to each offset they read in a SPX_BOUNDS_CHECK build.
bool validate_grid_index(const uint32_t *cell, uint64_t n_cell, const uint32_t *fine, uint64_t n_fine,
                         const uint32_t *ent, uint64_t n_ent, const int32_t *edges, uint64_t n_edge, int g, int sb,
                         uint32_t P, std::string &err);

// Heuristic coarse grid resolution from the polygon set alone.
int default_grid_log2(const int32_t *xy, const uint64_t *ring_off, uint32_t P);

} // namespace spx
