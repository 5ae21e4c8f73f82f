/*
 * pip_oracle.c -- TEST INFRASTRUCTURE, not part of the library.
 *
 * A plain, slow, obviously correct CPU oracle for SPADE's point-in-polygon
 * join, selection and count (§5.2 "Spatial Selection", "Spatial Joins",
 * "Spatial Aggregations").  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg and reference arm may load it.  It shares no code, header, table
 * or helper with the CUDA library.
 *
 * What it computes (the definition; every faster method must reach exactly it):
 *
 *   For points, intersection is the same as containment (§7, "Containment
 *   Queries"), so a point p meets polygon R iff p lies inside R.  Boundary
 *   locations need an exact test (§4.3, "Boundary Index"); the exact test here
 *   is the crossing number with a half-open rule on int32 fixed-point input:
 *
 *     inside(p, R) = parity of #{ edges (a, b) of R :
 *                      (a.y > p.y) != (b.y > p.y)                  [straddle]
 *                  and d = (b.x-a.x)(p.y-a.y) - (b.y-a.y)(p.x-a.x) != 0
 *                  and sign(d) == sign(b.y - a.y) }                [p left of
 *                                                                    the upward edge]
 *
 *   d is evaluated in int64 and is exact (|d| <= 2^61).  The rule decides
 *   whether p + (eps, eps^2), for an infinitesimal eps > 0, lies in the
 *   even-odd interior of R, so on a shared edge exactly one of two adjacent
 *   polygons takes the point.
 *
 *   join      = all (point_id, polygon_id) with inside = 1, sorted by point id,
 *               then polygon id (a join is a collection of selections, §5.2)
 *   counts[q] = number of join pairs with polygon q (aggregation = join + count)
 *   select    = for each query polygon, its ascending list of point ids
 *
 * Two modes:
 *   pure -- every edge of every polygon for every point.
 *   fast -- three shortcuts, each of which provably keeps the definition:
 *     (s1) half-open bbox reject: inside => xmin <= px < xmax and ymin <= py < ymax;
 *     (s2) y-slab edge buckets per polygon: only an edge with
 *          min(a.y, b.y) <= p.y < max(a.y, b.y) can straddle, and that is
 *          exactly the straddle test, so an edge outside p's slab never counts;
 *     (s3) a coarse bucket grid of polygon bounding boxes to find the polygons
 *          whose half-open bbox can contain p.
 *   The fast mode runs on several threads over contiguous point ranges.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_BOX_LOG2 30

/* one edge's contribution to the crossing parity (the rule above) */
static int edge_counts(int64_t px, int64_t py, int64_t ax, int64_t ay, int64_t bx, int64_t by)
{
    if ((ay > py) == (by > py))
        return 0;
    int64_t d = (bx - ax) * (py - ay) - (by - ay) * (px - ax);
    if (d == 0)
        return 0;
    return (d > 0) == (by > ay);
}

/* inside(p, R) over every edge of one ring of n vertices */
int oracle_point_in_ring(int32_t px, int32_t py, const int32_t *xy, uint64_t n)
{
    int in = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t j = (i + 1 == n) ? 0 : i + 1;
        in ^= edge_counts(px, py, xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1]);
    }
    return in;
}

/*
 * Pure join.  pairs (2 * cap uint32, may be NULL when cap = 0) receives the
 * first cap pairs in (point id, polygon id) order; counts (P uint64, may be
 * NULL) receives per-polygon pair counts.  Returns the total number of pairs.
 */
uint64_t oracle_join_pure(const int32_t *pts, uint64_t n, const int32_t *xy, const uint64_t *ring_off,
                          uint32_t P, uint32_t *pairs, uint64_t cap, uint64_t *counts)
{
    uint64_t total = 0;
    if (counts)
        memset(counts, 0, sizeof(uint64_t) * P);
    for (uint64_t i = 0; i < n; ++i) {
        for (uint32_t q = 0; q < P; ++q) {
            uint64_t b = ring_off[q], e = ring_off[q + 1];
            if (oracle_point_in_ring(pts[2 * i], pts[2 * i + 1], xy + 2 * b, e - b)) {
                if (total < cap) {
                    pairs[2 * total] = (uint32_t)i;
                    pairs[2 * total + 1] = q;
                }
                if (counts)
                    counts[q]++;
                total++;
            }
        }
    }
    return total;
}

/* ------------------------------------------------------------ fast mode */

typedef struct {
    int32_t xmin, ymin, xmax, ymax; /* closed bbox of the vertices */
    uint64_t vb, nv;                /* ring = xy[vb .. vb + nv) */
    int64_t slab_h;                 /* slab height, >= 1 */
    uint32_t nslab;
    uint64_t slab_begin;            /* into oracle->slab_off */
} opoly;

typedef struct {
    const int32_t *xy;   /* borrowed: the caller keeps the ring arrays alive */
    uint32_t P;
    opoly *poly;
    uint64_t *slab_off;  /* per polygon nslab+1 offsets into slab_edge (global) */
    uint32_t *slab_edge; /* edge index i within its ring (edge i -> i+1) */
    int bucket_log2;     /* bucket side = 2^bucket_log2 */
    int nb;              /* buckets per side */
    uint64_t *bucket_off;/* nb*nb + 1 */
    uint32_t *bucket_poly;
} oracle_t;

static int32_t edge_ylo(const int32_t *r, uint64_t n, uint64_t i, int32_t *hi)
{
    uint64_t j = (i + 1 == n) ? 0 : i + 1;
    int32_t a = r[2 * i + 1], b = r[2 * j + 1];
    *hi = a > b ? a : b;
    return a < b ? a : b;
}

void oracle_free(oracle_t *o)
{
    if (!o)
        return;
    free(o->poly);
    free(o->slab_off);
    free(o->slab_edge);
    free(o->bucket_off);
    free(o->bucket_poly);
    free(o);
}

/* Build the fast-mode acceleration structures.  Returns NULL on bad input. */
oracle_t *oracle_prepare(const int32_t *xy, const uint64_t *ring_off, uint32_t P)
{
    oracle_t *o = (oracle_t *)calloc(1, sizeof(oracle_t));
    if (!o)
        return NULL;
    o->xy = xy;
    o->P = P;
    o->poly = (opoly *)calloc(P ? P : 1, sizeof(opoly));
    uint64_t total_slabs = 0;
    for (uint32_t q = 0; q < P; ++q) {
        opoly *g = &o->poly[q];
        g->vb = ring_off[q];
        g->nv = ring_off[q + 1] - ring_off[q];
        g->xmin = g->ymin = INT32_MAX;
        g->xmax = g->ymax = INT32_MIN;
        for (uint64_t k = 0; k < g->nv; ++k) {
            int32_t x = xy[2 * (g->vb + k)], y = xy[2 * (g->vb + k) + 1];
            if (x < g->xmin) g->xmin = x;
            if (x > g->xmax) g->xmax = x;
            if (y < g->ymin) g->ymin = y;
            if (y > g->ymax) g->ymax = y;
        }
        if (g->nv == 0) {
            g->xmin = g->ymin = 0;
            g->xmax = g->ymax = 0;
        }
        uint64_t ns = g->nv / 4;
        if (ns < 1) ns = 1;
        if (ns > 4096) ns = 4096;
        int64_t hgt = (int64_t)g->ymax - g->ymin;
        if (hgt < 1) hgt = 1;
        g->slab_h = (hgt + (int64_t)ns - 1) / (int64_t)ns;
        g->nslab = (uint32_t)((hgt + g->slab_h - 1) / g->slab_h);
        g->slab_begin = total_slabs;
        total_slabs += g->nslab + 1;
    }
    /* (s2) y-slab buckets: edge i of polygon q goes to every slab that meets
     * [ylo, yhi).  Each polygon owns nslab + 1 slots of slab_off; after the
     * scan, slot s holds the begin of slab s and slot nslab the end of the last. */
    o->slab_off = (uint64_t *)calloc(total_slabs + 1, sizeof(uint64_t));
    uint64_t *cursor = (uint64_t *)calloc(total_slabs + 1, sizeof(uint64_t));
    for (int pass = 0; pass < 2; ++pass) {
        for (uint32_t q = 0; q < P; ++q) {
            opoly *g = &o->poly[q];
            const int32_t *r = xy + 2 * g->vb;
            for (uint64_t i = 0; i < g->nv; ++i) {
                int32_t hi;
                int32_t lo = edge_ylo(r, g->nv, i, &hi);
                if (hi <= lo)
                    continue; /* horizontal: never straddles */
                int64_t s0 = ((int64_t)lo - g->ymin) / g->slab_h;
                int64_t s1 = ((int64_t)hi - 1 - g->ymin) / g->slab_h;
                for (int64_t sl = s0; sl <= s1 && sl < (int64_t)g->nslab; ++sl) {
                    uint64_t slot = g->slab_begin + (uint64_t)sl;
                    if (pass == 0)
                        cursor[slot]++;
                    else
                        o->slab_edge[cursor[slot]++] = (uint32_t)i;
                }
            }
        }
        if (pass == 0) {
            uint64_t run = 0;
            for (uint64_t k = 0; k < total_slabs; ++k) {
                uint64_t c = cursor[k];
                o->slab_off[k] = run;
                cursor[k] = run;
                run += c;
            }
            o->slab_off[total_slabs] = run;
            o->slab_edge = (uint32_t *)malloc(sizeof(uint32_t) * (run ? run : 1));
        }
    }
    free(cursor);
    /* (s3) bucket grid over the box: 256 x 256 buckets */
    o->bucket_log2 = ORACLE_BOX_LOG2 - 8;
    o->nb = 1 << 8;
    uint64_t nbk = (uint64_t)o->nb * o->nb;
    o->bucket_off = (uint64_t *)calloc(nbk + 1, sizeof(uint64_t));
    for (int pass = 0; pass < 2; ++pass) {
        for (uint32_t q = 0; q < P; ++q) {
            opoly *g = &o->poly[q];
            if (g->xmax <= g->xmin || g->ymax <= g->ymin)
                continue; /* empty half-open bbox: nothing can be inside */
            int bx0 = g->xmin >> o->bucket_log2, bx1 = (g->xmax - 1) >> o->bucket_log2;
            int by0 = g->ymin >> o->bucket_log2, by1 = (g->ymax - 1) >> o->bucket_log2;
            if (bx1 >= o->nb) bx1 = o->nb - 1;
            if (by1 >= o->nb) by1 = o->nb - 1;
            for (int by = by0; by <= by1; ++by)
                for (int bx = bx0; bx <= bx1; ++bx) {
                    uint64_t k = (uint64_t)by * o->nb + bx;
                    if (pass == 0)
                        o->bucket_off[k + 1]++;
                    else
                        o->bucket_poly[o->bucket_off[k]++] = q;
                }
        }
        if (pass == 0) {
            for (uint64_t k = 0; k < nbk; ++k)
                o->bucket_off[k + 1] += o->bucket_off[k];
            o->bucket_poly = (uint32_t *)malloc(sizeof(uint32_t) * (o->bucket_off[nbk] ? o->bucket_off[nbk] : 1));
        } else {
            for (uint64_t k = nbk; k > 0; --k)
                o->bucket_off[k] = o->bucket_off[k - 1];
            o->bucket_off[0] = 0;
        }
    }
    return o;
}

/* inside(p, q) through the shortcuts s1 and s2 */
static int fast_inside(const oracle_t *o, uint32_t q, int32_t px, int32_t py)
{
    const opoly *g = &o->poly[q];
    if (px < g->xmin || px >= g->xmax || py < g->ymin || py >= g->ymax)
        return 0; /* (s1) */
    int64_t s = ((int64_t)py - g->ymin) / g->slab_h;
    const uint64_t *off = o->slab_off + g->slab_begin;
    const int32_t *r = o->xy + 2 * g->vb;
    int in = 0;
    for (uint64_t k = off[s]; k < off[s + 1]; ++k) { /* (s2) */
        uint64_t i = o->slab_edge[k];
        uint64_t j = (i + 1 == g->nv) ? 0 : i + 1;
        in ^= edge_counts(px, py, r[2 * i], r[2 * i + 1], r[2 * j], r[2 * j + 1]);
    }
    return in;
}

typedef struct {
    const oracle_t *o;
    const int32_t *pts;
    uint64_t lo, hi;
    int want_pairs;
    uint32_t *pairs; /* grown */
    uint64_t npairs, cap;
    uint64_t *counts;
} ojob;

static void *fast_worker(void *arg)
{
    ojob *j = (ojob *)arg;
    const oracle_t *o = j->o;
    for (uint64_t i = j->lo; i < j->hi; ++i) {
        int32_t px = j->pts[2 * i], py = j->pts[2 * i + 1];
        /* every vertex lies in [0, 2^30]^2 and the half-open rule leaves the
         * box's right and top sides outside, so a point outside [0, 2^30)^2 is
         * in no polygon (and has no bucket) */
        if (px < 0 || py < 0 || px >= (1 << ORACLE_BOX_LOG2) || py >= (1 << ORACLE_BOX_LOG2))
            continue;
        uint64_t k = (uint64_t)(py >> o->bucket_log2) * o->nb + (uint64_t)(px >> o->bucket_log2);
        for (uint64_t m = o->bucket_off[k]; m < o->bucket_off[k + 1]; ++m) { /* (s3) */
            uint32_t q = o->bucket_poly[m];
            if (!fast_inside(o, q, px, py))
                continue;
            j->counts[q]++;
            if (j->want_pairs) {
                if (j->npairs == j->cap) {
                    j->cap = j->cap ? 2 * j->cap : 1024;
                    j->pairs = (uint32_t *)realloc(j->pairs, sizeof(uint32_t) * 2 * j->cap);
                }
                j->pairs[2 * j->npairs] = (uint32_t)i;
                j->pairs[2 * j->npairs + 1] = q;
            }
            j->npairs++;
        }
    }
    return NULL;
}

/*
 * Fast join over nthreads threads (contiguous point ranges, results
 * concatenated in range order, so the order is the same as the pure join's).
 * pairs may be NULL (count only).  Returns the total number of pairs.
 */
uint64_t oracle_join_fast(const oracle_t *o, const int32_t *pts, uint64_t n, uint32_t *pairs, uint64_t cap,
                          uint64_t *counts, int nthreads)
{
    if (nthreads < 1)
        nthreads = 1;
    if ((uint64_t)nthreads > n && n > 0)
        nthreads = (int)n;
    ojob *jobs = (ojob *)calloc(nthreads, sizeof(ojob));
    pthread_t *th = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].o = o;
        jobs[t].pts = pts;
        jobs[t].lo = n * (uint64_t)t / nthreads;
        jobs[t].hi = n * (uint64_t)(t + 1) / nthreads;
        jobs[t].want_pairs = pairs != NULL;
        jobs[t].counts = (uint64_t *)calloc(o->P ? o->P : 1, sizeof(uint64_t));
        pthread_create(&th[t], NULL, fast_worker, &jobs[t]);
    }
    uint64_t total = 0;
    if (counts)
        memset(counts, 0, sizeof(uint64_t) * o->P);
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (pairs) {
            for (uint64_t k = 0; k < jobs[t].npairs && total + k < cap; ++k) {
                pairs[2 * (total + k)] = jobs[t].pairs[2 * k];
                pairs[2 * (total + k) + 1] = jobs[t].pairs[2 * k + 1];
            }
        }
        if (counts)
            for (uint32_t q = 0; q < o->P; ++q)
                counts[q] += jobs[t].counts[q];
        total += jobs[t].npairs;
        free(jobs[t].pairs);
        free(jobs[t].counts);
    }
    free(jobs);
    free(th);
    return total;
}


/*
 * Distance join of points with disks (SPADE §4.2 "Canvases for Distance-Based
 * Queries" and §5.2 "Distance-Based Queries": a point lies within distance r
 * of a centre c iff distance(p, c) <= r).  With integer coordinates the test is
 * exact in int64: (px - cx)^2 + (py - cy)^2 <= r^2 (|differences| < 2^31, so
 * each square is below 2^62; radii are below 2^30, so r^2 < 2^60 and the sum
 * of two squares that exceeds r^2 is detected before it could overflow).
 * Pairs (point id, disk id) in lexicographic order; counts[q] per disk.
 * Every disk is tested for every point: the definition, written out.
 */
uint64_t oracle_disk_join(const int32_t *pts, uint64_t n, const int32_t *cxy, const int32_t *r, uint32_t Q,
                          uint32_t *pairs, uint64_t cap, uint64_t *counts)
{
    uint64_t total = 0;
    for (uint32_t q = 0; q < Q; ++q)
        counts[q] = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const int64_t px = pts[2 * i], py = pts[2 * i + 1];
        /* the points' domain is [0, 2^30)^2; a point outside it is in no disk */
        if (px < 0 || py < 0 || px >= (1 << ORACLE_BOX_LOG2) || py >= (1 << ORACLE_BOX_LOG2))
            continue;
        for (uint32_t q = 0; q < Q; ++q) {
            const int64_t dx = px - cxy[2 * q], dy = py - cxy[2 * q + 1], rr = (int64_t)r[q] * r[q];
            const int64_t dx2 = dx * dx;
            if (dx2 > rr)
                continue;
            if (dx2 + dy * dy > rr)
                continue;
            if (pairs && total < cap) {
                pairs[2 * total] = (uint32_t)i;
                pairs[2 * total + 1] = q;
            }
            counts[q]++;
            total++;
        }
    }
    return total;
}


/* ------------------------------------------------ buffered polygons */

/*
 * Buffered-polygon join (SPADE §4.2 "Canvases for Distance-Based Queries": a
 * distance constraint of radius r around a polygon is drawn as the polygon
 * together with a rounded rectangle of radius r around each of its edges;
 * §5.2 "Distance-Based Queries"): point p meets the buffered polygon (R, r)
 * iff p lies inside R (the half-open rule above) or the distance from p to
 * some edge of R, taken as a closed segment, is at most r.  The union of R and
 * the rounded rectangles is exactly the set of points within distance r of R.
 *
 * Distance to the segment a -> b (d = b - a, w = p - a, t = w . d):
 *   t <= 0        : |p - a|
 *   t >= |d|^2    : |p - b|
 *   otherwise     : |d x w| / |d|   (the foot of the perpendicular lies inside)
 * Every comparison is exact: coordinates lie in [0, 2^30], so each product of
 * differences is below 2^60 in magnitude and sums of two stay below 2^62 in
 * int64; the perpendicular case compares (d x w)^2 <= r^2 |d|^2, both below
 * 2^123, in unsigned 128-bit arithmetic.  A ring's degenerate edge (a = b) has
 * |d|^2 = 0 and takes the first case.
 */
static int seg_within(int64_t px, int64_t py, int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t r)
{
    const int64_t dx = bx - ax, dy = by - ay, wx = px - ax, wy = py - ay, rr = r * r;
    const int64_t t = wx * dx + wy * dy;
    if (t <= 0)
        return wx * wx + wy * wy <= rr;
    const int64_t dd = dx * dx + dy * dy;
    if (t >= dd) {
        const int64_t ux = px - bx, uy = py - by;
        return ux * ux + uy * uy <= rr;
    }
    const int64_t c = dx * wy - dy * wx;
    const unsigned __int128 ca = (unsigned __int128)(uint64_t)(c < 0 ? -c : c);
    return ca * ca <= (unsigned __int128)(uint64_t)rr * (unsigned __int128)(uint64_t)dd;
}

/* p within distance r of an edge of the ring of n vertices (every edge) */
int oracle_near_ring(int32_t px, int32_t py, const int32_t *xy, uint64_t n, int32_t r)
{
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t j = (i + 1 == n) ? 0 : i + 1;
        if (seg_within(px, py, xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1], r))
            return 1;
    }
    return 0;
}

typedef struct {
    const int32_t *pts, *xy, *r;
    const uint64_t *ring_off;
    const int64_t *box; /* per polygon: closed vertex bbox grown by r (xmin, ymin, xmax, ymax) */
    uint32_t P;
    uint64_t lo, hi;
    int want_pairs;
    uint32_t *pairs;
    uint64_t npairs, cap;
    uint64_t *counts;
} bjob;

static void *buffer_worker(void *arg)
{
    bjob *j = (bjob *)arg;
    for (uint64_t i = j->lo; i < j->hi; ++i) {
        const int32_t px = j->pts[2 * i], py = j->pts[2 * i + 1];
        /* the points' domain is [0, 2^30)^2; a point outside it meets nothing */
        if (px < 0 || py < 0 || px >= (1 << ORACLE_BOX_LOG2) || py >= (1 << ORACLE_BOX_LOG2))
            continue;
        for (uint32_t q = 0; q < j->P; ++q) {
            const int64_t *b = j->box + 4 * (uint64_t)q;
            /* inside R implies inside its vertex bbox, and a point within r of
             * an edge lies within r of the edge's bbox: outside the bbox grown
             * by r, neither holds */
            if (px < b[0] || py < b[1] || px > b[2] || py > b[3])
                continue;
            const uint64_t v0 = j->ring_off[q], nv = j->ring_off[q + 1] - v0;
            if (!oracle_point_in_ring(px, py, j->xy + 2 * v0, nv) &&
                !oracle_near_ring(px, py, j->xy + 2 * v0, nv, j->r[q]))
                continue;
            j->counts[q]++;
            if (j->want_pairs) {
                if (j->npairs == j->cap) {
                    j->cap = j->cap ? 2 * j->cap : 1024;
                    j->pairs = (uint32_t *)realloc(j->pairs, sizeof(uint32_t) * 2 * j->cap);
                }
                j->pairs[2 * j->npairs] = (uint32_t)i;
                j->pairs[2 * j->npairs + 1] = q;
            }
            j->npairs++;
        }
    }
    return NULL;
}

/*
 * Buffered-polygon join over nthreads threads (contiguous point ranges,
 * concatenated in range order): pairs (point id, polygon id) sorted, the
 * first cap of them into pairs (may be NULL), counts (P, may be NULL).
 * r[q] in [0, 2^30).  Returns the total number of pairs.
 */
uint64_t oracle_buffer_join(const int32_t *pts, uint64_t n, const int32_t *xy, const uint64_t *ring_off, uint32_t P,
                            const int32_t *r, uint32_t *pairs, uint64_t cap, uint64_t *counts, int nthreads)
{
    int64_t *box = (int64_t *)malloc(sizeof(int64_t) * 4 * (P ? P : 1));
    for (uint32_t q = 0; q < P; ++q) {
        int64_t x0 = INT64_MAX, y0 = INT64_MAX, x1 = INT64_MIN, y1 = INT64_MIN;
        for (uint64_t v = ring_off[q]; v < ring_off[q + 1]; ++v) {
            x0 = xy[2 * v] < x0 ? xy[2 * v] : x0;
            x1 = xy[2 * v] > x1 ? xy[2 * v] : x1;
            y0 = xy[2 * v + 1] < y0 ? xy[2 * v + 1] : y0;
            y1 = xy[2 * v + 1] > y1 ? xy[2 * v + 1] : y1;
        }
        box[4 * q] = x0 - r[q];
        box[4 * q + 1] = y0 - r[q];
        box[4 * q + 2] = x1 + r[q];
        box[4 * q + 3] = y1 + r[q];
    }
    if (nthreads < 1)
        nthreads = 1;
    if ((uint64_t)nthreads > n && n > 0)
        nthreads = (int)n;
    bjob *jobs = (bjob *)calloc(nthreads, sizeof(bjob));
    pthread_t *th = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        bjob *j = &jobs[t];
        j->pts = pts;
        j->xy = xy;
        j->r = r;
        j->ring_off = ring_off;
        j->box = box;
        j->P = P;
        j->lo = n * (uint64_t)t / nthreads;
        j->hi = n * (uint64_t)(t + 1) / nthreads;
        j->want_pairs = pairs != NULL;
        j->counts = (uint64_t *)calloc(P ? P : 1, sizeof(uint64_t));
        pthread_create(&th[t], NULL, buffer_worker, j);
    }
    uint64_t total = 0;
    if (counts)
        memset(counts, 0, sizeof(uint64_t) * P);
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (pairs)
            for (uint64_t k = 0; k < jobs[t].npairs && total + k < cap; ++k) {
                pairs[2 * (total + k)] = jobs[t].pairs[2 * k];
                pairs[2 * (total + k) + 1] = jobs[t].pairs[2 * k + 1];
            }
        if (counts)
            for (uint32_t q = 0; q < P; ++q)
                counts[q] += jobs[t].counts[q];
        total += jobs[t].npairs;
        free(jobs[t].pairs);
        free(jobs[t].counts);
    }
    free(jobs);
    free(th);
    free(box);
    return total;
}
