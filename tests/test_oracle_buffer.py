"""Pins of the oracle's buffered-polygon join (SPADE §4.2 "Canvases for
Distance-Based Queries": a polygon's distance constraint is the polygon plus a
rounded rectangle of radius r around every edge; §5.2 "Distance-Based
Queries").  A point meets (R, r) iff it is inside R (half-open rule) or within
distance r of an edge of R taken as a closed segment.

Pinned against things other than the oracle's own formula:
* lattice-point counts of a buffered axis-parallel rectangle in closed form
  (bands of the rectangle grown by r along each axis, plus four quarter-disk
  corners counted by a column sum of integer square roots);
* exact equality cases of a 3-4-5 geometry (perpendicular foot inside the
  segment, and beyond each end);
* a one-vertex ring is a disk: equals the disk join (pinned by its own tests);
* r = 0 keeps every point of the plain join, adds exactly the points lying on
  an edge, and the result grows with r;
* the threaded run equals a loop over near_ring / point_in_ring.
"""
import math

import numpy as np
import pytest

import oracle


def quarter(r):
    """#{(i, j) : i >= 1, j >= 1, i^2 + j^2 <= r^2} (integer square roots)."""
    return sum(math.isqrt(r * r - i * i) for i in range(1, r + 1))


def rect(x0, y0, x1, y1):
    return np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], np.int32)


def lattice(x0, y0, x1, y1):
    xs, ys = np.meshgrid(np.arange(x0, x1 + 1), np.arange(y0, y1 + 1))
    return np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)


@pytest.mark.parametrize("W,H,r", [(20, 30, 7), (5, 3, 11), (0, 9, 4), (12, 12, 0), (1, 1, 1), (40, 2, 25)])
def test_buffered_rectangle_lattice_count(W, H, r):
    x0, y0 = 5000, 7000
    R = rect(x0, y0, x0 + W, y0 + H)
    pts = lattice(x0 - r - 3, y0 - r - 3, x0 + W + r + 3, y0 + H + r + 3)
    off = np.array([0, 4], np.uint64)
    pairs, counts = oracle.buffer_join(pts, R, off, np.array([r], np.int32), threads=3)
    # closed form: the rectangle grown by r in x (all rows of the rectangle),
    # the two bands above and below it, the four rounded corners
    want = (W + 2 * r + 1) * (H + 1) + 2 * (W + 1) * r + 4 * quarter(r)
    assert int(counts[0]) == want == pairs.shape[0]


def test_equality_cases_3_4_5():
    # segment (0,0)-(300,400) of length 500 as a degenerate two-vertex ring;
    # (110, 230) lies 50 from it, the foot of the perpendicular at its middle
    seg = np.array([[1000, 1000], [1300, 1400]], np.int32)
    p = (1000 + 110, 1000 + 230)
    assert oracle.near_ring(*p, seg, 50) and not oracle.near_ring(*p, seg, 49)
    # beyond the end b: (300 + 3k, 400 + 4k) lies 5k from b, the foot outside
    q = (1300 + 30, 1400 + 40)
    assert oracle.near_ring(*q, seg, 50) and not oracle.near_ring(*q, seg, 49)
    # before the end a
    s = (1000 - 24, 1000 - 7)  # 7-24-25
    assert oracle.near_ring(*s, seg, 25) and not oracle.near_ring(*s, seg, 24)
    # a point exactly on the segment is at distance 0
    assert oracle.near_ring(1000 + 150, 1000 + 200, seg, 0)
    assert not oracle.near_ring(1000 + 150, 1000 + 201, seg, 0)


def test_one_vertex_ring_is_a_disk():
    rng = np.random.default_rng(3)
    c = np.array([[40000, 50000], [41000, 50500], [90000, 10000]], np.int32)
    r = np.array([700, 1300, 0], np.int32)
    pts = rng.integers(37000, 52000, (20000, 2)).astype(np.int32)
    pts[:5] = [[40000, 50700], [40000, 50701], [90000, 10000], [41000 + 1300, 50500], [40700, 50000]]
    off = np.arange(4, dtype=np.uint64)
    got = oracle.buffer_join(pts, c, off, r)
    want = oracle.disk_join(pts, c, r)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_r0_and_monotone_in_r():
    rng = np.random.default_rng(5)
    # concave polygons with vertices on a coarse lattice, points on the same
    # lattice: many points fall exactly on edges
    rings = [np.array([[0, 0], [60, 0], [60, 60], [30, 20], [0, 60]]) * 10 + 1000,
             np.array([[0, 0], [80, 10], [40, 70]]) * 10 + 1200]
    v = np.concatenate(rings).astype(np.int32)
    off = np.array([0, 5, 8], np.uint64)
    pts = (rng.integers(0, 100, (30000, 2)) * 10 + 1000).astype(np.int32)
    plain, _ = oracle.join_pure(pts, v, off)
    zero, _ = oracle.buffer_join(pts, v, off, np.zeros(2, np.int32))
    as_set = lambda a: {(int(i), int(q)) for i, q in a}
    sp, sz = as_set(plain), as_set(zero)
    assert sp <= sz
    for i, q in sz - sp:
        ring = rings[q].astype(np.int32)
        assert oracle.near_ring(int(pts[i, 0]), int(pts[i, 1]), ring, 0)  # only points on an edge are added
    assert len(sz - sp) > 50
    prev = sz
    for r in (5, 17, 60, 250):
        cur = as_set(oracle.buffer_join(pts, v, off, np.full(2, r, np.int32))[0])
        assert prev <= cur
        prev = cur


def test_threads_equal_definition_loop():
    rng = np.random.default_rng(11)
    rings, off = [], [0]
    for k in range(6):
        n = int(rng.integers(3, 12))
        ang = np.sort(rng.uniform(0, 2 * np.pi, n))
        rad = rng.uniform(300, 900, n)
        c = rng.integers(2000, 6000, 2)
        rings.append(np.stack([c[0] + rad * np.cos(ang), c[1] + rad * np.sin(ang)], 1).round().astype(np.int32))
        off.append(off[-1] + n)
    v = np.concatenate(rings)
    off = np.array(off, np.uint64)
    r = rng.integers(0, 400, 6).astype(np.int32)
    pts = rng.integers(1000, 7000, (3000, 2)).astype(np.int32)
    pairs, counts = oracle.buffer_join(pts, v, off, r, threads=4)
    want = [(i, q) for i in range(pts.shape[0]) for q in range(6)
            if oracle.point_in_ring(pts[i, 0], pts[i, 1], rings[q]) or
            oracle.near_ring(pts[i, 0], pts[i, 1], rings[q], int(r[q]))]
    assert [tuple(x) for x in pairs.tolist()] == want
    assert counts.tolist() == [sum(1 for _, q in want if q == k) for k in range(6)]
