"""The seeded generators: determinism, ranges, and a valid tessellation
(no two cell boundaries cross, checked by brute force with exact integers)."""
import numpy as np
import pytest

from paper_2203_14362_gb300 import datagen as g


def test_deterministic_and_sliceable():
    a = g.mixture_points(50_000, 77)
    b = g.mixture_points(50_000, 77)
    assert np.array_equal(a, b)
    c = g.mixture_points(20_000, 77, start=30_000)
    assert np.array_equal(a[30_000:], c)
    u = g.uniform_points(10_000, 5)
    assert np.array_equal(u, g.uniform_points(10_000, 5))
    assert not np.array_equal(u, g.uniform_points(10_000, 6))


def test_ranges():
    for p in (g.uniform_points(100_000, 1), g.mixture_points(100_000, 2),
              g.mixture_points(100_000, 3, g.make_mixture(3, zipf_s=1.1))):
        assert p.dtype == np.int32 and p.min() >= 0 and p.max() < (1 << 30)
    v, o = g.star_polygons(4)
    assert len(o) == 257 and np.diff(o).min() >= 16 and np.diff(o).max() <= 64
    assert v.min() >= 0 and v.max() <= (1 << 30)
    mix = g.make_mixture(5)
    v, o = g.query_polygons(64, 5, mix)
    assert np.diff(o).min() >= 8 and np.diff(o).max() <= 5000
    assert v.min() >= 0 and v.max() <= (1 << 30)


def segments(t):
    v = t.verts.astype(np.int64)
    segs = []
    for q in range(len(t.ring_off) - 1):
        b, e = int(t.ring_off[q]), int(t.ring_off[q + 1])
        r = v[b:e]
        segs.append(np.concatenate([r, np.roll(r, -1, 0)], 1))
    s = np.concatenate(segs)
    # each interior edge appears twice (once per neighbour): keep one copy
    key = np.where((s[:, :2] < s[:, 2:]).all(1)[:, None] | ((s[:, 0] < s[:, 2]) | ((s[:, 0] == s[:, 2]) & (s[:, 1] < s[:, 3])))[:, None],
                   s, np.concatenate([s[:, 2:], s[:, :2]], 1))
    return np.unique(key, axis=0)


def orient(ax, ay, bx, by, cx, cy):
    return np.sign((bx - ax) * (cy - ay) - (by - ay) * (cx - ax))


@pytest.mark.parametrize("nx,ny,seed,kmax", [(3, 3, 1, 25), (4, 2, 7, 40), (2, 5, 13, 60)])
def test_tessellation_has_no_crossings(nx, ny, seed, kmax):
    t = g.quad_tessellation(nx, ny, seed, kmin=2, kmax=kmax)
    assert t.verts.min() >= 0 and t.verts.max() <= (1 << 30)
    s = segments(t)
    n = s.shape[0]
    i, j = np.triu_indices(n, 1)
    A, Bs = s[i], s[j]
    o1 = orient(A[:, 0], A[:, 1], A[:, 2], A[:, 3], Bs[:, 0], Bs[:, 1])
    o2 = orient(A[:, 0], A[:, 1], A[:, 2], A[:, 3], Bs[:, 2], Bs[:, 3])
    o3 = orient(Bs[:, 0], Bs[:, 1], Bs[:, 2], Bs[:, 3], A[:, 0], A[:, 1])
    o4 = orient(Bs[:, 0], Bs[:, 1], Bs[:, 2], Bs[:, 3], A[:, 2], A[:, 3])
    proper = (o1 * o2 < 0) & (o3 * o4 < 0)
    assert not proper.any()
    share = ((A[:, :2] == Bs[:, :2]).all(1) | (A[:, :2] == Bs[:, 2:]).all(1) |
             (A[:, 2:] == Bs[:, :2]).all(1) | (A[:, 2:] == Bs[:, 2:]).all(1))
    # touching without sharing an endpoint: one endpoint on the other segment
    def on_seg(P, S, o):
        return (o == 0) & (np.minimum(S[:, 0], S[:, 2]) <= P[:, 0]) & (P[:, 0] <= np.maximum(S[:, 0], S[:, 2])) & \
               (np.minimum(S[:, 1], S[:, 3]) <= P[:, 1]) & (P[:, 1] <= np.maximum(S[:, 1], S[:, 3]))
    touch = on_seg(Bs[:, :2], A, o1) | on_seg(Bs[:, 2:], A, o2) | on_seg(A[:, :2], Bs, o3) | on_seg(A[:, 2:], Bs, o4)
    # border edges are collinear runs along the box sides: neighbours there share endpoints only
    assert not (touch & ~share).any()
    # two segments sharing an endpoint must not overlap collinearly: with P the
    # shared endpoint and Q1, Q2 the others, overlap = collinear and (Q1-P).(Q2-P) > 0
    coll = share & (o1 == 0) & (o2 == 0)
    a0, a1, b0, b1 = A[coll, :2], A[coll, 2:], Bs[coll, :2], Bs[coll, 2:]
    P = np.where(((a0 == b0).all(1) | (a0 == b1).all(1))[:, None], a0, a1)
    Q1 = np.where((a0 == P).all(1)[:, None], a1, a0)
    Q2 = np.where((b0 == P).all(1)[:, None], b1, b0)
    assert not (((Q1 - P) * (Q2 - P)).sum(1) > 0).any()


def test_tessellation_vertex_counts():
    t = g.quad_tessellation(5, 4, 3, kmin=12, kmax=499)
    nv = np.diff(t.ring_off)
    assert nv.min() >= 4 + 4 * 12 and nv.max() <= 4 + 4 * 499


def test_mixture_points_parallel_is_identical():
    mix = g.make_mixture(91)
    n = (1 << 23) * 2 + 12345  # three chunks, the last ragged
    a = g.mixture_points_parallel(n, 91, mix, start=777, workers=3)
    b = g.mixture_points(n, 91, mix, start=777)
    assert a.dtype == np.int32 and a.shape == (n, 2)
    assert np.array_equal(a, b)
