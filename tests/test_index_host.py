"""The grid index built by libspx on the host, checked without a GPU.

For every probe point, the candidate lists of its cell are walked the way the
kernels walk them (INSIDE entries match, BOUNDARY entries take the crossing
parity over the listed edges) and the result must equal the oracle's join
exactly.  Structural invariants of the index are checked too: lists sorted by
polygon id and terminated, edge lists sorted by max x descending with every
max x right of the cell's left border.
"""
import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import datagen as g
from paper_2203_14362_gb300 import spx

MASK = (1 << 30) - 1


def parity(px, py, lst):
    """Crossing parity of each point (px, py arrays) over an edge list, exact int64."""
    if lst.shape[0] == 0:
        return np.zeros(px.shape[0], np.int64)
    e = lst.astype(np.int64)
    ax, ay, bx, by = (e[:, k][:, None] for k in range(4))
    X, Y = px[None, :], py[None, :]
    strad = (ay > Y) != (by > Y)
    d = (bx - ax) * (Y - ay) - (by - ay) * (X - ax)
    cnt = strad & (d != 0) & ((d > 0) == (by > ay))
    return cnt.sum(0) & 1


def walk(ix, pts, check_structure=True):
    """The kernels' traversal (coarse word, fine word of a mixed cell, entry
    list, crossing parity), vectorised over the points of each fine cell."""
    gl, sb = ix["g"], ix["sub"]
    sc, sf, F = 30 - gl, 30 - gl - sb, 1 << sb
    coarse, fine, ent, edges = ix["coarse"], ix["fine"], ix["entries"], ix["edges"]
    px = pts[:, 0].astype(np.int64)
    py = pts[:, 1].astype(np.int64)
    w = coarse[((py >> sc) << gl) | (px >> sc)].astype(np.int64)
    kind = w >> 30
    sub = kind == 2
    fidx = ((w & MASK) << (2 * sb)) | (((py >> sf) & (F - 1)) << sb) | ((px >> sf) & (F - 1))
    w = np.where(sub, fine[np.where(sub, fidx, 0)].astype(np.int64), w)
    kind = w >> 30
    out_pid, out_q = [np.nonzero(kind == 1)[0]], [(w[kind == 1] & MASK)]
    lst_pts = np.nonzero(kind == 2)[0]
    e0 = w[lst_pts] & MASK
    fcell = ((py[lst_pts] >> sf) << 20) | (px[lst_pts] >> sf)
    order = np.lexsort((fcell, e0))
    lst_pts, e0, fcell = lst_pts[order], e0[order], fcell[order]
    if lst_pts.size:
        brk = np.nonzero((np.diff(e0) != 0) | (np.diff(fcell) != 0))[0] + 1
        groups = np.split(np.arange(lst_pts.size), brk)
    else:
        groups = []
    for gi in groups:
        idx = lst_pts[gi]
        e = int(e0[gi[0]])
        x0 = int(px[idx[0]] >> sf) << sf
        last_q = -1
        while True:
            q, eb, ec, fl = (int(v) for v in ent[e])
            if check_structure:
                assert q > last_q, "cell list not sorted by polygon id"
            last_q = q
            if fl & 1:
                lst = edges[eb:eb + ec]
                if check_structure and ec:
                    xm = np.maximum(lst[:, 0], lst[:, 2]).astype(np.int64)
                    assert (np.diff(xm) <= 0).all(), "row edge list not sorted by max x"
                    assert (xm > x0).all(), "edge left of the cell in a BOUNDARY list"
                m = parity(px[idx], py[idx], lst).astype(bool)
                out_pid.append(idx[m])
                out_q.append(np.full(int(m.sum()), q, np.int64))
            else:
                out_pid.append(idx)
                out_q.append(np.full(idx.shape[0], q, np.int64))
            if fl & 2:
                break
            e += 1
    pid = np.concatenate(out_pid)
    q = np.concatenate(out_q)
    o = np.lexsort((q, pid))
    return np.stack([pid[o], q[o]], 1).astype(np.uint32)


def scaled_tiny(scale_log2=26):
    """Small hand-made rings scaled so every vertex lies on power-of-two grid lines."""
    rings = [
        [(2, 2), (10, 2), (10, 9), (2, 9)],
        [(0, 0), (8, 0), (0, 8)],
        [(3, 3), (12, 12), (12, 3), (3, 12)],
        [(2, 8), (8, 2), (14, 8), (8, 14), (8, 8)],
        [(1, 1), (5, 1), (5, 5), (9, 5), (9, 1), (13, 1), (13, 13), (1, 13)],
        [(0, 0), (16, 0), (16, 16), (0, 16)],
        [(5, 0), (10, 5), (5, 10), (0, 5)],
        [(1, 3), (7, 3), (7, 9), (11, 9), (11, 3), (15, 3), (15, 13), (1, 13)],
        [(3, 7), (13, 7), (13, 7)],
    ]
    s = 1 << scale_log2
    v = np.concatenate([np.array(r, np.int64) * s for r in rings]).astype(np.int32)
    off = np.zeros(len(rings) + 1, np.uint64)
    off[1:] = np.cumsum([len(r) for r in rings])
    lat = np.array([(x * s + dx, y * s + dy) for x in range(16) for y in range(16)
                    for dx in (0, 1) for dy in (0, 1)], dtype=np.int64)
    lat = np.concatenate([lat, np.array([(x * s - 1, y * s - 1) for x in range(1, 16) for y in range(1, 16)])])
    return v, off, lat.astype(np.int32)


def tess_points(t, n_random=4000, seed=3):
    rng = np.random.default_rng(seed)
    v = t.verts.astype(np.int64)
    pts = [rng.integers(0, 1 << 30, (n_random, 2)), v, v + 1, v - 1, v + [1, 0], v + [0, 1]]
    p = np.concatenate(pts)
    ok = (p >= 0).all(1) & (p < (1 << 30)).all(1)
    return p[ok].astype(np.int32)


CASES = {}


def case(name):
    if name in CASES:
        return CASES[name]
    if name == "stars":
        v, o = g.star_polygons(g.SEED_BASE + 1)
        pts = g.uniform_points(6000, 3)
        pts = np.concatenate([pts, v[:3000]])
    elif name == "tess":
        t = g.quad_tessellation(7, 6, 11, kmin=3, kmax=60)
        v, o, pts = t.verts, t.ring_off, tess_points(t)
    elif name == "queries":
        mix = g.make_mixture(21)
        v, o = g.query_polygons(24, 21, mix, vmax=600, r_med=0.05)
        pts = np.concatenate([g.mixture_points(6000, 21, mix), v[:: max(1, len(v) // 2000)]])
    elif name == "grid_aligned":
        v, o, pts = scaled_tiny()
    else:
        raise KeyError(name)
    pts = pts[(pts >= 0).all(1) & (pts < (1 << 30)).all(1)]
    pairs, counts = oracle.join_fast(pts, v, o)
    CASES[name] = (v, o, pts, pairs)
    return CASES[name]


@pytest.mark.parametrize("name", ["stars", "tess", "queries", "grid_aligned"])
@pytest.mark.parametrize("gl,sb", [(1, 1), (3, 3), (6, 1), (6, 3), (9, 2), (11, 3)])
def test_host_index_matches_oracle(name, gl, sb):
    v, o, pts, want = case(name)
    ix = spx.host_index(v, o, gl, sb)
    assert ix["g"] == gl and ix["sub"] == sb and ix["coarse"].shape[0] == 1 << (2 * gl)
    got = walk(ix, pts)
    assert np.array_equal(got, want)


def test_default_grid_choice():
    v, o = g.star_polygons(g.SEED_BASE + 1)
    ix = spx.host_index(v, o, 0, 0)
    assert 5 <= ix["g"] <= 11 and ix["sub"] == 3


def test_library_exports_every_declared_symbol():
    import ctypes
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "spx.h")).read()
    declared = set(re.findall(r"^\s*(?:spx_status|void|const char \*)\s*(spx_\w+)\s*\(", hdr, re.M))
    assert declared, "no declarations parsed"
    lib = ctypes.CDLL(spx.LIB_PATH)
    missing = [d for d in sorted(declared) if not hasattr(lib, d)]
    assert not missing, missing
    assert declared <= set(spx.EXPORTS)
