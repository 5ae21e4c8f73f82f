"""The edge grid of the buffered-polygon index, built on the host
(spx_host_buffer_edges_build), checked on the CPU against the oracle's
distance predicate (SPADE §4.2: a polygon's distance constraint is the polygon
plus a rounded rectangle of radius r around each edge).

At sampled points, for every polygon q whose edges come within r[q] of the
point (oracle.near_ring), the point's cell must name q: either a flagged item
(q's r-region holds the whole cell) or one of q's edges that is itself within
r[q] of the point.  Every flagged item must be true at the point, every listed
edge must be an edge of q, and each cell lists its polygons in ascending
order.  Sampled points include lattice points exactly at the radius from
edges and corners.
"""
import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import datagen as g
from paper_2203_14362_gb300 import spx

FULL = np.uint32(1 << 31)


def rings_of(v, o):
    return [v[int(o[q]):int(o[q + 1])] for q in range(o.shape[0] - 1)]


def edge_set(ring):
    n = ring.shape[0]
    return {(int(ring[i, 0]), int(ring[i, 1]), int(ring[(i + 1) % n, 0]), int(ring[(i + 1) % n, 1]))
            for i in range(n)}


def poly_set(name):
    if name == "queries":
        mix = g.make_mixture(71)
        v, o = g.query_polygons(10, 71, mix, vmax=60, r_med=0.04)
        rng = np.random.default_rng(71)
        r = rng.integers(0, 1 << 23, o.shape[0] - 1).astype(np.int32)
        r[::4] = 0
        pts = np.concatenate([g.mixture_points(3000, 71, mix), g.uniform_points(1000, 72)])
        return v, o, r, pts
    if name == "lattice":
        S = 1 << 18
        rings = [np.array([[100, 100], [130, 100], [130, 125], [100, 125]]) * S,
                 np.array([[200, 150], [260, 150], [200, 230]]) * S,
                 np.array([[600, 600]]) * S,                              # a disk
                 np.array([[700, 300], [900, 420]]) * S]                  # a capsule
        v = np.concatenate(rings).astype(np.int32)
        o = np.array([0, 4, 7, 8, 10], np.uint64)
        r = np.array([5 * S, 13 * S, 25 * S, 17 * S], np.int32)
        rng = np.random.default_rng(73)
        pts = (rng.integers(60, 1000, (4000, 2)) * S).astype(np.int32)     # on the lattice: exact distances
        return v, o, r, pts
    raise KeyError(name)


@pytest.mark.parametrize("name", ["queries", "lattice"])
@pytest.mark.parametrize("gl", [0, 5, 8, 10])
def test_edge_grid_names_every_near_polygon(name, gl):
    v, o, r, pts = poly_set(name)
    e = spx.host_buffer_edges(v, o, r, grid_log2=gl)
    G = e["g"]
    assert 5 <= G <= 12 and (gl == 0 or G == gl)
    off, iq, seg = e["cell_off"], e["item_q"], e["item_seg"]
    assert off.shape[0] == (1 << (2 * G)) + 1 and off[-1] == iq.shape[0]
    rings = rings_of(v, o)
    edges = [edge_set(rg) for rg in rings]
    sh = 30 - G
    n_full = n_listed = 0
    for px, py in pts.tolist():
        c = ((py >> sh) << G) | (px >> sh)
        a, b = int(off[c]), int(off[c + 1])
        qs = iq[a:b] & ~FULL
        assert np.all(np.diff(qs.astype(np.int64)) >= 0)  # polygons ascending within the cell
        for q in range(len(rings)):
            near = oracle.near_ring(px, py, rings[q], int(r[q]))
            mine = np.nonzero(qs == q)[0] + a
            flagged = [k for k in mine if iq[k] & FULL]
            listed = [k for k in mine if not iq[k] & FULL]
            assert len(flagged) <= 1 and not (flagged and listed)
            for k in listed:
                assert tuple(int(x) for x in seg[k]) in edges[q]
            if flagged:
                assert near, f"cell {c} flagged full for polygon {q}, but ({px}, {py}) is farther than r"
                n_full += 1
            elif near:
                ok = any(oracle.near_ring(px, py, seg[k].reshape(2, 2), int(r[q])) for k in listed)
                assert ok, f"({px}, {py}) is within r of polygon {q}, but no listed edge of cell {c} is"
                n_listed += 1
    assert n_listed > 0
    if name == "lattice" and G >= 8:
        assert n_full > 0  # the radii are several cells wide: whole cells lie within r


def test_edge_grid_refusals():
    v, o, r, _ = poly_set("lattice")
    bad = r.copy()
    bad[0] = -1
    with pytest.raises(spx.SpxError):
        spx.host_buffer_edges(v, o, bad)
    with pytest.raises(spx.SpxError):
        spx.host_buffer_edges(v, o, r, grid_log2=13)
    w = v.copy()
    w[0, 0] = (1 << 30) + 1
    with pytest.raises(spx.SpxError):
        spx.host_buffer_edges(w, o, r)
