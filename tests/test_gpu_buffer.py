"""Buffered-polygon distance queries on the GPU against the oracle (SPADE §4.2
"Canvases for Distance-Based Queries": a polygon's distance constraint is the
polygon plus a rounded rectangle of radius r around each edge; §5.2
"Distance-Based Queries").

spx_build_buffer_index + spx_join / spx_select / spx_aggregate must give
exactly oracle.buffer_join's pairs (point, polygon), in order, and counts:
for overlapping concave query polygons with per-polygon radii (zero among
them), a tessellation (a point near a shared edge meets both cells), rings of
one vertex (disks), two vertices (capsules) and zero area, rings on the box's
edges, lattice points at exactly the radius from edges and corners, points
outside the box, several edge grids, and ragged table sizes.
"""
import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import datagen as g

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_14362_gb300 import spx  # noqa: E402


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = spx.Engine(0)
    yield e
    e.close()


def poly_set(name):
    if name == "queries":
        mix = g.make_mixture(61)
        v, o = g.query_polygons(24, 61, mix, vmax=400, r_med=0.03)
        rng = np.random.default_rng(61)
        r = rng.integers(0, 1 << 22, o.shape[0] - 1).astype(np.int32)
        r[::5] = 0
        return v, o, r, g.mixture_points(300_007, 61, mix)
    if name == "tess":
        t = g.quad_tessellation(9, 7, 62, kmin=3, kmax=30)
        r = np.full(t.ring_off.shape[0] - 1, 1 << 20, np.int32)
        return t.verts, t.ring_off, r, g.mixture_points(250_003, 62)
    if name == "degenerate":
        B = 1 << 30
        rings = [
            [(1 << 28, 1 << 28)],                                            # one vertex: a disk
            [(3 << 27, 1 << 28), (5 << 27, 3 << 28)],                        # two vertices: a capsule
            [(1 << 29, 1 << 29), (5 << 27, 5 << 27), (3 << 28, 3 << 28)],    # zero area (collinear)
            [(0, 0), (B, 0), (B, 1 << 20)],                                  # on the box's lower edge
            [(B - 5, B - 5), (B, B - 5), (B, B), (B - 5, B)],                # the box's far corner
            [(10 << 24, 10 << 24), (20 << 24, 10 << 24), (10 << 24, 20 << 24), (20 << 24, 20 << 24)],  # bow tie
        ]
        v = np.concatenate([np.array(x, np.int64) for x in rings]).astype(np.int32)
        o = np.zeros(len(rings) + 1, np.uint64)
        o[1:] = np.cumsum([len(x) for x in rings])
        r = np.array([1 << 24, 1 << 23, 1 << 22, 1 << 21, 7, 1 << 22], np.int32)
        pts = g.uniform_points(200_001, 63)
        pts[:4] = [[-1, 5], [5, -7], [B, 3], [3, B]]  # outside the box: no pairs
        return v, o, r, pts
    if name == "lattice":
        # a square and a triangle on a coarse lattice, points on the same
        # lattice: many points lie exactly r from an edge or a corner
        S = 1 << 16
        rings = [np.array([[100, 100], [130, 100], [130, 125], [100, 125]]) * S,
                 np.array([[200, 150], [260, 150], [200, 230]]) * S]
        v = np.concatenate(rings).astype(np.int32)
        o = np.array([0, 4, 7], np.uint64)
        r = np.array([5 * S, 13 * S], np.int32)  # 3-4-5 and 5-12-13 distances occur exactly
        rng = np.random.default_rng(64)
        pts = (rng.integers(80, 280, (150_001, 2)) * S + rng.integers(-1, 2, (150_001, 2))).astype(np.int32)
        return v, o, r, pts
    raise KeyError(name)


def run_join(eng, pts, v, o, r, gl):
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_buffer_index(gh, r, grid_log2=gl)
    P = o.shape[0] - 1
    want_p, want_c = oracle.buffer_join(pts, v, o, r)
    pairs = torch.full((want_p.shape[0] + 64, 2), -1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(max(P, 1), dtype=torch.int64, device="cuda")
    n = eng.join(ph, ih, pairs, counts)
    got = pairs.cpu().numpy()
    info = eng.index_info(ih)
    return dict(eng=eng, dpts=dpts, ph=ph, gh=gh, ih=ih, n=n, got=got, counts=counts.cpu().numpy()[:P],
                want_p=want_p, want_c=want_c, info=info, P=P)


def free(d):
    d["eng"].free(d["ih"])
    d["eng"].free(d["gh"])
    d["eng"].free(d["ph"])


@pytest.mark.parametrize("name", ["queries", "tess", "degenerate", "lattice"])
@pytest.mark.parametrize("gl", [0, 6, 10, 12])
def test_buffer_join_equals_oracle(eng, name, gl):
    v, o, r, pts = poly_set(name)
    d = run_join(eng, pts, v, o, r, gl)
    try:
        assert d["info"]["edge_grid_log2"] == (gl or d["info"]["edge_grid_log2"]) and d["info"]["n_edge_items"] > 0
        assert d["n"] == d["want_p"].shape[0]
        assert np.array_equal(d["got"][:d["n"]].view(np.uint32), d["want_p"])
        assert (d["got"][d["n"]:] == -1).all()
        assert np.array_equal(d["counts"].view(np.uint64), d["want_c"])
    finally:
        free(d)


def test_buffer_zero_radius_adds_on_edge_points(eng):
    # r = 0: the plain join's pairs plus the points lying on an edge
    v, o, _, pts = poly_set("lattice")
    pts = (pts // (1 << 16)) * (1 << 16)  # exactly on the lattice
    r = np.zeros(2, np.int32)
    d = run_join(eng, pts, v, o, r, 0)
    try:
        plain, _ = oracle.join_fast(pts, v, o)
        got = {tuple(x) for x in d["got"][:d["n"]].view(np.uint32).tolist()}
        assert {tuple(x) for x in plain.tolist()} <= got and len(got) > plain.shape[0]
        assert np.array_equal(d["got"][:d["n"]].view(np.uint32), d["want_p"])
    finally:
        free(d)


def test_buffer_select_and_aggregate(eng):
    v, o, r, pts = poly_set("queries")
    dpts = torch.from_numpy(pts).cuda()
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_buffer_index(gh, r)
    P = o.shape[0] - 1
    want_p, want_c = oracle.buffer_join(pts, v, o, r)
    want_ids, want_off = oracle.group_by_polygon(want_p, want_c)
    ids = torch.full((want_ids.shape[0] + 16,), -1, dtype=torch.int32, device="cuda")
    offs = torch.zeros(P + 1, dtype=torch.int64, device="cuda")
    n = eng.select(ph, ih, ids, offs)
    assert n == want_ids.shape[0]
    assert np.array_equal(ids.cpu().numpy()[:n].view(np.uint32), want_ids)
    assert np.array_equal(offs.cpu().numpy().view(np.uint64), want_off)
    counts = torch.full((P,), 5, dtype=torch.int64, device="cuda")
    eng.aggregate(ph, ih, counts)
    assert np.array_equal(counts.cpu().numpy().view(np.uint64), want_c)
    # over capacity: the required total, nothing written past cap
    small = torch.full((10, 2), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(spx.SpxError) as ei:
        eng.join(ph, ih, small[:4], None)
    assert ei.value.status == spx.SPX_ECAPACITY
    assert (small[4:] == -1).all()
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    del dpts


def test_buffer_bad_parameters(eng):
    v, o, r, _ = poly_set("tess")
    gh = eng.load_polygons(v, o)
    bad = r.copy()
    bad[3] = 1 << 30
    for rr, gl in ((bad, 0), (r, 13), (r, -1)):
        with pytest.raises(spx.SpxError) as ei:
            eng.build_buffer_index(gh, rr, grid_log2=gl)
        assert ei.value.status == spx.SPX_EINVAL
    ih = eng.build_buffer_index(gh, r)
    # calls that take only polygon indexes refuse it
    with pytest.raises(spx.SpxError):
        eng.index_arrays(ih)
    eng.free(ih)
    eng.free(gh)
