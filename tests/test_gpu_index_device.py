"""The polygon grid index built on the device (spx_build_index_device) against
the host build, byte for byte, and joins through it against the oracle.

The device build runs every stage of the host build as kernels (conservative
marks, corner-row parities, sorted fine-row edge lists, the merge by cell), so
its coarse words, fine blocks, entries and edges must be exactly the host's:
for the families the host build is checked on (star polygons, a noisy
tessellation, overlapping query polygons, rings on power-of-two grid lines),
at grids 1-13 and subdivisions 1-3; for degenerate rings, horizontal edges on
row borders, rings touching the box's far borders, an empty set; and for the
benchmark's 2000-cell tessellation at its default grid.
"""
import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import datagen as g

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_14362_gb300 import spx  # noqa: E402
from test_index_host import scaled_tiny  # noqa: E402


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = spx.Engine(0)
    yield e
    e.close()


def family(name):
    if name == "stars":
        return g.star_polygons(g.SEED_BASE + 1)
    if name == "tess":
        t = g.quad_tessellation(7, 6, 11, kmin=3, kmax=60)
        return t.verts, t.ring_off
    if name == "queries":
        mix = g.make_mixture(21)
        return g.query_polygons(24, 21, mix, vmax=600, r_med=0.05)
    if name == "grid_aligned":
        v, o, _ = scaled_tiny()
        return v, o
    if name == "edge_cases":
        B = 1 << 30
        rings = [
            [(0, 0), (B, 0), (B, B // 3)],                              # touches the far border
            [(B - 5, B - 5), (B, B - 5), (B, B), (B - 5, B)],           # a corner square at the box's far corner
            [(1 << 20, 1 << 20), (3 << 20, 1 << 20)],                   # two vertices: nothing inside
            [(7 << 22, 7 << 22), (9 << 22, 7 << 22), (9 << 22, 7 << 22)],  # zero area
            [(1 << 24, 1 << 24), (5 << 24, 1 << 24), (5 << 24, 3 << 24), (3 << 24, 3 << 24),
             (3 << 24, 5 << 24), (1 << 24, 5 << 24)],                  # horizontal edges on row borders
            [(10 << 24, 10 << 24), (20 << 24, 10 << 24), (10 << 24, 20 << 24), (20 << 24, 20 << 24)],  # bow tie
            [(30 << 24, 30 << 24)] * 4,                                 # one repeated vertex
        ]
        v = np.concatenate([np.array(r, np.int64) for r in rings]).astype(np.int32)
        o = np.zeros(len(rings) + 1, np.uint64)
        o[1:] = np.cumsum([len(r) for r in rings])
        return v, o
    raise KeyError(name)


def both(eng, v, o, gl, sb):
    """Arrays and info of the host-built and the device-built index; when the
    host build refuses (a limit of the index format), the device build must
    refuse with the same message, and both are None."""
    gh = eng.load_polygons(v, o)
    try:
        try:
            ih = eng.build_index(gh, grid_log2=gl, sub_log2=sb)
        except spx.SpxError as err:
            with pytest.raises(spx.SpxError) as ei:
                eng.build_index(gh, grid_log2=gl, sub_log2=sb, on_device=True)
            assert ei.value.status == err.status
            assert str(err).split("build_index: ")[-1] == str(ei.value).split("build_index_device: ")[-1]
            return None
        idv = eng.build_index(gh, grid_log2=gl, sub_log2=sb, on_device=True)
        a, b = eng.index_arrays(ih), eng.index_arrays(idv)
        ia, ib = eng.index_info(ih), eng.index_info(idv)
        eng.free(ih)
        eng.free(idv)
        return a, b, ia, ib
    finally:
        eng.free(gh)


def assert_same(a, b, ia, ib, what):
    for k in ("coarse", "fine", "entries", "edges"):
        assert a[k].shape == b[k].shape, f"{what}: {k} sizes {a[k].shape} vs {b[k].shape}"
        assert np.array_equal(a[k], b[k]), f"{what}: {k} differ"
    for k in ("n_blocks", "n_entries", "n_inside", "n_mixed", "n_boundary", "n_edge_refs", "device_bytes",
              "use_sum"):
        assert ia[k] == ib[k], f"{what}: {k} {ia[k]} vs {ib[k]}"
    assert abs(ia["sum_resolved"] - ib["sum_resolved"]) < 1e-12


@pytest.mark.parametrize("name", ["stars", "tess", "queries", "grid_aligned", "edge_cases"])
@pytest.mark.parametrize("gl,sb", [(1, 1), (3, 3), (5, 2), (6, 1), (8, 3), (9, 2), (11, 3), (13, 3)])
def test_device_index_equals_host_index(eng, name, gl, sb):
    v, o = family(name)
    r = both(eng, v, o, gl, sb)
    if r is None:  # both builds refused the same index-format limit (a box-covering polygon at g = 13)
        assert name == "grid_aligned" and gl == 13
        return
    a, b, ia, ib = r
    assert_same(a, b, ia, ib, f"{name} g={gl} sub={sb}")
    # and the host-only build (spx_host_index_build) is the same bytes too
    h = spx.host_index(v, o, gl, sb)
    for k in ("coarse", "fine", "entries", "edges"):
        assert np.array_equal(h[k], b[k]), f"{name} g={gl} sub={sb}: {k} differ from the host-only build"


def test_empty_polygon_set(eng):
    v = np.zeros((0, 2), np.int32)
    o = np.zeros(1, np.uint64)
    a, b, ia, ib = both(eng, v, o, 4, 2)
    assert_same(a, b, ia, ib, "empty set")
    assert not b["coarse"].any()


def test_benchmark_tessellation_and_join(eng):
    # the 2000-cell tessellation at its default grid; a join through the
    # device-built index equals the oracle
    nx, ny = g.tessellation_shape(2000)
    t = g.quad_tessellation(nx, ny, g.SEED_BASE + 2, kmin=12, kmax=499)
    a, b, ia, ib = both(eng, t.verts, t.ring_off, 11, 3)
    assert_same(a, b, ia, ib, "tess2000 g=11 sub=3")
    pts = g.mixture_points(400_000, g.SEED_BASE + 2)
    want_p, want_c = oracle.join_fast(pts, t.verts, t.ring_off)
    dpts = torch.from_numpy(pts).cuda()
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(t.verts, t.ring_off)
    ih = eng.build_index(gh, grid_log2=11, sub_log2=3, on_device=True)
    pairs = torch.full((pts.shape[0] + 8, 2), -1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(t.ring_off.shape[0] - 1, dtype=torch.int64, device="cuda")
    n = eng.join(ph, ih, pairs, counts)
    assert n == want_p.shape[0]
    assert np.array_equal(pairs[:n].cpu().numpy().view(np.uint32), want_p)
    assert np.array_equal(counts.cpu().numpy().view(np.uint64), want_c)
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    del dpts


def test_bad_parameters(eng):
    v, o = family("stars")
    gh = eng.load_polygons(v, o)
    for gl, sb in ((14, 1), (13, 4), (12, 5)):
        with pytest.raises(spx.SpxError) as ei:
            eng.build_index(gh, grid_log2=gl, sub_log2=sb, on_device=True)
        assert ei.value.status == spx.SPX_EINVAL
    eng.free(gh)
