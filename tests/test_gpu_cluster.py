"""GPU tests of the cell-clustered point table (spx_cluster_points).

The clustered copy must be a permutation of the table, grouped by grid cell
(points outside the box last), and the count-only aggregate over it must equal
the aggregate over the original table and the oracle's counts, byte for byte.
The join, the selection and the server must refuse it.
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


class _DevView:
    """A (n, 2) int32 device array given by address, for torch.as_tensor."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n, 2), "typestr": "<i4", "data": (ptr, False), "version": 3}


def _keys(xy, c):
    x, y = xy[:, 0].astype(np.int64), xy[:, 1].astype(np.int64)
    inside = (x >= 0) & (x < (1 << 30)) & (y >= 0) & (y < (1 << 30))
    sh = 30 - c
    k = ((y >> sh) << c) | (x >> sh)
    return np.where(inside, k, 1 << (2 * c))


@pytest.mark.parametrize("c", [12, 7, 1])
def test_cluster_is_grouped_permutation_with_same_counts(eng, c):
    seed = g.SEED_BASE + 70
    mix = g.make_mixture(seed, zipf_s=1.1)
    pts = g.mixture_points(3_000_000 + 4321, seed, mix)
    # a few points outside the box (a borrowed device table is not validated)
    bad = np.array([[-1, 5], [1 << 30, 7], [3, -2], [2**31 - 1, 2**31 - 1]], np.int32)
    pts = np.concatenate([pts[:1000], bad, pts[1000:]])
    t = g.quad_tessellation(16, 12, seed, kmin=4, kmax=60)
    v, o = t.verts, t.ring_off
    P = o.shape[0] - 1
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    ph = eng.load_points(dpts)
    ch = eng.cluster_points(ph, c)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh)
    try:
        info = eng.points_info(ch)
        assert info["n"] == pts.shape[0] and info["cluster_log2"] == c and info["ptr"]
        clus = torch.as_tensor(_DevView(info["ptr"], info["n"]), device="cuda").cpu().numpy().copy()
        # a permutation of the table
        a = pts[np.lexsort((pts[:, 1], pts[:, 0]))]
        b = clus[np.lexsort((clus[:, 1], clus[:, 0]))]
        assert np.array_equal(a, b)
        # grouped by cell, row-major, outside points last
        k = _keys(clus, c)
        assert np.all(np.diff(k) >= 0)
        assert np.array_equal(np.bincount(k, minlength=(1 << (2 * c)) + 1),
                              np.bincount(_keys(pts, c), minlength=(1 << (2 * c)) + 1))
        # the same counts as the original table and as the oracle
        c1 = torch.zeros(P, dtype=torch.int64, device="cuda")
        c2 = torch.zeros(P, dtype=torch.int64, device="cuda")
        eng.aggregate(ph, ih, c1)
        eng.aggregate(ch, ih, c2)
        torch.cuda.synchronize()
        ref = oracle.Prepared(v, o)
        want = ref.counts(pts)
        ref.close()
        assert np.array_equal(c1.cpu().numpy().view(np.uint64), want)
        assert np.array_equal(c2.cpu().numpy().view(np.uint64), want)
    finally:
        eng.free(ih)
        eng.free(gh)
        eng.free(ch)
        eng.free(ph)
        del dpts


def test_cluster_refused_where_row_order_matters(eng):
    pts = g.uniform_points(50_000, g.SEED_BASE + 71)
    ph = eng.load_points(pts)
    ch = eng.cluster_points(ph)
    v, o = g.star_polygons(g.SEED_BASE + 71)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh)
    try:
        assert eng.points_info(ch)["cluster_log2"] == 12
        pairs = torch.empty((100_000, 2), dtype=torch.int32, device="cuda")
        with pytest.raises(spx.SpxError) as ei:
            eng.join(ch, ih, pairs)
        assert ei.value.status == spx.SPX_EINVAL
        ids = torch.empty(100_000, dtype=torch.int32, device="cuda")
        offs = torch.zeros(257, dtype=torch.int64, device="cuda")
        with pytest.raises(spx.SpxError) as ei:
            eng.select(ch, ih, ids, offs)
        assert ei.value.status == spx.SPX_EINVAL
        with pytest.raises(spx.SpxError):
            spx.Server(eng, ch, [ih])
        with pytest.raises(spx.SpxError):
            eng.cluster_points(ph, 14)
        # an empty table clusters to an empty table
        e0 = eng.load_points(np.zeros((0, 2), np.int32))
        e1 = eng.cluster_points(e0, 5)
        assert eng.points_info(e1)["n"] == 0
        eng.free(e1)
        eng.free(e0)
    finally:
        eng.free(ih)
        eng.free(gh)
        eng.free(ch)
        eng.free(ph)


@pytest.mark.parametrize("c,gl", [(13, 13), (13, 11), (12, 12), (12, 9), (10, 6), (8, 8), (6, 9)])
def test_aggregate_through_the_cell_directory(eng, c, gl):
    # with the clustering grid at least as fine as the coarse grid (c >= g),
    # cells in coarse cells INSIDE one polygon are counted from the directory
    # without reading their points; the result must stay the oracle's, and
    # every point must be accounted as scanned once (c < g: the plain path)
    seed = g.SEED_BASE + 72
    mix = g.make_mixture(seed)
    pts = g.mixture_points(2_000_003, seed, mix)
    bad = np.array([[-1, 5], [1 << 30, 7], [3, -2]], np.int32)
    pts = np.concatenate([bad, pts])
    cases = [g.quad_tessellation(12, 10, seed, kmin=4, kmax=80), g.star_polygons(seed)]
    for case in cases:
        v, o = (case.verts, case.ring_off) if hasattr(case, "verts") else case
        P = o.shape[0] - 1
        ref = oracle.Prepared(v, o)
        want = ref.counts(pts)
        ref.close()
        dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
        ph = eng.load_points(dpts)
        ch = eng.cluster_points(ph, c)
        gh = eng.load_polygons(v, o)
        try:
            for fp32 in (True, False):
                ih = eng.build_index(gh, grid_log2=gl, fp32_filter=fp32)
                counts = torch.full((P,), 5, dtype=torch.int64, device="cuda")
                eng.stats(reset=True)
                eng.aggregate(ch, ih, counts)
                torch.cuda.synchronize()
                st = eng.stats(reset=True)
                assert np.array_equal(counts.cpu().numpy().view(np.uint64), want), (c, gl, fp32)
                assert st["points_scanned"] == pts.shape[0]
                eng.free(ih)
        finally:
            eng.free(gh)
            eng.free(ch)
            eng.free(ph)
            del dpts
