"""GPU edge cases across the C ABI: empty tables, counts-only calls, a single
query covering the box, and the autotuner over a clustered copy."""
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


def test_host_join_empty_and_counts_only(eng):
    v, o = g.star_polygons(g.SEED_BASE + 80)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=8)
    try:
        p, c, n = eng.join_host(np.zeros((0, 2), np.int32), ih, cap=0, n_polys=256)
        assert n == 0 and p.shape[0] == 0 and not c.any()
        pts = g.uniform_points(300_001, g.SEED_BASE + 80)
        want_p, want_c = oracle.join_fast(pts, v, o)
        # capacity 0: the total and the counts come back, no pairs
        with pytest.raises(spx.SpxError) as ei:
            eng.join_host(pts, ih, cap=0, n_polys=256)
        assert ei.value.status == spx.SPX_ECAPACITY and str(want_p.shape[0]) in str(ei.value)
        counts = np.zeros(256, np.uint64)
        with pytest.raises(spx.SpxError):
            eng.join_host(pts, ih, cap=0, n_polys=256, counts_out=counts)
        assert np.array_equal(counts, want_c)
    finally:
        eng.free(ih)
        eng.free(gh)


def test_aggregate_and_select_on_empty_table(eng):
    v, o = g.star_polygons(g.SEED_BASE + 81)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=6)
    ph = eng.load_points(np.zeros((0, 2), np.int32))
    try:
        counts = torch.full((256,), 7, dtype=torch.int64, device="cuda")
        eng.aggregate(ph, ih, counts)
        torch.cuda.synchronize()
        assert not counts.any()
        ids = torch.empty(1, dtype=torch.int32, device="cuda")
        offs = torch.full((257,), 5, dtype=torch.int64, device="cuda")
        assert eng.select(ph, ih, ids, offs) == 0
        assert not offs.any()
    finally:
        eng.free(ph)
        eng.free(ih)
        eng.free(gh)


def test_server_on_empty_table(eng):
    v, o = g.star_polygons(g.SEED_BASE + 82)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh)
    ph = eng.load_points(np.zeros((0, 2), np.int32))
    srv = spx.Server(eng, ph, [ih])
    try:
        for kind in (spx.SPX_REQ_JOIN, spx.SPX_REQ_SELECT):
            rid = srv.submit(kind, 0)
            res = srv.wait(rid, 30_000)
            assert res is not None and res["status"] == spx.SPX_OK and res["total"] == 0
            a, b = srv.read(rid, res)
            assert a.shape[0] == 0 and not b.any()
            srv.release(rid)
    finally:
        srv.close()
        eng.free(ph)
        eng.free(ih)
        eng.free(gh)


def test_select_one_query_covering_the_box(eng):
    box = 1 << 30
    v = np.array([[0, 0], [box, 0], [box, box], [0, box]], np.int32)
    o = np.array([0, 4], np.uint64)
    pts = g.mixture_points(200_003, g.SEED_BASE + 83)
    ph = eng.load_points(pts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=4)
    try:
        ids = torch.empty(pts.shape[0], dtype=torch.int32, device="cuda")
        offs = torch.zeros(2, dtype=torch.int64, device="cuda")
        n = eng.select(ph, ih, ids, offs)
        assert n == pts.shape[0]
        assert np.array_equal(ids.cpu().numpy(), np.arange(pts.shape[0], dtype=np.int32))
        assert offs.cpu().tolist() == [0, pts.shape[0]]
    finally:
        eng.free(ih)
        eng.free(gh)
        eng.free(ph)


def test_autotune_on_clustered_table(eng):
    t = g.quad_tessellation(10, 10, g.SEED_BASE + 84, kmin=4, kmax=60)
    pts = g.mixture_points(2_000_000, g.SEED_BASE + 84)
    ph = eng.load_points(pts)
    ch = eng.cluster_points(ph, 10)
    gh = eng.load_polygons(t.verts, t.ring_off)
    try:
        params, trials, ih = eng.autotune(ch, gh, grid_min=6, grid_max=10, reps=2)
        counts = torch.zeros(100, dtype=torch.int64, device="cuda")
        eng.aggregate(ch, ih, counts)
        torch.cuda.synchronize()
        ref = oracle.Prepared(t.verts, t.ring_off)
        want = ref.counts(pts)
        ref.close()
        assert np.array_equal(counts.cpu().numpy().view(np.uint64), want)
        eng.free(ih)
    finally:
        eng.free(gh)
        eng.free(ch)
        eng.free(ph)
