"""GPU parity of the counting path for more polygons than the shared-memory
histogram holds (more than 11776): per-polygon counts go to global memory with
warp-aggregated atomics, in the join and in the count-only aggregate (SPADE
§5.2 "Spatial Aggregations": aggregation without materialising the join).

Two polygon sets, both compared with the oracle byte for byte:
* a 120 x 100 tessellation (12000 cells, few vertices per cell) over 2M
  mixture points, at two grids, with the FP32 filter on and off;
* the 40000-cell tessellation of the count workload (200 x 200 cells,
  15-8784 vertices per cell, 55.8M vertices; its Zipf-weighted mixture) over
  3M points taken from the middle of that workload's table, at the grid the
  benchmark runs (g = 12, sub = 3) and a coarser one, so that the per-row edge
  lists reach the lengths the count workload walks.
Each set is checked through spx_aggregate on the row-order table, spx_aggregate
on the cell-clustered copy, and spx_join (pairs + counts).
"""
import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import datagen as g

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_14362_gb300 import spx  # noqa: E402

HIST_MAX = 11776  # polygons counted in shared memory; above it counts go to global memory


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = spx.Engine(0)
    yield e
    e.close()


@pytest.fixture(scope="module")
def tess12000():
    t = g.quad_tessellation(120, 100, g.SEED_BASE + 21, kmin=2, kmax=40)
    mix = g.make_mixture(g.SEED_BASE + 21)
    pts = g.mixture_points_parallel(2_000_003, g.SEED_BASE + 21, mix)
    pairs, counts = oracle.join_fast(pts, t.verts, t.ring_off)
    return pts, t.verts, t.ring_off, pairs, counts


@pytest.fixture(scope="module")
def tess40000():
    seed = g.SEED_BASE + 5
    nx, ny = g.tessellation_shape(40000)
    t = g.quad_tessellation(nx, ny, seed, kmin=2, kmax=2499)
    mix = g.make_mixture(seed, zipf_s=1.1)
    pts = g.mixture_points_parallel(3_000_001, seed, mix, start=1_234_567_891)
    pairs, counts = oracle.join_fast(pts, t.verts, t.ring_off)
    return pts, t.verts, t.ring_off, pairs, counts


def check_all_paths(eng, pts, v, o, want_pairs, want_counts, gl, sub, fp32, cluster_log2):
    P = o.shape[0] - 1
    assert P > HIST_MAX
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()  # borrowed by the handle: kept alive below
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=gl, fp32_filter=fp32, sub_log2=sub)
    try:
        # count-only aggregate, row order
        counts = torch.full((P,), 7, dtype=torch.int64, device="cuda")  # stale values must be overwritten
        eng.aggregate(ph, ih, counts)
        torch.cuda.synchronize()
        assert np.array_equal(counts.cpu().numpy().view(np.uint64), want_counts)
        # count-only aggregate over the cell-clustered copy
        pc = eng.cluster_points(ph, cluster_log2)
        counts.fill_(7)
        eng.aggregate(pc, ih, counts)
        torch.cuda.synchronize()
        assert np.array_equal(counts.cpu().numpy().view(np.uint64), want_counts)
        eng.free(pc)
        # the join: every pair, in (point, polygon) order, and the counts
        cap = pts.shape[0] + 64
        pairs = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
        counts.fill_(7)
        n = eng.join(ph, ih, pairs, counts)
        torch.cuda.synchronize()
        assert n == want_pairs.shape[0]
        assert np.array_equal(pairs[:n].cpu().numpy().view(np.uint32), want_pairs)
        assert (pairs[n:].cpu().numpy() == -1).all()
        assert np.array_equal(counts.cpu().numpy().view(np.uint64), want_counts)
    finally:
        eng.free(ih)
        eng.free(gh)
        eng.free(ph)
        del dpts


@pytest.mark.parametrize("gl,fp32", [(9, True), (11, True), (11, False)])
def test_12000_cells_counts_in_global_memory(eng, tess12000, gl, fp32):
    pts, v, o, want_pairs, want_counts = tess12000
    # the tessellation covers the box: every point in exactly one cell
    assert int(want_counts.sum()) == pts.shape[0] == want_pairs.shape[0]
    check_all_paths(eng, pts, v, o, want_pairs, want_counts, gl, 3, fp32, cluster_log2=10)


@pytest.mark.parametrize("gl,sub", [(12, 3), (10, 2)])
def test_count_workload_tessellation(eng, tess40000, gl, sub):
    pts, v, o, want_pairs, want_counts = tess40000
    assert o.shape[0] - 1 == 40000
    assert int(want_counts.sum()) == pts.shape[0] == want_pairs.shape[0]
    check_all_paths(eng, pts, v, o, want_pairs, want_counts, gl, sub, True, cluster_log2=12)
