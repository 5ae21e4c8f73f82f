"""GPU parity of batched selection (spx_select) against the oracle, bit for bit.

Each query polygon's list must hold exactly the oracle's point ids, ascending;
the offsets must match the oracle's per-query counts.  Repeated calls replay a
captured CUDA graph and must give the same bytes.  Cases: overlapping query
polygons (points in several queries), disjoint stars, polygons with vertices
on grid lines, ragged sizes, an overflowing capacity, too many queries.
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


def run_select(eng, pts, v, o, gl=0, reps=1, cap=None):
    P = o.shape[0] - 1
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()  # borrowed by the handle
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=gl)
    cap = 4 * pts.shape[0] + 8 if cap is None else cap
    ids = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    offs = torch.zeros(P + 1, dtype=torch.int64, device="cuda")
    outs = []
    try:
        for _ in range(reps):
            ids.fill_(-1)
            n = eng.select(ph, ih, ids, offs)
            outs.append((ids[:min(n, cap)].cpu().numpy().view(np.uint32).copy(),
                         offs.cpu().numpy().view(np.uint64).copy(), n))
    finally:
        eng.free(ih)
        eng.free(gh)
        eng.free(ph)
        del dpts
    return outs


def oracle_select(pts, v, o):
    pr = oracle.Prepared(v, o)
    ids, offs = pr.select(pts)
    pr.close()
    return ids, offs


@pytest.mark.parametrize("gl", [0, 7, 10])
def test_overlapping_queries(eng, gl):
    mix = g.make_mixture(17)
    v, o = g.query_polygons(96, 17, mix, vmax=2500, r_med=0.03)
    pts = g.mixture_points(300_001, 17, mix)
    want_ids, want_off = oracle_select(pts, v, o)
    assert want_ids.shape[0] > pts.shape[0] * 0.05
    for got_ids, got_off, n in run_select(eng, pts, v, o, gl, reps=3):
        assert n == want_ids.shape[0]
        assert np.array_equal(got_off, want_off)
        assert np.array_equal(got_ids, want_ids)


def test_disjoint_stars_ragged(eng):
    v, o = g.star_polygons(g.SEED_BASE + 1)
    for n in (1, 32767, 32769, 100_003):
        pts = g.uniform_points(n, n)
        want_ids, want_off = oracle_select(pts, v, o)
        got_ids, got_off, m = run_select(eng, pts, v, o, 8)[0]
        assert m == want_ids.shape[0] and np.array_equal(got_off, want_off) and np.array_equal(got_ids, want_ids)


def test_grid_aligned_overlaps(eng):
    s = 1 << 26
    rings = [[(2, 2), (10, 2), (10, 9), (2, 9)], [(0, 0), (8, 0), (0, 8)], [(3, 3), (12, 12), (12, 3), (3, 12)],
             [(0, 0), (16, 0), (16, 16), (0, 16)], [(5, 0), (10, 5), (5, 10), (0, 5)]]
    v = np.concatenate([np.array(r, np.int64) * s for r in rings]).astype(np.int32)
    o = np.zeros(len(rings) + 1, np.uint64)
    o[1:] = np.cumsum([len(r) for r in rings])
    pts = np.array([(x * s + dx, y * s + dy) for x in range(16) for y in range(16)
                    for dx in (-1, 0, 1) for dy in (-1, 0, 1)], dtype=np.int64)
    pts = pts[(pts >= 0).all(1) & (pts < (1 << 30)).all(1)].astype(np.int32)
    want_ids, want_off = oracle_select(pts, v, o)
    for gl in (2, 4, 9):
        got_ids, got_off, n = run_select(eng, pts, v, o, gl)[0]
        assert n == want_ids.shape[0] and np.array_equal(got_off, want_off) and np.array_equal(got_ids, want_ids)


def test_capacity_and_limits(eng):
    mix = g.make_mixture(23)
    v, o = g.query_polygons(16, 23, mix, vmax=200, r_med=0.05)
    pts = g.mixture_points(50_000, 23, mix)
    want_ids, _ = oracle_select(pts, v, o)
    with pytest.raises(spx.SpxError) as ei:
        run_select(eng, pts, v, o, 8, cap=10)
    assert ei.value.status == spx.SPX_ECAPACITY and str(want_ids.shape[0]) in str(ei.value)
    # more query polygons than one batched selection takes
    rings = [g.rect_polygon(10 * k, 10, 10 * k + 5, 20) for k in range(1025)]
    rv = np.concatenate(rings)
    ro = np.arange(0, 4 * 1026, 4, dtype=np.uint64)
    with pytest.raises(spx.SpxError) as ei:
        run_select(eng, pts, rv, ro, 8)
    assert ei.value.status == spx.SPX_EINVAL
