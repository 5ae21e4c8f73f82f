"""The join's per-point results at both widths, on both sides of the limit.

Between its passes the join keeps one result per point: a 16-bit word when
the index has at most 65534 polygons (a polygon id, none, or, for a point in
several polygons, their number, told apart by the row bitmap of the first
pass), else a 32-bit word.  SPADE's join (§5.1 "Spatial Joins") emits every
(point, polygon) pair, so both widths must give the oracle's pairs and counts
byte for byte, also for points that lie in two or three polygons.

The polygon sets: a 252 x 260 quad tessellation (65520 cells) followed by 14
or 15 overlapping axis-parallel rectangles, 65534 polygons (the widest narrow
case) or 65535 (the first wide one).  Every point inside a rectangle is also in
a tessellation cell; where rectangles overlap, a point is in three polygons.
"""
import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import datagen as g

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_14362_gb300 import spx  # noqa: E402

NARROW_MAX_P = 65534


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = spx.Engine(0)
    yield e
    e.close()


@pytest.fixture(scope="module")
def base():
    t = g.quad_tessellation(252, 260, g.SEED_BASE + 41, kmin=2, kmax=6)
    mix = g.make_mixture(g.SEED_BASE + 41)
    pts = g.mixture_points_parallel(1_500_007, g.SEED_BASE + 41, mix)
    return t, pts


def with_rectangles(t, k):
    """The tessellation's rings, then k rectangles, rectangle r of 2^27 x
    (2^27 + r 2^22) box units; neighbours are 3/8 of a side apart in x and half
    a side in y, so they overlap."""
    rings = []
    for r in range(k):
        x0 = (1 << 25) + r * (3 << 24)
        y0 = (1 << 26) + (r % 3) * (1 << 26)
        x1, y1 = x0 + (1 << 27), y0 + (1 << 27) + r * (1 << 22)
        rings.append([(x0, y0), (x1, y0), (x1, y1), (x0, y1)])
    v = np.concatenate([t.verts] + [np.array(rg, np.int32) for rg in rings])
    o = np.concatenate([t.ring_off, t.ring_off[-1] + 4 * np.arange(1, k + 1, dtype=np.uint64)])
    return v, o


@pytest.mark.parametrize("k", [14, 15])
@pytest.mark.parametrize("gl", [10, 11])
def test_result_width_limit(eng, base, k, gl):
    t, pts = base
    v, o = with_rectangles(t, k)
    P = o.shape[0] - 1
    assert P == NARROW_MAX_P + (k - 14)
    want_pairs, want_counts = oracle.join_fast(pts, v, o)
    multi = np.bincount(want_pairs[:, 0], minlength=pts.shape[0])
    assert (multi >= 2).sum() > 1000 and (multi >= 3).sum() > 100  # the several-polygon rows are exercised
    dpts = torch.from_numpy(pts).cuda()
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=gl)
    cap = want_pairs.shape[0] + 16
    for rep in range(2):  # the second call runs on the scratch the first left
        pairs = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
        counts = torch.zeros(P, dtype=torch.int64, device="cuda")
        n = eng.join(ph, ih, pairs, counts)
        assert n == want_pairs.shape[0]
        got = pairs.cpu().numpy()
        assert np.array_equal(got[:n].view(np.uint32), want_pairs), f"P={P} g={gl} call {rep}"
        assert (got[n:] == -1).all()
        assert np.array_equal(counts.cpu().numpy().view(np.uint64), want_counts)
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    del dpts
