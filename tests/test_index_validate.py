"""The index validator (spx_host_index_validate), on the CPU.

The kernels of a SPX_BOUNDS_CHECK build apply the same predicate to every
offset they read from an index; spx_build_index applies it to every index
before upload.  A valid index passes; a truncated or corrupted one fails with
a message naming the first violation: edges cut off, a fine word pointing past
the entries, a polygon id past the polygon set, a coarse word naming a fine
block that does not exist, a list without its last-entry flag, missing
sentinels.
"""
import numpy as np
import pytest

from paper_2203_14362_gb300 import datagen as g
from paper_2203_14362_gb300 import spx

MASK = (1 << 30) - 1


@pytest.fixture(scope="module")
def index():
    t = g.quad_tessellation(7, 6, 11, kmin=3, kmax=60)
    P = t.ring_off.shape[0] - 1
    return spx.host_index(t.verts, t.ring_off, 8, 3), P


def copy(ix):
    return {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in ix.items()}


def test_valid_index_passes(index):
    ix, P = index
    ok, msg = spx.validate_index(ix, P)
    assert ok, msg
    for name in ("stars", "queries"):
        if name == "stars":
            v, o = g.star_polygons(g.SEED_BASE + 1)
        else:
            v, o = g.query_polygons(24, 21, g.make_mixture(21), vmax=600, r_med=0.05)
        for gl, sb in ((3, 1), (9, 3)):
            ok, msg = spx.validate_index(spx.host_index(v, o, gl, sb), o.shape[0] - 1)
            assert ok, (name, gl, sb, msg)


def test_truncated_edges_fail(index):
    ix, P = index
    bad = copy(ix)
    bad["edges"] = np.concatenate([bad["edges"][:-41], np.zeros((1, 4), np.int32)])  # 40 edges cut, sentinel kept
    ok, msg = spx.validate_index(bad, P)
    assert not ok and "past the edge array" in msg


def test_fine_word_past_the_entries_fails(index):
    ix, P = index
    bad = copy(ix)
    f = np.nonzero((bad["fine"] >> 30) == 2)[0][0]
    bad["fine"][f] = (2 << 30) | (bad["entries"].shape[0] - 2)  # points into the sentinels
    ok, msg = spx.validate_index(bad, P)
    assert not ok and "runs past the entries" in msg


def test_polygon_id_past_the_set_fails(index):
    ix, P = index
    bad = copy(ix)
    c = np.nonzero((bad["coarse"] >> 30) == 1)[0][0]
    bad["coarse"][c] = (1 << 30) | P
    ok, msg = spx.validate_index(bad, P)
    assert not ok and "names polygon" in msg
    ok, _ = spx.validate_index(ix, P - 1)  # the same index against a smaller set
    assert not ok


def test_missing_block_or_last_flag_fails(index):
    ix, P = index
    bad = copy(ix)
    c = np.nonzero((bad["coarse"] >> 30) == 2)[0][0]
    bad["coarse"][c] = (2 << 30) | (bad["fine"].shape[0] // 64)  # one block past the fine level
    ok, msg = spx.validate_index(bad, P)
    assert not ok and "fine block" in msg
    bad = copy(ix)
    bad["entries"][:-4, 3] &= ~np.uint32(2)  # no list ends
    ok, msg = spx.validate_index(bad, P)
    assert not ok and "runs past the entries" in msg


def test_missing_sentinels_fail(index):
    ix, P = index
    bad = copy(ix)
    bad["entries"] = bad["entries"][:-4]
    ok, msg = spx.validate_index(bad, P)
    assert not ok and "sentinel" in msg
    bad = copy(ix)
    bad["edges"] = bad["edges"][:-1]
    ok, msg = spx.validate_index(bad, P)
    assert not ok
