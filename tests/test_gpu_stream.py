"""GPU tests of host tables streamed through the device (spx_join_host in
streamed mode, spx_aggregate_host).

Small slices (2^16 points) make a 1M-point table run through the four-slot
ring many times; results must equal the oracle byte for byte, with pairs
written straight into pageable or pinned host memory.
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


@pytest.fixture(scope="module")
def data():
    seed = g.SEED_BASE + 90
    mix = g.make_mixture(seed)
    pts = g.mixture_points(1_000_000 + 12_345, seed, mix)
    v, o = g.query_polygons(30, seed, mix, r_med=0.05, r_clip=(0.01, 0.2))
    ref = oracle.Prepared(v, o)
    want_p, want_c = ref.join(pts)
    ref.close()
    assert np.any(np.bincount(want_p[:, 0].astype(np.int64)) > 1)  # overlapping queries
    return pts, v, o, want_p, want_c


@pytest.mark.parametrize("mode,pinned", [(2, False), (2, True), (1, False)])
def test_join_host_modes(eng, data, mode, pinned):
    pts, v, o, want_p, want_c = data
    P = o.shape[0] - 1
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh)
    eng.set_host_streaming(mode, 16)
    try:
        cap = want_p.shape[0] + 3
        hp = torch.empty((cap, 2), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32) if pinned else None
        p, c, n = eng.join_host(pts, ih, cap=cap, n_polys=P, pairs_out=hp)
        assert n == want_p.shape[0]
        assert np.array_equal(p, want_p) and np.array_equal(c, want_c)
        # capacity runs out part-way: the first cap pairs, then SPX_ECAPACITY with the total
        small = want_p.shape[0] // 3
        buf = np.zeros((small, 2), np.uint32)
        with pytest.raises(spx.SpxError) as ei:
            eng.join_host(pts, ih, cap=small, n_polys=P, pairs_out=buf)
        assert ei.value.status == spx.SPX_ECAPACITY and str(want_p.shape[0]) in str(ei.value)
        assert np.array_equal(buf, want_p[:small])
    finally:
        eng.set_host_streaming(0, 0)
        eng.free(ih)
        eng.free(gh)


def test_aggregate_host(eng, data):
    pts, v, o, _, want_c = data
    P = o.shape[0] - 1
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh)
    try:
        eng.set_host_streaming(0, 16)
        assert np.array_equal(eng.aggregate_host(pts, ih, P), want_c)
        eng.set_host_streaming(0, 0)  # one slice of 2^23 holds the whole table
        assert np.array_equal(eng.aggregate_host(pts, ih, P), want_c)
        assert not eng.aggregate_host(np.zeros((0, 2), np.int32), ih, P).any()
        with pytest.raises(spx.SpxError):
            eng.set_host_streaming(3, 0)
        with pytest.raises(spx.SpxError):
            eng.set_host_streaming(0, 15)
    finally:
        eng.set_host_streaming(0, 0)
        eng.free(ih)
        eng.free(gh)
