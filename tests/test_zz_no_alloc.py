"""The allocation-free join (spx_join_plain_static) against the allocating one.

spx_join_plain_static serves callers that cannot allocate device memory at
call time (memory held by another allocator, latency-bound request loops, a
fixed audited budget): its scratch is a fixed 512 KiB array inside libspx.  It
must give exactly what spx_join_plain gives, call after call (the array keeps
the previous call's contents), and refuse tables above its 2^24-point limit.
This file is collected last so that a stopping run has already run the rest.
"""
import numpy as np
import pytest

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


def _join_both(eng, pts, v, o, gl):
    P = o.shape[0] - 1
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()  # borrowed by the handle below
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=gl)
    cap = 2 * pts.shape[0] + 8
    ref_pairs = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
    ref_counts = torch.zeros(P, dtype=torch.int64, device="cuda")
    n_ref = eng.join(ph, ih, ref_pairs, ref_counts, plain=True)
    outs = []
    for _ in range(2):  # two calls in a row share the static scratch
        pairs = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
        counts = torch.zeros(P, dtype=torch.int64, device="cuda")
        total = torch.zeros(1, dtype=torch.int64, device="cuda")
        eng.join_plain_static(ph, ih, pairs, counts, total)
        torch.cuda.synchronize()
        outs.append((pairs.cpu().numpy().copy(), counts.cpu().numpy().copy(), int(total.item())))
    ref = (ref_pairs.cpu().numpy(), ref_counts.cpu().numpy())
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    del dpts
    return n_ref, ref, outs


@pytest.mark.parametrize("case", ["stars", "tessellation", "overlapping"])
def test_static_join_equals_allocating_join(eng, case):
    if case == "stars":
        v, o = g.star_polygons(g.SEED_BASE + 1)
        pts = g.uniform_points(1_000_003, g.SEED_BASE + 1)
        gl = 9
    elif case == "tessellation":
        t = g.quad_tessellation(20, 15, 7, kmin=4, kmax=200)
        v, o = t.verts, t.ring_off
        pts = g.mixture_points(3_000_000, 7)
        gl = 10
    else:
        mix = g.make_mixture(5)
        v, o = g.query_polygons(64, 5, mix, vmax=1500, r_med=0.03)
        pts = g.mixture_points(500_000, 5, mix)
        gl = 9
    n_ref, (ref_pairs, ref_counts), outs = _join_both(eng, pts, v, o, gl)
    for pairs, counts, total in outs:
        assert total == n_ref
        assert np.array_equal(pairs[:n_ref], ref_pairs[:n_ref])   # same pairs, same order, bit for bit
        assert (pairs[n_ref:] == -1).all()                         # nothing written past the total
        assert np.array_equal(counts, ref_counts)


def test_static_join_rejects_oversized_table(eng):
    n = (1 << 24) + 1
    dpts = torch.zeros((n, 2), dtype=torch.int32, device="cuda")
    ph = eng.load_points(dpts)
    v, o = g.star_polygons(3)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=6)
    pairs = torch.empty((16, 2), dtype=torch.int32, device="cuda")
    counts = torch.zeros(256, dtype=torch.int64, device="cuda")
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(spx.SpxError) as ei:
        eng.join_plain_static(ph, ih, pairs, counts, total)
    assert ei.value.status == spx.SPX_EINVAL and "16777216" in str(ei.value)
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    del dpts
