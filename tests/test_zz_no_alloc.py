"""The allocation-free join (spx_join_plain_static) against the oracle and the
allocating join.

spx_join_plain_static serves callers that cannot allocate device memory at
call time (memory held by another allocator, latency-bound request loops, a
fixed audited budget): its scratch is a fixed 512 KiB array inside libspx.  It
must give exactly the oracle's pairs and counts, and exactly what
spx_join_plain gives, call after call (the array keeps the previous call's
contents); it must take a table of exactly 2^24 points (the whole array, one
block scan over 65536 block totals), report the full pair total when the
output overflows its capacity while writing nothing past it, and refuse
tables above its limit.  This file is collected last so that a stopping run
has already run the rest.
"""
import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import datagen as g

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_14362_gb300 import spx  # noqa: E402

MAX_POINTS = 1 << 24


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = spx.Engine(0)
    yield e
    e.close()


def _static_calls(eng, ph, ih, P, cap, calls=2):
    outs = []
    for _ in range(calls):  # calls in a row share the static scratch
        pairs = torch.full((max(cap, 1) + 64, 2), -1, dtype=torch.int32, device="cuda")  # 64 guard rows
        counts = torch.full((P,), 7, dtype=torch.int64, device="cuda")  # stale values must be overwritten
        total = torch.zeros(1, dtype=torch.int64, device="cuda")
        eng.join_plain_static(ph, ih, pairs, counts, total, cap=cap)
        torch.cuda.synchronize()
        outs.append((pairs.cpu().numpy().copy(), counts.cpu().numpy().view(np.uint64).copy(), int(total.item())))
    return outs


def _setup(eng, pts, v, o, gl):
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()  # borrowed by the handle below
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=gl)
    return dpts, ph, gh, ih


def _case(case):
    if case == "stars":
        v, o = g.star_polygons(g.SEED_BASE + 1)
        return v, o, g.uniform_points(1_000_003, g.SEED_BASE + 1), 9
    if case == "tessellation":
        t = g.quad_tessellation(20, 15, 7, kmin=4, kmax=200)
        return t.verts, t.ring_off, g.mixture_points(3_000_000, 7), 10
    mix = g.make_mixture(5)
    v, o = g.query_polygons(64, 5, mix, vmax=1500, r_med=0.03)
    return v, o, g.mixture_points(500_000, 5, mix), 9


@pytest.mark.parametrize("case", ["stars", "tessellation", "overlapping"])
def test_static_join_equals_oracle_and_allocating_join(eng, case):
    v, o, pts, gl = _case(case)
    P = o.shape[0] - 1
    want_pairs, want_counts = oracle.join_fast(pts, v, o)
    dpts, ph, gh, ih = _setup(eng, pts, v, o, gl)
    cap = 2 * pts.shape[0] + 8
    ref_pairs = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
    ref_counts = torch.zeros(P, dtype=torch.int64, device="cuda")
    n_ref = eng.join(ph, ih, ref_pairs, ref_counts, plain=True)
    ref_pairs = ref_pairs.cpu().numpy()
    outs = _static_calls(eng, ph, ih, P, cap)
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    del dpts
    assert n_ref == want_pairs.shape[0]
    for pairs, counts, total in outs:
        assert total == want_pairs.shape[0]
        assert np.array_equal(pairs[:total].view(np.uint32), want_pairs)  # the oracle's pairs, in order
        assert np.array_equal(pairs[:total], ref_pairs[:total])            # and the allocating join's
        assert (pairs[total:] == -1).all()                                  # nothing written past the total
        assert np.array_equal(counts, want_counts)


def test_static_join_at_its_limit(eng):
    # exactly 2^24 points: every slot of the static array is a block total
    v, o = g.star_polygons(g.SEED_BASE + 1)
    pts = g.uniform_points(MAX_POINTS, g.SEED_BASE + 31)
    want_pairs, want_counts = oracle.join_fast(pts, v, o)
    dpts, ph, gh, ih = _setup(eng, pts, v, o, 8)
    outs = _static_calls(eng, ph, ih, o.shape[0] - 1, want_pairs.shape[0])
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    del dpts
    for pairs, counts, total in outs:
        assert total == want_pairs.shape[0]
        assert np.array_equal(pairs[:total].view(np.uint32), want_pairs)
        assert (pairs[total:] == -1).all()
        assert np.array_equal(counts, want_counts)


def test_static_join_output_over_capacity(eng):
    # the call is asynchronous and has no host out-parameter: *total_dev is
    # the caller's only sign of an overflow; the first cap pairs are written,
    # nothing after them, and the counts are complete
    v, o, pts, gl = _case("overlapping")
    want_pairs, want_counts = oracle.join_fast(pts, v, o)
    n = want_pairs.shape[0]
    cap = n // 3
    dpts, ph, gh, ih = _setup(eng, pts, v, o, gl)
    outs = _static_calls(eng, ph, ih, o.shape[0] - 1, cap)
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    del dpts
    for pairs, counts, total in outs:
        assert total == n
        assert np.array_equal(pairs[:cap].view(np.uint32), want_pairs[:cap])
        assert (pairs[cap:] == -1).all()
        assert np.array_equal(counts, want_counts)


def test_static_join_rejects_oversized_table(eng):
    n = MAX_POINTS + 1
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
