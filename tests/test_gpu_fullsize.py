"""GPU parity at the benchmark's full sizes, in the launch configuration the
benchmark times.

* 100M mixture points x the 2000-cell tessellation (the default benchmark
  line): the whole join, every pair and every count, against the oracle.
* 500M mixture points x 256 overlapping query polygons (the batched
  selection): properties of the whole output (offsets, ascending lists, ids in
  range) and, for a seeded sample of 100k points, exactly the queries the
  oracle puts them in.
* 100M mixture points x 1024 disks (the distance join): properties of the
  whole output (order, counts) and, for a seeded sample of 100k points, exactly
  the disks the oracle puts them in.

The inputs are the benchmark's own (`bench.make_workload`).
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import bench  # noqa: E402
from paper_2203_14362_gb300 import spx  # noqa: E402

SAMPLE = 100_000


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = spx.Engine(0)
    yield e
    e.close()


def _sample(n, seed):
    return np.unique(np.random.default_rng(seed).integers(0, n, SAMPLE)).astype(np.int64)


def _restrict(pairs, ids):
    """The rows of pairs (sorted by point id) whose point id is in ids (sorted)."""
    lo = np.searchsorted(pairs[:, 0], ids, "left")
    hi = np.searchsorted(pairs[:, 0], ids, "right")
    take = np.concatenate([np.arange(a, b) for a, b in zip(lo, hi)]) if len(ids) else np.zeros(0, np.int64)
    return pairs[take.astype(np.int64)]


def _oracle_on(pairs_local, ids):
    out = pairs_local.astype(np.int64).copy()
    out[:, 0] = ids[out[:, 0]]
    return out


def test_tess2000_100m_whole_join(eng):
    pts, v, o, _ = bench.make_workload("tess2000_100m", None, 0)
    N, P = pts.shape[0], o.shape[0] - 1
    dpts = torch.from_numpy(pts).cuda()
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=0, fp32_filter=True, sub_log2=0)
    try:
        pairs = torch.empty((N, 2), dtype=torch.int32, device="cuda")
        counts = torch.zeros(P, dtype=torch.int64, device="cuda")
        n = eng.join(ph, ih, pairs, counts)
        assert n == N  # a tessellation: every point in exactly one cell
        got_p = pairs.cpu().numpy().view(np.uint32)
        got_c = counts.cpu().numpy().view(np.uint64)
    finally:
        eng.free(ih)
        eng.free(gh)
        eng.free(ph)
        del dpts
    ref = oracle.Prepared(v, o)
    want_p, want_c = ref.join(pts)
    ref.close()
    assert np.array_equal(got_c, want_c)
    assert np.array_equal(got_p, want_p)


@pytest.mark.parametrize("params", [(0, 0), (13, 3)])  # default index; the autotuner's choice
def test_select256_500m_sampled(eng, params):
    pts, v, o, _ = bench.make_workload("select256_500m", None, 0)
    N, Q = pts.shape[0], o.shape[0] - 1
    dpts = torch.from_numpy(pts).cuda()
    del pts  # regenerated below only where needed
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=params[0], fp32_filter=True, sub_log2=params[1])
    try:
        offs = torch.zeros(Q + 1, dtype=torch.int64, device="cuda")
        probe = torch.empty(1, dtype=torch.int32, device="cuda")
        with pytest.raises(spx.SpxError) as ei:
            eng.select(ph, ih, probe, offs)
        assert ei.value.status == spx.SPX_ECAPACITY
        total = int(str(ei.value).split("needs ")[1].split(" ")[0])
        ids = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
        assert eng.select(ph, ih, ids, offs) == total
        got_ids = ids[:total].cpu().numpy().view(np.uint32).astype(np.int64)
        got_off = offs.cpu().numpy()
        sample = _sample(N, 0x5E1EC7)
        sample_pts = dpts[torch.from_numpy(sample).cuda()].cpu().numpy()
    finally:
        eng.free(ih)
        eng.free(gh)
        eng.free(ph)
        del dpts
    # the whole output: offsets, ascending lists, ids in range
    assert got_off[0] == 0 and got_off[-1] == total and np.all(np.diff(got_off) >= 0)
    q_of = np.repeat(np.arange(Q), np.diff(got_off))
    same_q = q_of[1:] == q_of[:-1]
    assert np.all(got_ids[1:][same_q] > got_ids[:-1][same_q])
    assert got_ids.min(initial=0) >= 0 and got_ids.max(initial=0) < N
    # the sample: exactly the oracle's (point, query) pairs
    keep = np.isin(got_ids, sample)
    got = np.stack([got_ids[keep], q_of[keep]], 1)
    got = got[np.lexsort((got[:, 1], got[:, 0]))]
    ref = oracle.Prepared(v, o)
    wp, _ = ref.join(sample_pts)
    ref.close()
    assert np.array_equal(got, _oracle_on(wp, sample))


def test_dist1024_100m_sampled(eng):
    pts, centers, radii, _ = bench.make_workload("dist1024_100m", None, 0)
    N, Q = pts.shape[0], centers.shape[0]
    dpts = torch.from_numpy(pts).cuda()
    ph = eng.load_points(dpts)
    ih = eng.build_disk_index(centers, radii, 0)
    try:
        pairs = torch.empty((N, 2), dtype=torch.int32, device="cuda")
        counts = torch.zeros(Q, dtype=torch.int64, device="cuda")
        n = eng.join(ph, ih, pairs, counts)
        got_p = pairs[:n].cpu().numpy().view(np.uint32).astype(np.int64)
        got_c = counts.cpu().numpy().view(np.uint64)
        c2 = torch.zeros(Q, dtype=torch.int64, device="cuda")
        eng.aggregate(ph, ih, c2)
        torch.cuda.synchronize()
        assert np.array_equal(c2.cpu().numpy().view(np.uint64), got_c)
    finally:
        eng.free(ih)
        eng.free(ph)
        del dpts
    # the whole output: (point, disk) order, counts
    key = got_p[:, 0] * Q + got_p[:, 1]
    assert np.all(np.diff(key) > 0)
    assert np.array_equal(np.bincount(got_p[:, 1], minlength=Q).astype(np.uint64), got_c)
    # the sample: exactly the oracle's pairs
    sample = _sample(N, 0xD15C)
    wp, _ = oracle.disk_join(pts[sample], centers, radii)
    assert np.array_equal(_restrict(got_p, sample), _oracle_on(wp, sample))
