"""GPU tests of the index autotuner (spx_autotune).

The tuner times candidate grid resolutions on a sample of the resident points.
The resolution must never change a result: the chosen index's join equals the
oracle byte for byte, every timed candidate gave the same per-polygon counts
(the call fails otherwise), and the choice is the fastest trial.
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


def _join(eng, ph, ih, n, P):
    pairs = torch.full((n + 16, 2), -1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(max(P, 1), dtype=torch.int64, device="cuda")
    total = eng.join(ph, ih, pairs, counts)
    torch.cuda.synchronize()
    return (pairs[:total].cpu().numpy().view(np.uint32).copy(), counts[:P].cpu().numpy().view(np.uint64).copy())


@pytest.mark.parametrize("case", ["tess", "stars"])
def test_autotune_choice_and_parity(eng, case):
    if case == "tess":
        nx, ny = 16, 12
        t = g.quad_tessellation(nx, ny, g.SEED_BASE + 40, kmin=4, kmax=60)
        v, o = t.verts, t.ring_off
        pts = g.mixture_points(3_000_000 + 77, g.SEED_BASE + 40, g.make_mixture(g.SEED_BASE + 40))
    else:
        v, o = g.star_polygons(g.SEED_BASE + 41)
        pts = g.uniform_points(2_000_000 + 5, g.SEED_BASE + 41)
    P = o.shape[0] - 1
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    params, trials, ih = eng.autotune(ph, gh, grid_min=4, grid_max=11, reps=3)
    try:
        assert 4 <= params["grid_log2"] <= 11 and 1 <= params["sub_log2"] <= 3
        assert params["fp32_filter"] == 1
        keys = [(t["grid_log2"], t["sub_log2"]) for t in trials]
        assert len(keys) == len(set(keys)) >= 2
        assert all(t["ms"] > 0 and t["device_bytes"] > 0 for t in trials)
        fastest = min(trials, key=lambda t: t["ms"])
        assert (params["grid_log2"], params["sub_log2"]) == (fastest["grid_log2"], fastest["sub_log2"])
        info = eng.index_info(ih)
        assert (info["grid_log2"], info["sub_log2"]) == (params["grid_log2"], params["sub_log2"])
        # the tuned index gives the oracle's join, byte for byte
        pairs, counts = _join(eng, ph, ih, pts.shape[0], P)
        ref = oracle.Prepared(v, o)
        rp, rc = ref.join(pts)
        ref.close()
        assert np.array_equal(pairs, rp)
        assert np.array_equal(counts, rc)
        # and so does the returned parameter set when rebuilt
        ih2 = eng.build_index(gh, grid_log2=params["grid_log2"], sub_log2=params["sub_log2"])
        pairs2, _ = _join(eng, ph, ih2, pts.shape[0], P)
        eng.free(ih2)
        assert np.array_equal(pairs2, rp)
    finally:
        eng.free(ih)
        eng.free(gh)
        eng.free(ph)
        del dpts


def test_autotune_sample_and_limits(eng):
    v, o = g.star_polygons(g.SEED_BASE + 42)
    pts = g.uniform_points(100_003, g.SEED_BASE + 42)
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    try:
        # a sample larger than the table is clamped; one grid only; no index kept
        params, trials, ih = eng.autotune(ph, gh, sample_points=10**9, grid_min=7, grid_max=7, reps=1,
                                          fp32_filter=False, keep_index=False)
        assert ih is None
        assert params["grid_log2"] == 7 and params["fp32_filter"] == 0
        assert sorted(t["sub_log2"] for t in trials) == [1, 2, 3]
        # settings out of range
        for kw in ({"grid_min": 9, "grid_max": 8}, {"grid_max": 14}, {"reps": 1001}):
            with pytest.raises(spx.SpxError) as ei:
                eng.autotune(ph, gh, **kw)
            assert ei.value.status == spx.SPX_EINVAL
        # every candidate over the memory limit
        with pytest.raises(spx.SpxError) as ei:
            eng.autotune(ph, gh, grid_min=6, grid_max=7, max_index_bytes=1024)
        assert ei.value.status == spx.SPX_EINVAL and "max_index_bytes" in str(ei.value)
    finally:
        eng.free(gh)
        eng.free(ph)
        del dpts


def test_autotune_empty_table(eng):
    v, o = g.star_polygons(g.SEED_BASE + 43)
    ph = eng.load_points(np.zeros((0, 2), np.int32))
    gh = eng.load_polygons(v, o)
    try:
        with pytest.raises(spx.SpxError) as ei:
            eng.autotune(ph, gh)
        assert ei.value.status == spx.SPX_EINVAL
    finally:
        eng.free(gh)
        eng.free(ph)
