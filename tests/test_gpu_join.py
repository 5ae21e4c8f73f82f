"""GPU parity: libspx's CUDA kernels against the CPU oracle, bit for bit.

Every call goes through the C ABI (ctypes binding).  Pairs and counts must be
identical to the oracle's; the FP32 filter must not change a single byte; the
plain comparison kernels must agree too.  Sizes span many 2048-point tiles and
a ragged tail; edge cases cover empty and one-point tables, points outside the
box, degenerate and overlapping polygons, and an output that overflows its
capacity.
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


def run_join(eng, pts, v, o, gl, fp32=True, plain=False, cap=None, sub=0):
    P = o.shape[0] - 1
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()  # borrowed: keep alive while the handle is used
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=gl, fp32_filter=fp32, sub_log2=sub)
    cap = pts.shape[0] * 2 + 16 if cap is None else cap
    pairs = torch.full((max(cap, 1), 2), -1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(max(P, 1), dtype=torch.int64, device="cuda")
    n = eng.join(ph, ih, pairs, counts, plain=plain)
    torch.cuda.synchronize()
    out = pairs[:min(n, cap)].cpu().numpy().view(np.uint32).copy()
    cnt = counts[:P].cpu().numpy().view(np.uint64).copy()
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    del dpts
    return out, cnt, n


def run_aggregate(eng, pts, v, o, gl, fp32=True, sub=0):
    P = o.shape[0] - 1
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=gl, fp32_filter=fp32, sub_log2=sub)
    counts = torch.zeros(max(P, 1), dtype=torch.int64, device="cuda")
    eng.aggregate(ph, ih, counts)
    torch.cuda.synchronize()
    cnt = counts[:P].cpu().numpy().view(np.uint64).copy()
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    del dpts
    return cnt


def scaled_tiny(s_log2=26):
    rings = [
        [(2, 2), (10, 2), (10, 9), (2, 9)], [(0, 0), (8, 0), (0, 8)], [(3, 3), (12, 12), (12, 3), (3, 12)],
        [(2, 8), (8, 2), (14, 8), (8, 14), (8, 8)],
        [(1, 1), (5, 1), (5, 5), (9, 5), (9, 1), (13, 1), (13, 13), (1, 13)],
        [(0, 0), (16, 0), (16, 16), (0, 16)], [(5, 0), (10, 5), (5, 10), (0, 5)],
        [(1, 3), (7, 3), (7, 9), (11, 9), (11, 3), (15, 3), (15, 13), (1, 13)], [(3, 7), (13, 7), (13, 7)],
        [(4, 4), (4, 4)], [(6, 6)],
    ]
    s = 1 << s_log2
    v = np.concatenate([np.array(r, np.int64) * s for r in rings]).astype(np.int32)
    off = np.zeros(len(rings) + 1, np.uint64)
    off[1:] = np.cumsum([len(r) for r in rings])
    pts = np.array([(x * s + dx, y * s + dy) for x in range(16) for y in range(16)
                    for dx in (-1, 0, 1) for dy in (-1, 0, 1)], dtype=np.int64)
    pts = pts[(pts >= 0).all(1) & (pts < (1 << 30)).all(1)].astype(np.int32)
    return pts, v, off


def check(eng, pts, v, o, gls=(4, 8, 11), aggregate=True, subs=(3,)):
    want_p, want_c = oracle.join_fast(pts, v, o)
    cap = want_p.shape[0] + 5
    for gl in gls:
        for sub in subs:
            for fp32 in (True, False):
                p, c, n = run_join(eng, pts, v, o, gl, fp32, cap=cap, sub=sub)
                assert n == want_p.shape[0]
                assert np.array_equal(p, want_p), f"pairs differ at g={gl} sub={sub} fp32={fp32}"
                assert np.array_equal(c, want_c), f"counts differ at g={gl} sub={sub} fp32={fp32}"
                if aggregate:
                    assert np.array_equal(run_aggregate(eng, pts, v, o, gl, fp32, sub), want_c)
    p, c, n = run_join(eng, pts, v, o, gls[0], plain=True, cap=cap)
    assert np.array_equal(p, want_p) and np.array_equal(c, want_c), "plain kernels differ"


def test_grid_aligned_tiny(eng):
    pts, v, o = scaled_tiny()
    check(eng, pts, v, o, gls=(1, 2, 4, 5, 9), subs=(1, 2, 3))


def test_stars_uniform(eng):
    v, o = g.star_polygons(g.SEED_BASE + 1)
    pts = g.uniform_points(300_001, g.SEED_BASE + 1)  # ragged tail
    pts = np.concatenate([pts, v[(v < (1 << 30)).all(1)]])  # vertices as points
    check(eng, pts, v, o)


def test_tessellation_mixture(eng):
    t = g.quad_tessellation(20, 15, 5, kmin=4, kmax=200)
    pts = g.mixture_points(400_000, 5)
    vv = t.verts.astype(np.int64)
    extra = np.concatenate([vv, vv + 1, vv - 1])
    extra = extra[(extra >= 0).all(1) & (extra < (1 << 30)).all(1)].astype(np.int32)
    pts = np.concatenate([pts, extra])
    want_p, want_c = oracle.join_fast(pts, t.verts, t.ring_off)
    assert int(want_c.sum()) == pts.shape[0]  # tessellation invariant holds on the oracle side
    check(eng, pts, t.verts, t.ring_off, gls=(6, 9, 12), subs=(1, 3))


def test_block_summary_on_and_off(eng):
    # pass 1a reads the coarse level's block summary from shared memory when
    # enough of its blocks are resolved (large polygons), and reads every
    # coarse word from the index otherwise (small polygons); both must give
    # the oracle's bytes, including points on block and cell borders
    cases = []
    for nx, ny, gl in ((20, 15, 12), (6, 5, 8), (120, 100, 8), (120, 100, 5)):
        t = g.quad_tessellation(nx, ny, 40 + nx, kmin=2, kmax=60)
        pts = g.mixture_points(300_000, 40 + nx)
        border = np.array([(x << 22) + d for x in range(0, 256, 3) for d in (-1, 0, 1)], np.int64)
        bx, by = np.meshgrid(border, border[::7])
        extra = np.stack([bx.ravel(), by.ravel()], 1)
        extra = extra[(extra >= 0).all(1) & (extra < (1 << 30)).all(1)].astype(np.int32)
        pts = np.concatenate([pts, extra])
        want_p, want_c = oracle.join_fast(pts, t.verts, t.ring_off)
        gh = eng.load_polygons(t.verts, t.ring_off)
        ih = eng.build_index(gh, grid_log2=gl)
        info = eng.index_info(ih)
        eng.free(ih)
        eng.free(gh)
        cases.append(info["use_sum"])
        p, c, n = run_join(eng, pts, t.verts, t.ring_off, gl)
        assert n == want_p.shape[0] and np.array_equal(p, want_p) and np.array_equal(c, want_c), (nx, gl)
    assert 1 in cases and 0 in cases, cases


def test_overlapping_queries(eng):
    mix = g.make_mixture(9)
    v, o = g.query_polygons(64, 9, mix, vmax=2000, r_med=0.03)
    pts = g.mixture_points(200_000, 9, mix)
    want_p, _ = oracle.join_fast(pts, v, o)
    assert (np.bincount(want_p[:, 0].astype(np.int64)) > 1).any()  # multi-match points exist
    check(eng, pts, v, o, gls=(5, 8, 11))


def test_empty_and_single(eng):
    v, o = g.star_polygons(3)
    for n in (0, 1, 2, 2047, 2048, 2049):
        pts = g.uniform_points(n, 77) if n else np.zeros((0, 2), np.int32)
        want_p, want_c = oracle.join_fast(pts, v, o) if n else (np.zeros((0, 2), np.uint32),
                                                               np.zeros(256, np.uint64))
        p, c, m = run_join(eng, pts, v, o, 6)
        assert m == want_p.shape[0] and np.array_equal(p, want_p) and np.array_equal(c, want_c)
        assert np.array_equal(run_aggregate(eng, pts, v, o, 6), want_c)


def test_points_outside_box_are_in_no_polygon(eng):
    v = np.array([[0, 0], [1 << 30, 0], [1 << 30, 1 << 30], [0, 1 << 30]], np.int32)
    o = np.array([0, 4], np.uint64)
    pts = np.array([[5, 5], [-1, 5], [5, -1], [1 << 30, 5], [5, 1 << 30], [-(1 << 31), 7], [(1 << 31) - 1, 0]],
                   np.int32)
    p, c, n = run_join(eng, pts, v, o, 3)
    assert n == 1 and p.tolist() == [[0, 0]] and c.tolist() == [1]


def test_capacity_overflow_reports_size(eng):
    v, o = g.star_polygons(4)
    pts = g.uniform_points(50_000, 4)
    want_p, _ = oracle.join_fast(pts, v, o)
    with pytest.raises(spx.SpxError) as ei:
        run_join(eng, pts, v, o, 7, cap=100)
    assert ei.value.status == spx.SPX_ECAPACITY
    assert str(want_p.shape[0]) in str(ei.value)


def test_deterministic_and_stats(eng):
    t = g.quad_tessellation(10, 10, 8, kmin=4, kmax=100)
    pts = g.mixture_points(500_000, 8)
    eng.stats(reset=True)
    a = run_join(eng, pts, t.verts, t.ring_off, 10)
    s = eng.stats(reset=True)
    b = run_join(eng, pts, t.verts, t.ring_off, 10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert s["points_scanned"] == pts.shape[0]
    assert s["pairs_emitted"] == a[2]
    assert s["fp32_escalations"] <= s["edge_tests"]


def test_join_host_end_to_end(eng):
    v, o = g.star_polygons(g.SEED_BASE + 1)
    pts = g.uniform_points(123_457, 11)
    want_p, want_c = oracle.join_fast(pts, v, o)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh, grid_log2=9)
    p, c, n = eng.join_host(pts, ih, cap=pts.shape[0], n_polys=256)
    assert n == want_p.shape[0] and np.array_equal(p, want_p) and np.array_equal(c, want_c)
    eng.free(ih)
    eng.free(gh)


@pytest.mark.parametrize("pinned", [False, True])
def test_join_host_slices(eng, pinned):
    # three 2^23-point slices, the last one ragged, overlapping polygons (a
    # point can have several pairs, so slice offsets do not follow point ids)
    mix = g.make_mixture(g.SEED_BASE + 60)
    pts = g.mixture_points((1 << 24) + 123_457, g.SEED_BASE + 60, mix)
    v, o = g.query_polygons(40, g.SEED_BASE + 60, mix, r_med=0.05, r_clip=(0.01, 0.2))
    ref = oracle.Prepared(v, o)
    want_p, want_c = ref.join(pts)
    ref.close()
    assert want_p.shape[0] > 0 and np.any(np.bincount(want_p[:, 0].astype(np.int64)) > 1)
    gh = eng.load_polygons(v, o)
    ih = eng.build_index(gh)
    P = o.shape[0] - 1
    cap = want_p.shape[0] + 5
    if pinned:
        hp = torch.empty((cap, 2), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
        hx = torch.empty(pts.shape, dtype=torch.int32, pin_memory=True).numpy()
        hx[:] = pts
    else:
        hp, hx = None, pts
    p, c, n = eng.join_host(hx, ih, cap=cap, n_polys=P, pairs_out=hp)
    assert n == want_p.shape[0] and np.array_equal(p, want_p) and np.array_equal(c, want_c)
    # a capacity that runs out in the middle slice: the first cap pairs, then the error
    small = want_p.shape[0] // 2
    buf = np.zeros((small, 2), np.uint32)
    with pytest.raises(spx.SpxError) as ei:
        eng.join_host(hx, ih, cap=small, n_polys=P, pairs_out=buf)
    assert ei.value.status == spx.SPX_ECAPACITY
    assert np.array_equal(buf, want_p[:small])
    eng.free(ih)
    eng.free(gh)


def test_bad_arguments(eng):
    with pytest.raises(spx.SpxError):
        eng.load_points(np.array([[1 << 30, 0]], np.int32))
    with pytest.raises(spx.SpxError):
        eng.load_polygons(np.array([[0, 0], [(1 << 30) + 1, 0], [0, 5]], np.int32), np.array([0, 3], np.uint64))
    gh = eng.load_polygons(*g.star_polygons(1))
    with pytest.raises(spx.SpxError):
        eng.build_index(gh, grid_log2=14)
    ih = eng.build_index(gh, grid_log2=5)
    with pytest.raises(spx.SpxError):
        eng.free(gh)  # index still alive
    eng.free(ih)
    eng.free(gh)


def test_summary_grows_between_calls_in_a_fresh_process():
    # pass 1a opts its kernels in to their shared memory once per process and
    # device; a first join through a small block summary (g = 7, 32 KB) must
    # not keep a later one through the full 128 KB summary (g = 8 and up)
    # from launching.  A fresh process fixes the order of the calls.
    import os
    import subprocess
    import sys
    code = r'''
import numpy as np, torch
import oracle
from paper_2203_14362_gb300 import datagen as g, spx
eng = spx.Engine(0)
v, o = g.star_polygons(g.SEED_BASE + 41)
pts = g.uniform_points(300_001, g.SEED_BASE + 41)
want_p, want_c = oracle.join_fast(pts, v, o)
dpts = torch.from_numpy(pts).cuda()
ph = eng.load_points(dpts)
gh = eng.load_polygons(v, o)
for gl, sb in ((7, 1), (8, 1), (11, 3), (5, 2), (9, 2)):
    ih = eng.build_index(gh, grid_log2=gl, sub_log2=sb)
    pairs = torch.full((pts.shape[0] + 8, 2), -1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(256, dtype=torch.int64, device="cuda")
    n = eng.join(ph, ih, pairs, counts)
    assert n == want_p.shape[0], (gl, sb, n)
    assert np.array_equal(pairs[:n].cpu().numpy().view(np.uint32), want_p), (gl, sb)
    assert np.array_equal(counts.cpu().numpy().view(np.uint64), want_c), (gl, sb)
    eng.free(ih)
print("ok")
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]
