"""The bounds-checked debug build (libspx_checked.so, SPX_BOUNDS_CHECK) and the
bounded-wait error path, on the GPU.

In the checked build every offset and id the kernels read from an index is
compared with the index's array sizes before it is used; a violation sets the
error word, which the host reports as SPX_EKERNEL.  Indexes are built valid
(the host build is validated before upload; the device build equals it), so
the checks are exercised here on valid inputs only, where they must stay
silent and change no result: joins (with points in several polygons),
aggregates (row order and cell-clustered), selections and the plain join,
through indexes built on the host and on the device, against the oracle.
The error path itself is shown with the bounded wait of pass 1a's bulk-copy
staging run against a barrier nothing completes: it must end with
SPX_ETIMEOUT and leave the context usable.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2203_14362_gb300 import build as b
from paper_2203_14362_gb300 import datagen as g

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_14362_gb300 import spx  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHECKED_RUN = r'''
import numpy as np, torch
import oracle
from paper_2203_14362_gb300 import datagen as g, spx
assert spx.LIB_PATH.endswith("libspx_checked.so")
eng = spx.Engine(0)
cases = []
t = g.quad_tessellation(20, 15, 5, kmin=4, kmax=200)
cases.append((t.verts, t.ring_off, g.mixture_points(300_000, 5), 10))
mix = g.make_mixture(9)
v, o = g.query_polygons(64, 9, mix, vmax=2000, r_med=0.03)
cases.append((v, o, g.mixture_points(200_000, 9, mix), 11))
v, o = g.star_polygons(g.SEED_BASE + 1)
cases.append((v, o, g.uniform_points(200_001, 3), 6))
for v, o, pts, gl in cases:
    P = o.shape[0] - 1
    want_p, want_c = oracle.join_fast(pts, v, o)
    dpts = torch.from_numpy(pts).cuda()
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    for dev in (False, True):
        ih = eng.build_index(gh, grid_log2=gl, on_device=dev)
        pairs = torch.full((pts.shape[0] * 2 + 8, 2), -1, dtype=torch.int32, device="cuda")
        counts = torch.zeros(P, dtype=torch.int64, device="cuda")
        for plain in (False, True):
            n = eng.join(ph, ih, pairs, counts, plain=plain)
            assert n == want_p.shape[0]
            assert np.array_equal(pairs[:n].cpu().numpy().view(np.uint32), want_p)
            assert np.array_equal(counts.cpu().numpy().view(np.uint64), want_c)
        eng.aggregate(ph, ih, counts)
        pc = eng.cluster_points(ph, 10)
        c2 = torch.zeros(P, dtype=torch.int64, device="cuda")
        eng.aggregate(pc, ih, c2)
        torch.cuda.synchronize()
        assert np.array_equal(counts.cpu().numpy().view(np.uint64), want_c)
        assert np.array_equal(c2.cpu().numpy().view(np.uint64), want_c)
        eng.free(pc)
        if P <= 1024:
            ids = torch.empty(max(want_p.shape[0], 1), dtype=torch.int32, device="cuda")
            offs = torch.zeros(P + 1, dtype=torch.int64, device="cuda")
            assert eng.select(ph, ih, ids, offs) == want_p.shape[0]
            want_ids, want_offs = oracle.group_by_polygon(want_p, want_c)
            assert np.array_equal(ids.cpu().numpy().view(np.uint32), want_ids)
            assert np.array_equal(offs.cpu().numpy().view(np.uint64), want_offs)
        eng.stats(reset=True)  # reads the error word: raises if a check fired
        eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    del dpts
eng.close()
print("checked build: all results equal the oracle, no bounds check fired")
'''


def test_checked_build_is_silent_on_valid_indexes():
    lib = b.build(checked=True)
    env = dict(os.environ, SPX_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHECKED_RUN], capture_output=True, text=True, timeout=900, cwd=ROOT,
                       env=env)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "no bounds check fired" in r.stdout


def test_bounded_wait_reports_timeout_and_the_context_stays_usable():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    eng = spx.Engine(0)
    try:
        for _ in range(2):
            assert eng.check_bounded_wait(2000) == spx.SPX_ETIMEOUT
        # the error word was read and cleared: the context works as before
        v, o = g.star_polygons(3)
        pts = g.uniform_points(10_000, 3)
        dpts = torch.from_numpy(pts).cuda()
        ph = eng.load_points(dpts)
        gh = eng.load_polygons(v, o)
        ih = eng.build_index(gh, grid_log2=6)
        pairs = torch.empty((20_000, 2), dtype=torch.int32, device="cuda")
        counts = torch.zeros(256, dtype=torch.int64, device="cuda")
        n = eng.join(ph, ih, pairs, counts)
        assert n == int(counts.sum().item())
        eng.free(ih)
        eng.free(gh)
        eng.free(ph)
    finally:
        eng.close()
