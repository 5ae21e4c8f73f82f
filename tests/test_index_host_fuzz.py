"""Property test of the polygon index's host build on adversarial geometry.

Rings are drawn with vertices snapped onto the borders of coarse and fine
cells (and one unit beside them), with horizontal edges lying exactly on row
borders, repeated vertices, self-intersections and collinear runs.  Probe
points sit on and beside every vertex, on cell corners and at random.  Walking
the host-built index the way the kernels walk it (test_index_host.walk) must
give exactly the oracle's pairs, at random grid and subdivision sizes.  The
examples are derandomised, so the test is the same on every run.
"""
import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import spx

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")

from test_index_host import walk  # noqa: E402

BOX = 1 << 30


@st.composite
def scene(draw):
    gl = draw(st.integers(1, 9))
    sb = draw(st.integers(1, 3))
    S = 1 << min(30 - gl - sb, 26)  # a unit whose multiples include every fine cell border
    P = draw(st.integers(1, 5))
    rings = []
    for _ in range(P):
        n = draw(st.integers(3, 10))
        # a centre cell and vertices a few fine cells around it, on a cell
        # border, one unit beside it, or anywhere in the cell
        cx = draw(st.integers(5, (BOX // S) - 6))
        cy = draw(st.integers(5, (BOX // S) - 6))
        ring = []
        for _ in range(n):
            kx, ky = draw(st.integers(-4, 4)), draw(st.integers(-4, 4))
            mode = draw(st.sampled_from(["on", "on", "minus", "plus", "any"]))
            dx = {"on": 0, "minus": -1, "plus": 1}.get(mode, draw(st.integers(0, S - 1)))
            dy = {"on": 0, "minus": -1, "plus": 1}.get(mode, draw(st.integers(0, S - 1)))
            ring.append(((cx + kx) * S + dx, (cy + ky) * S + dy))
            if draw(st.booleans()) and len(ring) < n:  # a horizontal edge on the row border
                ring.append(((cx + draw(st.integers(-4, 4))) * S, (cy + ky) * S + dy))
            if draw(st.integers(0, 9)) == 0:  # a repeated vertex
                ring.append(ring[-1])
        rings.append(ring)
    seed = draw(st.integers(0, 2**31))
    return gl, sb, rings, seed


def probes(v, seed, S):
    rng = np.random.default_rng(seed)
    v = v.astype(np.int64)
    near = [v + d for d in ([0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, -1])]
    corners = (v // S) * S
    lo, hi = v.min(0) - S, v.max(0) + S
    rnd = np.column_stack([rng.integers(lo[0], hi[0] + 1, 300), rng.integers(lo[1], hi[1] + 1, 300)])
    p = np.concatenate(near + [corners, corners - 1, rnd])
    return p[(p >= 0).all(1) & (p < BOX).all(1)].astype(np.int32)


@hyp.settings(max_examples=150, deadline=None, derandomize=True, database=None,
              suppress_health_check=list(hyp.HealthCheck))
@hyp.given(scene())
def test_host_index_on_adversarial_rings(sc):
    gl, sb, rings, seed = sc
    v = np.array([p for r in rings for p in r], np.int64)
    assert (v >= 0).all() and (v <= BOX).all()
    v = v.astype(np.int32)
    off = np.zeros(len(rings) + 1, np.uint64)
    off[1:] = np.cumsum([len(r) for r in rings])
    pts = probes(v, seed, 1 << (30 - gl - sb))
    want, _ = oracle.join_fast(pts, v, off)
    ix = spx.host_index(v, off, gl, sb)
    got = walk(ix, pts)
    assert np.array_equal(got, want)
