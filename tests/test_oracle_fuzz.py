"""Property test of the oracle at full coordinate range (2^30): the pure and
fast modes against the independent formulation of test_oracle_pins (a
concrete point off every edge line, signed winding number in exact Python
integers).  Rings are drawn anywhere in [0, 2^30]^2, with vertices snapped to
a coarse lattice to make collinear runs, shared heights and horizontal edges
likely; probes sit on the vertices, one unit beside them, on exact lattice
points of the edges (steps of the edge direction divided by its gcd) and at
random.  Products of coordinate differences reach 2^61 here, which a
narrower integer type would overflow.  Examples are derandomised."""
import math

import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")

from test_oracle_pins import inside_winding  # noqa: E402

BOX = 1 << 30


@st.composite
def ring_and_points(draw):
    unit = 1 << draw(st.integers(0, 28))
    n = draw(st.integers(3, 9))
    ring = []
    for _ in range(n):
        x = min(draw(st.integers(0, BOX // unit)) * unit + draw(st.sampled_from([0, 0, 1, -1])), BOX)
        y = min(draw(st.integers(0, BOX // unit)) * unit + draw(st.sampled_from([0, 0, 1, -1])), BOX)
        ring.append((max(x, 0), max(y, 0)))
        if draw(st.integers(0, 3)) == 0:  # a horizontal edge
            ring.append((min(draw(st.integers(0, BOX // unit)) * unit, BOX), ring[-1][1]))
    pts = []
    for (x, y) in ring:
        for dx, dy in ((0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, -1)):
            pts.append((x + dx, y + dy))
    for i in range(len(ring)):
        (ax, ay), (bx, by) = ring[i], ring[(i + 1) % len(ring)]
        gd = math.gcd(abs(bx - ax), abs(by - ay))
        if gd:
            k = draw(st.integers(0, gd))
            sx, sy = (bx - ax) // gd, (by - ay) // gd
            px, py = ax + k * sx, ay + k * sy
            pts += [(px, py), (px + 1, py), (px, py + 1), (px - 1, py)]
    for _ in range(6):
        pts.append((draw(st.integers(0, BOX - 1)), draw(st.integers(0, BOX - 1))))
    pts = [(x, y) for x, y in pts if 0 <= x < BOX and 0 <= y < BOX]
    return np.array(ring, np.int64), np.array(pts, np.int64).reshape(-1, 2)


@hyp.settings(max_examples=200, deadline=None, derandomize=True, database=None,
              suppress_health_check=list(hyp.HealthCheck))
@hyp.given(ring_and_points())
def test_oracle_matches_winding_at_full_range(rp):
    ring, pts = rp
    want = np.array([inside_winding(px, py, ring) for px, py in pts.tolist()], bool)
    r32 = ring.astype(np.int32)
    got = np.array([oracle.point_in_ring(px, py, r32) for px, py in pts.tolist()], bool)
    assert np.array_equal(got, want)
    v, off = r32, np.array([0, len(ring)], np.uint64)
    p32 = pts.astype(np.int32)
    fast, _ = oracle.join_fast(p32, v, off)
    pure, _ = oracle.join_pure(p32, v, off)
    ids = np.nonzero(want)[0].astype(np.uint32)
    assert np.array_equal(fast[:, 0], ids) and np.array_equal(pure[:, 0], ids)
