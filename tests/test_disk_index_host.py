"""CPU checks of the disk index's host build (spx_host_disk_index_build: the
arrays spx_build_disk_index uploads), against the oracle's distance join.

A point is resolved through the index exactly as its layout documents it (cell
word; INSIDE-one cell; list of disk << 1 | boundary, boundary entries taking
the exact test), in Python integers, and the (point, disk) pairs must equal
the oracle's.  The points include the adversarial ones for a cell
classification: points exactly on circles (Pythagorean offsets), on both
sides of cell borders, at the corners of the box, and outside it.  The
structural invariants of the lists are checked too.
"""
import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import spx

BOX = 1 << 30
MASK = (1 << 30) - 1


def resolve(idx, pts, centers, radii):
    cell, ent, g = idx["cell"], idx["entries"], idx["g"]
    sh = 30 - g
    out = []
    for i, (x, y) in enumerate(pts.tolist()):
        if not (0 <= x < BOX and 0 <= y < BOX):
            continue
        w = int(cell[((y >> sh) << g) | (x >> sh)])
        kind, pay = w >> 30, w & MASK
        if kind == 1:
            out.append((i, pay))
        elif kind == 2:
            n = int(ent[pay])
            for k in range(1, n + 1):
                e = int(ent[pay + k])
                q = e >> 1
                if not e & 1:
                    out.append((i, q))
                else:
                    dx, dy, r = x - int(centers[q, 0]), y - int(centers[q, 1]), int(radii[q])
                    if dx * dx + dy * dy <= r * r:
                        out.append((i, q))
        else:
            assert kind == 0 and pay == 0
    return np.array(out, np.uint32).reshape(-1, 2)


def check_lists(idx, Q):
    cell, ent = idx["cell"], idx["entries"]
    kinds = cell >> 30
    assert np.all(kinds <= 2)
    assert np.all(cell[kinds == 1] & MASK < Q)
    for w in cell[kinds == 2][:5000].tolist():
        off = w & MASK
        n = int(ent[off])
        assert n >= 1
        ids = ent[off + 1: off + 1 + n] >> 1
        assert np.all(np.diff(ids.astype(np.int64)) > 0)  # disk order, no repeats
        assert np.all(ids < Q)
        # a single INSIDE entry would have been a kind-1 cell word
        assert not (n == 1 and not ent[off + 1] & 1)


def crafted(seed, g):
    """Disks whose circle passes exactly through a cell's far corner X (a
    Pythagorean offset: the cell is INSIDE, closed disk) or just inside it
    (r = isqrt(|X - c|^2 - 1): X is outside, so the cell is not INSIDE), with
    the centre below and left of the cell so that X is its farthest point.
    Returns the centres, radii and the corners X."""
    rng = np.random.default_rng(seed)
    S = 1 << (30 - g)
    n = 1 << g
    cs, rs, xs = [], [], []
    for t in range(4):
        # a disk that reaches the cell only in its last column (or row): its
        # circle touches the cell's border point X from outside
        i, j = (int(v) for v in rng.integers(n // 4, n - 1, 2))
        a = int(rng.integers(1, S))
        if t % 2 == 0:
            X = np.array([i * S + S - 1, j * S + S // 2], np.int64)
            c = X + [a, 0]
        else:
            X = np.array([i * S + S // 2, j * S + S - 1], np.int64)
            c = X + [0, a]
        cs.append(c)
        rs.append(a)
        xs.append(X)
    for t in range(12):
        i, j = (int(v) for v in rng.integers(n // 2, n, 2))
        X = np.array([i * S + S - 1, j * S + S - 1], np.int64)
        if t < 4:
            m = int(S // 3 + 1 + rng.integers(0, S // 4))
            off, r = np.array([3 * m, 4 * m]), 5 * m
        else:
            off = rng.integers(S, 2 * S, 2).astype(np.int64)
            r = int(np.floor(np.sqrt(float(off @ off - 1))))
            while r * r > int(off @ off) - 1:
                r -= 1
            while (r + 1) * (r + 1) <= int(off @ off) - 1:
                r += 1
        c = X - off
        if c.min() < 0 or r >= BOX:
            continue
        cs.append(c)
        rs.append(r)
        xs.append(X)
    return np.array(cs, np.int64), np.array(rs, np.int64), np.array(xs, np.int64)


def disk_set(seed):
    rng = np.random.default_rng(seed)
    Q = 60
    c = rng.integers(0, BOX + 1, (Q, 2))
    r = np.exp(rng.normal(np.log(3e6), 1.2, Q)).astype(np.int64)
    # corners and edges of the box, a zero radius, a disk covering most of the box
    c[:6] = [[0, 0], [BOX, BOX], [0, BOX], [BOX // 2, 0], [12345, 67890], [BOX // 2, BOX // 2]]
    r[:6] = [5_000_000, 7_000_000, 1 << 22, 0, 40, (1 << 27) + 3]
    # Pythagorean radii (5k, 13k) for exact on-circle points
    r[6:10] = [5 * 1000, 13 * 4096, 5 * 123457, 13 * 77]
    return c.astype(np.int32), np.clip(r, 0, BOX - 1).astype(np.int32)


def probe_points(seed, centers, radii, g):
    rng = np.random.default_rng(seed + 1)
    S = 1 << (30 - g)
    pts = [rng.integers(0, BOX, (3000, 2))]
    # around every centre: near it, and on both sides of the nearest cell borders
    for (cx, cy), r in zip(centers.astype(np.int64), radii.astype(np.int64)):
        pts.append(np.column_stack([cx + rng.integers(-2 * r - 2, 2 * r + 3, 40),
                                    cy + rng.integers(-2 * r - 2, 2 * r + 3, 40)]))
        bx, by = (cx // S) * S, (cy // S) * S
        for dx in (-1, 0):
            for dy in (-1, 0):
                pts.append(np.array([[bx + dx, by + dy], [bx + S + dx, by + dy], [cx + r, by + dy],
                                     [bx + dx, cy - r], [cx - r + dx, cy], [cx, cy + r + dy]]))
    # exactly on the Pythagorean circles, and one unit outside
    for k, (a, b, h) in zip(range(6, 10), [(3, 4, 5), (5, 12, 13), (3, 4, 5), (5, 12, 13)]):
        m = int(radii[k]) // h
        cx, cy = int(centers[k, 0]), int(centers[k, 1])
        for sx in (-1, 1):
            for sy in (-1, 1):
                pts.append(np.array([[cx + sx * a * m, cy + sy * b * m], [cx + sx * b * m, cy + sy * a * m],
                                     [cx + sx * (a * m + 1), cy + sy * b * m]]))
    # where a cell's classification is decided: for the cells along each
    # circle and their neighbours, the four corners (an INSIDE cell must hold
    # all of them) and the point nearest the centre (a cell the disk reaches
    # must list it)
    n = 1 << g
    for (cx, cy), r in zip(centers.astype(np.int64).tolist(), radii.astype(np.int64).tolist()):
        for t in range(16):
            th = 2 * np.pi * (t + 0.5) / 16
            ci = min(max(int(cx + round(r * np.cos(th))) // S, 0), n - 1)
            cj = min(max(int(cy + round(r * np.sin(th))) // S, 0), n - 1)
            for i in range(max(ci - 1, 0), min(ci + 2, n)):
                for j in range(max(cj - 1, 0), min(cj + 2, n)):
                    x0, y0 = i * S, j * S
                    x1, y1 = x0 + S - 1, y0 + S - 1
                    pts.append(np.array([[x0, y0], [x1, y0], [x0, y1], [x1, y1],
                                         [min(max(cx, x0), x1), min(max(cy, y0), y1)]]))
    # corners of the box and points outside it
    pts.append(np.array([[0, 0], [BOX - 1, BOX - 1], [0, BOX - 1], [BOX - 1, 0], [-1, 5], [5, BOX], [BOX, BOX]]))
    p = np.concatenate(pts)
    p = p[(p >= -(1 << 31)).all(1) & (p < (1 << 31)).all(1)]
    return p.astype(np.int32)


@pytest.mark.parametrize("grid", [0, 3, 8, 11, 13])
def test_host_disk_index_resolves_like_the_oracle(grid):
    centers, radii = disk_set(0xD15C0 + grid)
    corners = np.zeros((0, 2), np.int64)
    if grid:
        cc, cr, corners = crafted(0xC0 + grid, grid)
        assert len(cr) == 16
        centers = np.concatenate([centers, cc.astype(np.int32)])
        radii = np.concatenate([radii, cr.astype(np.int32)])
    idx = spx.host_disk_index(centers, radii, grid)
    assert grid == 0 or idx["g"] == grid
    assert idx["cell"].shape[0] == 1 << (2 * idx["g"])
    check_lists(idx, centers.shape[0])
    pts = probe_points(0xD15C0 + grid, centers, radii, idx["g"])
    # the crafted corners and their neighbours across the cell borders
    near = np.concatenate([corners + d for d in ([0, 0], [1, 0], [0, 1], [1, 1], [-1, 0], [0, -1])])
    pts = np.concatenate([pts, near[(near < BOX).all(1)].astype(np.int32)])
    got = resolve(idx, pts, centers, radii)
    want, counts = oracle.disk_join(pts, centers, radii)
    assert np.array_equal(got, want)
    assert counts.sum() == want.shape[0] > 1000
    if grid:
        # a cell wholly inside a disk needs no test: the crafted cells whose
        # far corner lies exactly on the circle hold the disk as INSIDE
        q0 = centers.shape[0] - 16
        for k in range(4, 8):
            X = corners[k]
            w = int(idx["cell"][((int(X[1]) >> (30 - grid)) << grid) | (int(X[0]) >> (30 - grid))])
            q = q0 + k
            if w >> 30 == 1:
                assert w & MASK == q
            else:
                assert w >> 30 == 2
                off = w & MASK
                lst = idx["entries"][off + 1: off + 1 + int(idx["entries"][off])].astype(np.int64)
                assert (q << 1) in lst.tolist()


def test_host_disk_index_lattice_counts():
    # disc of radius h*k around a lattice point: the Gauss circle counts
    # (OEIS A000328), with cells much larger and much smaller than the disc
    h, c = 1024, 1 << 29
    ij = np.array([(i, j) for i in range(-11, 12) for j in range(-11, 12)], np.int64)
    pts = (c + h * ij).astype(np.int32)
    for grid in (3, 13, 0):
        for k, want in enumerate([1, 5, 13, 29, 49, 81, 113, 149, 197, 253, 317]):
            idx = spx.host_disk_index(np.array([[c, c]], np.int32), np.array([h * k], np.int32), grid)
            assert resolve(idx, pts, np.array([[c, c]]), np.array([h * k])).shape[0] == want


def test_host_disk_index_rejects_bad_input():
    c = np.array([[5, 5]], np.int32)
    for cc, rr in [([[-1, 5]], [3]), ([[5, BOX + 1]], [3]), ([[5, 5]], [-1]), ([[5, 5]], [BOX])]:
        with pytest.raises(spx.SpxError):
            spx.host_disk_index(np.array(cc, np.int32), np.array(rr, np.int32))
    with pytest.raises(spx.SpxError):
        spx.host_disk_index(c, np.array([3], np.int32), 14)  # finer than the largest grid
    empty = spx.host_disk_index(np.zeros((0, 2), np.int32), np.zeros(0, np.int32), 4)
    assert empty["g"] == 4 and not np.any(empty["cell"])
