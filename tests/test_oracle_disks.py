"""Pins of the oracle's distance join (SPADE §5.2 "Distance-Based Queries":
pairs with distance(point, centre) <= r).

The expected values do not come from the oracle: the number of lattice points
in a closed disc of integer radius r (the Gauss circle problem; the sequence
1, 5, 13, 29, 49, ... is OEIS A000328, and its first terms are easy to count by
hand), Pythagorean triples that put a point exactly on the circle, and
invariance under translation.
"""
import numpy as np
import pytest

import oracle

# lattice points (x, y) in Z^2 with x^2 + y^2 <= r^2, r = 0..10
LATTICE_IN_DISC = [1, 5, 13, 29, 49, 81, 113, 149, 197, 253, 317]


@pytest.fixture(scope="module")
def olib():
    return oracle.load()


def test_lattice_counts(olib):
    h, c = 1024, 1 << 29
    ij = np.array([(i, j) for i in range(-12, 13) for j in range(-12, 13)], np.int64)
    pts = (c + h * ij).astype(np.int32)
    centers = np.array([[c, c]] * len(LATTICE_IN_DISC), np.int32)
    radii = np.array([h * r for r in range(len(LATTICE_IN_DISC))], np.int32)
    pairs, counts = oracle.disk_join(pts, centers, radii, olib)
    assert counts.tolist() == LATTICE_IN_DISC
    # every lattice point of disc r is in disc r + 1 (nested discs, same centre)
    by_q = [set(pairs[pairs[:, 1] == q, 0].tolist()) for q in range(len(LATTICE_IN_DISC))]
    assert all(by_q[q] <= by_q[q + 1] for q in range(len(by_q) - 1))


def test_boundary_is_inside(olib):
    c = 1 << 29
    k = 1000
    # (3k, 4k) is at distance exactly 5k; one unit further in x is outside
    pts = np.array([[c + 3 * k, c + 4 * k], [c + 3 * k + 1, c + 4 * k], [c - 5 * k, c], [c, c - 5 * k - 1]], np.int32)
    for r, want in ((5 * k, [0, 2]), (5 * k - 1, []), (5 * k + 1, [0, 1, 2, 3])):
        pairs, counts = oracle.disk_join(pts, np.array([[c, c]], np.int32), np.array([r], np.int32), olib)
        assert pairs[:, 0].tolist() == want and counts.tolist() == [len(want)]


def test_zero_radius_and_far_points(olib):
    c = 1 << 29
    pts = np.array([[c, c], [c + 1, c], [-(1 << 31), -(1 << 31)], [(1 << 31) - 1, (1 << 31) - 1], [0, 0]], np.int32)
    centers = np.array([[c, c], [0, 0]], np.int32)
    radii = np.array([0, (1 << 30) - 1], np.int32)
    pairs, counts = oracle.disk_join(pts, centers, radii, olib)
    # a zero radius holds its centre only; the far corners are outside even the large disc
    assert pairs.tolist() == [[0, 0], [0, 1], [1, 1], [4, 1]]
    assert counts.tolist() == [1, 3]


def test_points_outside_the_domain(olib):
    # points lie in [0, 2^30)^2; one outside is in no disk, even a disk around it
    pts = np.array([[-1, 0], [0, -3], [1 << 30, 5], [0, 0], [2, 0]], np.int32)
    pairs, counts = oracle.disk_join(pts, np.array([[0, 0]], np.int32), np.array([5], np.int32), olib)
    assert pairs[:, 0].tolist() == [3, 4] and counts.tolist() == [2]


def test_translation_invariance_and_order(olib):
    rng = np.random.default_rng(5)
    pts = rng.integers(1 << 20, 1 << 21, size=(20_000, 2)).astype(np.int32)
    centers = rng.integers(1 << 20, 1 << 21, size=(40, 2)).astype(np.int32)
    radii = rng.integers(0, 1 << 17, size=40).astype(np.int32)
    a, ca = oracle.disk_join(pts, centers, radii, olib)
    off = np.array([123_457, (1 << 28) + 5], np.int32)
    b, cb = oracle.disk_join(pts + off, centers + off, radii, olib)
    assert np.array_equal(a, b) and np.array_equal(ca, cb)
    key = a[:, 0].astype(np.int64) * 64 + a[:, 1]
    assert np.all(np.diff(key) > 0)  # sorted by (point, disk), no duplicates
    assert ca.sum() == a.shape[0] > 0
