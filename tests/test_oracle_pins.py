"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* brute force on tiny inputs against an independent formulation: the
  perturbed point p + (eps, eps^2) is replaced by a concrete scaled point that
  lies off every edge line, and containment is decided by a signed winding
  number in exact Python integers (even-odd = winding mod 2);
* hand-worked boundary cases (tests/golden/boundary_cases.json);
* closed forms for axis-aligned rectangles (half-open boxes) and lattice counts;
* additivity over a fan triangulation and the tessellation invariant (every
  point of the box in exactly one cell);
* metamorphic invariants: integer translation, ring reversal, cyclic rotation,
  duplicated vertices;
* pure mode == fast mode (the shortcuts s1-s3 keep the definition).

`battery(lib)` runs the pins that a planted mistake must trip; the mutation
test compiles mistaken copies of the oracle and checks that each one fails it.
"""
import json
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import datagen as g

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------ independent formulation
def inside_winding(px, py, ring):
    """Containment of p + (eps, eps^2) by a signed winding number (Sunday's
    crossing rule) around the concrete point (S*px + 2M, S*py + 1) of the ring
    scaled by S = 4M^2.  With M bounding every coordinate difference, that
    point lies on no edge line and at no vertex height, and each orientation
    has the sign of the perturbed one: S^2 * d dominates S * (dx - 2M * dy)
    when d != 0, and -2M * dy dominates dx when d == 0."""
    xs = [int(v[0]) for v in ring] + [int(px)]
    ys = [int(v[1]) for v in ring] + [int(py)]
    M = 2 * (max(xs + ys) - min(xs + ys)) + 1
    S = 4 * M * M
    qx, qy = S * int(px) + 2 * M, S * int(py) + 1
    wn = 0
    n = len(ring)
    for i in range(n):
        ax, ay = S * int(ring[i][0]), S * int(ring[i][1])
        bx, by = S * int(ring[(i + 1) % n][0]), S * int(ring[(i + 1) % n][1])
        left = (bx - ax) * (qy - ay) - (qx - ax) * (by - ay)
        if ay <= qy:
            if by > qy and left > 0:
                wn += 1
        elif by <= qy and left < 0:
            wn -= 1
    return wn % 2 != 0


def tiny_polygons(seed=7, n_random=60):
    """Hand-made and random rings with vertices in [0, 16]^2: collinear edges,
    vertices on lattice points, horizontal and vertical edges, spikes,
    self-intersections, repeated vertices."""
    polys = [
        [(2, 2), (10, 2), (10, 9), (2, 9)],                     # rectangle
        [(2, 2), (6, 2), (10, 2), (10, 9), (2, 9), (2, 5)],     # collinear extra vertices
        [(0, 0), (8, 0), (0, 8)],                               # right triangle
        [(1, 1), (15, 1), (8, 15)],                             # triangle, slanted edges
        [(3, 3), (12, 12), (12, 3), (3, 12)],                   # bow-tie (self-intersecting)
        [(2, 8), (8, 2), (14, 8), (8, 14), (8, 8)],             # spike to the centre
        [(1, 1), (5, 1), (5, 5), (9, 5), (9, 1), (13, 1), (13, 13), (1, 13)],  # concave notch
        [(4, 4), (4, 4), (12, 4), (12, 12), (12, 12), (4, 12)],  # duplicated vertices
        [(0, 0), (16, 0), (16, 16), (0, 16)],                   # whole small box
        [(5, 0), (10, 5), (5, 10), (0, 5)],                     # diamond: vertices at extreme y
        [(3, 7), (13, 7), (13, 7)],                             # degenerate (zero area)
        [(2, 2), (14, 2), (8, 2)],                              # degenerate collinear
        [(1, 3), (7, 3), (7, 9), (11, 9), (11, 3), (15, 3), (15, 13), (1, 13)],  # horizontal runs at one y
    ]
    rng = np.random.default_rng(seed)
    for k in range(n_random):
        n = int(rng.integers(3, 9))
        polys.append([tuple(int(c) for c in rng.integers(0, 17, 2)) for _ in range(n)])
    return [np.array(p, dtype=np.int32) for p in polys]


def pack(rings):
    off = np.zeros(len(rings) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(r) for r in rings])
    return np.concatenate(rings).astype(np.int32), off


LATTICE16 = np.array([(x, y) for y in range(17) for x in range(17)], dtype=np.int32)


# ------------------------------------------------------------------ the pins
def pin_brute_force(lib):
    bad = []
    for ri, ring in enumerate(tiny_polygons()):
        for px, py in LATTICE16:
            want = inside_winding(px, py, ring)
            got = oracle.point_in_ring(px, py, ring, lib)
            if want != got:
                bad.append((ri, int(px), int(py), want, got))
    return bad


def pin_golden(lib):
    with open(os.path.join(HERE, "golden", "boundary_cases.json")) as f:
        fx = json.load(f)
    polys = {k: np.array(v, dtype=np.int32) for k, v in fx["polygons"].items()}
    bad = []
    for name, px, py, want in fx["cases"]:
        if int(oracle.point_in_ring(px, py, polys[name], lib)) != want:
            bad.append((name, px, py, want))
    return bad


def pin_rectangles(lib, seed=11, n_rect=40, n_pts=4000):
    """count = #{x0 <= px < x1, y0 <= py < y1} on points that hit the rectangle
    sides and corners often, through both the pure and the fast join."""
    rng = np.random.default_rng(seed)
    bad = []
    def aligned():
        # a corner on a power-of-two boundary (+-1): hits the edges of any
        # power-of-two bucket or grid cell exactly
        r = int(rng.integers(16, 26))
        return int(rng.integers(1, (1 << 30) >> r)) * (1 << r) + int(rng.integers(-1, 2))

    for k in range(n_rect):
        if k % 2:
            x0, x1 = sorted(aligned() for _ in range(2))
            y0, y1 = sorted(aligned() for _ in range(2))
        else:
            x0, x1 = sorted(int(v) for v in rng.integers(0, 1 << 30, 2))
            y0, y1 = sorted(int(v) for v in rng.integers(0, 1 << 30, 2))
        if k % 7 == 0:
            x1 = x0  # degenerate
        cand_x = np.array([x0 - 1, x0, x0 + 1, x1 - 1, x1, x1 + 1], dtype=np.int64)
        cand_y = np.array([y0 - 1, y0, y0 + 1, y1 - 1, y1, y1 + 1], dtype=np.int64)
        px = np.where(rng.random(n_pts) < 0.5, rng.choice(cand_x, n_pts), rng.integers(0, 1 << 30, n_pts))
        py = np.where(rng.random(n_pts) < 0.5, rng.choice(cand_y, n_pts), rng.integers(0, 1 << 30, n_pts))
        ok = (px >= 0) & (px < (1 << 30)) & (py >= 0) & (py < (1 << 30))
        pts = np.stack([px[ok], py[ok]], 1).astype(np.int32)
        want = int(((pts[:, 0] >= x0) & (pts[:, 0] < x1) & (pts[:, 1] >= y0) & (pts[:, 1] < y1)).sum())
        ring = g.rect_polygon(x0, y0, x1, y1)
        variants = [ring, ring[::-1], np.roll(ring, 1, 0),
                    np.array([[x0, y0], [(x0 + x1) // 2, y0], [x1, y0], [x1, y1], [x0, y1], [x0, y1]], np.int32)]
        v, o = pack(variants)
        _, cp = oracle.join_pure(pts, v, o, lib) if pts.shape[0] <= 600 else (None, None)
        p = oracle.Prepared(v, o, lib)
        _, cf = p.join(pts, threads=2)
        p.close()
        for c in ([cf] + ([cp] if cp is not None else [])):
            if any(int(x) != want for x in c):
                bad.append((k, want, [int(x) for x in c]))
    # lattice closed form: origin o, spacing h
    for k in range(10):
        h = int(rng.integers(1, 50))
        ox, oy = int(rng.integers(0, 1000)), int(rng.integers(0, 1000))
        xs = ox + h * np.arange(60)
        ys = oy + h * np.arange(60)
        pts = np.stack(np.meshgrid(xs, ys, indexing="ij"), -1).reshape(-1, 2).astype(np.int32)
        x0, x1 = sorted(int(v) for v in rng.integers(ox, ox + 60 * h, 2))
        y0, y1 = sorted(int(v) for v in rng.integers(oy, oy + 60 * h, 2))
        ceil = lambda a, b: -((-a) // b)
        want = (ceil(x1 - ox, h) - ceil(x0 - ox, h)) * (ceil(y1 - oy, h) - ceil(y0 - oy, h))
        v, o = pack([g.rect_polygon(x0, y0, x1, y1)])
        p = oracle.Prepared(v, o, lib)
        _, cf = p.join(pts, threads=2)
        p.close()
        if int(cf[0]) != want:
            bad.append(("lattice", k, want, int(cf[0])))
    return bad


def pin_fan_additivity(lib, seed=5):
    """A convex polygon and the triangles of its fan partition it, so every
    point is counted by the polygon iff by exactly one triangle."""
    rng = np.random.default_rng(seed)
    bad = []
    for k in range(12):
        n = int(rng.integers(4, 12))
        ang = np.sort(rng.random(n)) * 2 * np.pi
        c = rng.integers(300, 700, 2)
        r = int(rng.integers(50, 300))
        ring = np.stack([c[0] + r * np.cos(ang), c[1] + r * np.sin(ang)], 1).round().astype(np.int32)
        tris = [np.stack([ring[0], ring[i], ring[i + 1]]) for i in range(1, n - 1)]
        v, o = pack([ring] + tris)
        # dense lattice around the polygon hits vertices, edges and diagonals
        xs = np.arange(c[0] - r - 2, c[0] + r + 3)
        ys = np.arange(c[1] - r - 2, c[1] + r + 3)
        pts = np.stack(np.meshgrid(xs, ys, indexing="ij"), -1).reshape(-1, 2).astype(np.int32)
        p = oracle.Prepared(v, o, lib)
        pairs, counts = p.join(pts, threads=2)
        p.close()
        in_poly = np.zeros(pts.shape[0], np.int64)
        in_tris = np.zeros(pts.shape[0], np.int64)
        m = pairs[:, 1] == 0
        in_poly[pairs[m, 0]] += 1
        np.add.at(in_tris, pairs[~m, 0], 1)
        if not np.array_equal(in_poly, in_tris):
            bad.append((k, int((in_poly != in_tris).sum())))
    return bad


def tess_probe_points(t: g.Tessellation, seed=3, n_random=20000):
    """Random points plus every mesh vertex, every polygon vertex and lattice
    points exactly on polygon edges (inside the box)."""
    rng = np.random.default_rng(seed)
    pts = [rng.integers(0, 1 << 30, (n_random, 2))]
    pts.append(t.verts.astype(np.int64))
    v = t.verts.astype(np.int64)
    nxt = np.roll(np.arange(len(v)), -1)
    for q in range(len(t.ring_off) - 1):
        b, e = int(t.ring_off[q]), int(t.ring_off[q + 1])
        idx = np.arange(b, e)
        nxt[idx] = np.roll(idx, -1)
    d = v[nxt] - v
    gcd = np.gcd(np.abs(d[:, 0]), np.abs(d[:, 1]))
    m = gcd > 1
    pts.append(v[m] + d[m] // gcd[m, None])         # first lattice point along the edge
    pts.append(v[m] + (d[m] // gcd[m, None]) * (gcd[m, None] // 2))
    # points on the axis-parallel border edges
    pts.append(np.stack([np.zeros(200, np.int64), rng.integers(0, 1 << 30, 200)], 1))
    pts.append(np.stack([rng.integers(0, 1 << 30, 200), np.zeros(200, np.int64)], 1))
    pts = np.concatenate(pts)
    ok = (pts >= 0).all(1) & (pts < (1 << 30)).all(1)
    return pts[ok].astype(np.int32)


def pin_tessellation(lib, nx=5, ny=4, seed=9):
    t = g.quad_tessellation(nx, ny, seed, kmin=2, kmax=30)
    pts = tess_probe_points(t)
    p = oracle.Prepared(t.verts, t.ring_off, lib)
    pairs, counts = p.join(pts, threads=2)
    p.close()
    hits = np.bincount(pairs[:, 0].astype(np.int64), minlength=pts.shape[0])
    bad = []
    if not (hits == 1).all():
        bad.append(("tess", int((hits != 1).sum())))
    if int(counts.sum()) != pts.shape[0]:
        bad.append(("tess-sum", int(counts.sum()), pts.shape[0]))
    return bad


def battery(lib):
    return {
        "brute_force": pin_brute_force(lib),
        "golden": pin_golden(lib),
        "rectangles": pin_rectangles(lib, n_rect=12, n_pts=1500),
        "fan": pin_fan_additivity(lib),
        "tessellation": pin_tessellation(lib),
    }


# ------------------------------------------------------------------ tests
def test_brute_force_tiny(olib):
    assert pin_brute_force(olib) == []


def test_golden_boundary_cases(olib):
    assert pin_golden(olib) == []


def test_rectangles_closed_form(olib):
    assert pin_rectangles(olib) == []


def test_fan_triangulation_additivity(olib):
    assert pin_fan_additivity(olib) == []


@pytest.mark.parametrize("nx,ny,seed", [(5, 4, 9), (3, 7, 21), (8, 8, 2)])
def test_tessellation_invariant(olib, nx, ny, seed):
    assert pin_tessellation(olib, nx, ny, seed) == []


def test_join_pure_brute_force_pairs(olib):
    """The pure join's pairs are exactly the brute-force pairs, in order."""
    rings = tiny_polygons(seed=3, n_random=20)
    v, o = pack(rings)
    pairs, counts = oracle.join_pure(LATTICE16, v, o, olib)
    want = [(i, q) for i, (px, py) in enumerate(LATTICE16) for q, r in enumerate(rings) if inside_winding(px, py, r)]
    assert [tuple(map(int, p)) for p in pairs] == want
    assert counts.tolist() == np.bincount([q for _, q in want], minlength=len(rings)).tolist()


def test_pure_equals_fast(olib):
    cases = []
    v, o = g.star_polygons(g.SEED_BASE + 1)
    cases.append((g.uniform_points(3000, 5), v, o))
    t = g.quad_tessellation(6, 5, 4, kmin=2, kmax=40)
    cases.append((np.concatenate([g.mixture_points(2000, 4), tess_probe_points(t, n_random=0)[:1500]]), t.verts, t.ring_off))
    mix = g.make_mixture(8)
    qv, qo = g.query_polygons(12, 8, mix, vmax=300)
    cases.append((g.mixture_points(3000, 8, mix), qv, qo))
    rings = tiny_polygons(seed=4, n_random=30)
    tv, to = pack(rings)
    cases.append((LATTICE16, tv, to))
    for pts, v, o in cases:
        pp, cp = oracle.join_pure(pts, v, o, olib)
        for th in (1, 3):
            pr = oracle.Prepared(v, o, olib)
            pf, cf = pr.join(pts, threads=th)
            pr.close()
            assert np.array_equal(pp, pf)
            assert np.array_equal(cp, cf)


def test_points_outside_the_box(olib):
    # vertices lie in [0, 2^30]^2: a point outside [0, 2^30)^2 is in no polygon
    # (the box's right and top sides are outside under the half-open rule);
    # the pure mode tests every edge, the fast mode must agree
    box = 1 << 30
    v = np.array([[0, 0], [box, 0], [box, box], [0, box]], np.int32)
    o = np.array([0, 4], np.uint64)
    pts = np.array([[5, 5], [-1, 5], [5, -1], [box, 5], [5, box], [-(1 << 31), 7], [(1 << 31) - 1, 0],
                    [(1 << 31) - 1, (1 << 31) - 1], [box - 1, box - 1], [0, 0]], np.int32)
    t = g.quad_tessellation(4, 3, 9, kmin=2, kmax=20)
    for vv, oo in ((v, o), (t.verts, t.ring_off)):
        pp, cp = oracle.join_pure(pts, vv, oo, olib)
        pr = oracle.Prepared(vv, oo, olib)
        pf, cf = pr.join(pts, threads=2)
        pr.close()
        assert np.array_equal(pp, pf) and np.array_equal(cp, cf)
        assert sorted(set(pp[:, 0].tolist())) == [0, 8, 9]  # only the three points inside the box


def test_metamorphic_translation_reversal_rotation(olib):
    rng = np.random.default_rng(17)
    mix = g.make_mixture(12)
    v, o = g.query_polygons(10, 12, mix, vmax=200)
    v = v.astype(np.int64)
    # keep clear of the box border so the translation stays in range
    v = np.clip(v, 1 << 20, (1 << 30) - (1 << 20))
    pts = g.mixture_points(5000, 12, mix)
    pts = np.clip(pts, 1 << 20, (1 << 30) - (1 << 20))
    # put some points exactly on vertices
    pts[:200] = v[rng.integers(0, len(v), 200)]
    base_p, base_c = oracle.join_fast(pts, v.astype(np.int32), o)
    tx, ty = 12345, -54321
    p2, c2 = oracle.join_fast((pts + [tx, ty]).astype(np.int32), (v + [tx, ty]).astype(np.int32), o)
    assert np.array_equal(base_p, p2) and np.array_equal(base_c, c2)
    rings = [v[int(o[q]):int(o[q + 1])] for q in range(len(o) - 1)]
    for tf in (lambda r: r[::-1], lambda r: np.roll(r, 3, 0), lambda r: np.concatenate([r, r[:1]])):
        rv, ro = pack([tf(r).astype(np.int32) for r in rings])
        p3, c3 = oracle.join_fast(pts, rv, ro)
        assert np.array_equal(base_p, p3) and np.array_equal(base_c, c3)


def test_star_polygons_disjoint(olib):
    v, o = g.star_polygons(g.SEED_BASE + 1)
    pts = g.uniform_points(200000, g.SEED_BASE + 1)
    pairs, counts = oracle.join_fast(pts, v, o)
    assert np.unique(pairs[:, 0]).size == pairs.shape[0]          # each point at most once
    cell = (1 << 30) // 16
    q = (pts[:, 1] // cell) * 16 + pts[:, 0] // cell
    cx = (pts[:, 0] // cell) * cell + cell / 2
    cy = (pts[:, 1] // cell) * cell + cell / 2
    r = np.hypot(pts[:, 0] - cx, pts[:, 1] - cy)
    far = r > 0.46 * cell                                         # outside every star's max radius
    near = r < 0.29 * cell                                        # inside every star's min radius (stars are star-shaped)
    hit = np.zeros(pts.shape[0], bool)
    hit[pairs[:, 0]] = True
    assert not hit[far].any()
    assert hit[near].all()
    assert np.array_equal(pairs[:, 1], q[pairs[:, 0]].astype(np.uint32))


def test_select_groups_ascending(olib):
    mix = g.make_mixture(31)
    v, o = g.query_polygons(16, 31, mix, vmax=400, r_med=0.05)
    pts = g.mixture_points(20000, 31, mix)
    pr = oracle.Prepared(v, o, olib)
    ids, off = pr.select(pts)
    pairs, counts = pr.join(pts)
    pr.close()
    for q in range(16):
        lst = ids[int(off[q]):int(off[q + 1])]
        assert np.all(np.diff(lst.astype(np.int64)) > 0)
        assert np.array_equal(lst, pairs[pairs[:, 1] == q, 0])


# ----------------------------------------------------------- planted mistakes
MUTANTS = {
    "straddle_ge": ("if ((ay > py) == (by > py))", "if ((ay >= py) == (by >= py))"),
    "count_on_edge": ("    if (d == 0)\n        return 0;\n    return (d > 0) == (by > ay);",
                      "    return (d >= 0) == (by > ay);"),
    "wrong_sign": ("return (d > 0) == (by > ay);", "return (d > 0) != (by > ay);"),
    "transposed": ("int64_t d = (bx - ax) * (py - ay) - (by - ay) * (px - ax);",
                   "int64_t d = (bx - ax) * (px - ax) - (by - ay) * (py - ay);"),
    "dropped_term": ("int64_t d = (bx - ax) * (py - ay) - (by - ay) * (px - ax);",
                     "int64_t d = (bx - ax) * (py - ay);"),
    "open_ring": ("uint64_t j = (i + 1 == n) ? 0 : i + 1;\n        in ^=",
                  "uint64_t j = (i + 1 == n) ? i : i + 1;\n        in ^="),
    "bbox_open_left": ("if (px < g->xmin || px >= g->xmax", "if (px <= g->xmin || px >= g->xmax"),
    "bucket_last_row": ("by1 = (g->ymax - 1) >> o->bucket_log2", "by1 = (g->ymax - 2) >> o->bucket_log2"),
    "slab_off_by_one": ("int64_t s1 = ((int64_t)hi - 1 - g->ymin) / g->slab_h;",
                        "int64_t s1 = ((int64_t)hi - 2 - g->ymin) / g->slab_h;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "pip_oracle.c")).read()
    old, new = MUTANTS[name]
    assert old in src, f"mutation site for {name} not found"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", str(mut), "-o", str(so)])
    lib = oracle.load(str(so))
    res = battery(lib)
    res["pure_vs_fast"] = []
    # the fast-mode-only mutants show up as pure/fast disagreement or as pin failures
    t = g.quad_tessellation(4, 4, 6, kmin=2, kmax=20)
    pts = tess_probe_points(t, n_random=3000)
    pp, cp = oracle.join_pure(pts[:2500], t.verts, t.ring_off, lib)
    pr = oracle.Prepared(t.verts, t.ring_off, lib)
    pf, cf = pr.join(pts[:2500], threads=2)
    pr.close()
    if not (np.array_equal(pp, pf) and np.array_equal(cp, cf)):
        res["pure_vs_fast"] = ["differ"]
    assert any(len(v) for v in res.values()), f"mutant {name} passed every pin"


def test_battery_clean_on_real_oracle(olib):
    res = battery(olib)
    assert all(len(v) == 0 for v in res.values()), res
