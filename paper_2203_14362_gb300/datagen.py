"""Seeded synthetic inputs for the point-in-polygon join, selection and count.

This module only draws inputs: it holds none of the join's arithmetic, and both
the CUDA path and the CPU oracle are fed from it.  Every random number comes from
one counter-based generator, SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output i of a stream with key k is
mix(k + (i + 1) * 0x9E3779B97F4A7C15), so any slice of a stream can be drawn
without drawing the part before it.

The shapes follow the workloads of SPADE's evaluation (§6.1 Table 1, §6.2, §6.6):
city-scale clustered points, tessellations of irregular polygons with tens to
thousands of vertices, and query polygons of 8-5000 vertices.  The real datasets
(taxi pickups, tweets, neighbourhood / census / county / zip polygons) are not
available; these generators stand in for them.

Coordinates are int32 fixed point.  Points lie in [0, 2^30)^2; polygon vertices
lie in [0, 2^30]^2 (closed, so a tessellation can close the box).

Layouts (shared by every consumer):
  points   int32 array (N, 2), C-contiguous, rows (x, y); point id = row index
  polygons (verts int32 (V, 2), ring_off uint64 (P + 1)); polygon q is the ring
           verts[ring_off[q]:ring_off[q + 1]], implicitly closed
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BOX = 1 << 30  # side of the coordinate box
GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


# --------------------------------------------------------------------------- RNG
def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, *path: int | str) -> np.uint64:
    """Derive the key of a named sub-stream from a seed and a path of labels."""
    k = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    for p in path:
        if isinstance(p, str):
            v = 0
            for ch in p.encode():
                v = (v * 131 + ch) & 0xFFFFFFFFFFFFFFFF
        else:
            v = int(p) & 0xFFFFFFFFFFFFFFFF
        with np.errstate(over="ignore"):
            k = _mix(k ^ np.array([v], dtype=np.uint64)) + GOLDEN
    return k[0]


def u64(key: np.uint64, start: int, count: int, idx: np.ndarray | None = None) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream with this key
    (or the outputs at the given indices when `idx` is passed)."""
    if idx is None:
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    else:
        idx = idx.astype(np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(key) + idx * GOLDEN)


def unif(key: np.uint64, start: int, count: int, idx: np.ndarray | None = None) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the stream."""
    return (u64(key, start, count, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(key: np.uint64, start: int, count: int, idx: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Two independent standard normals per index (Box-Muller on two sub-streams)."""
    u1 = unif(stream_key(int(key), "bm1"), start, count, idx)
    u2 = unif(stream_key(int(key), "bm2"), start, count, idx)
    r = np.sqrt(-2.0 * np.log1p(-u1))
    t = 2.0 * math.pi * u2
    return r * np.cos(t), r * np.sin(t)


# ------------------------------------------------------------------------ points
def uniform_points(n: int, seed: int) -> np.ndarray:
    """n points uniform on the integer lattice [0, 2^30)^2."""
    out = np.empty((n, 2), dtype=np.int32)
    kx, ky = stream_key(seed, "ux"), stream_key(seed, "uy")
    for s in range(0, n, _CHUNK):
        c = min(_CHUNK, n - s)
        out[s:s + c, 0] = (u64(kx, s, c) >> np.uint64(34)).astype(np.int32)
        out[s:s + c, 1] = (u64(ky, s, c) >> np.uint64(34)).astype(np.int32)
    return out


@dataclass
class Mixture:
    """A Gaussian mixture over the box plus a uniform background share."""
    centers: np.ndarray   # (K, 2) float64
    sigmas: np.ndarray    # (K,) float64, in coordinate units
    cdf: np.ndarray       # (K,) cumulative component weights, last = 1
    background: float


def make_mixture(seed: int, k: int = 64, sigma_frac=(0.005, 0.05), background: float = 0.10,
                 zipf_s: float | None = None) -> Mixture:
    """64 Gaussians with centres uniform in the box and sigma uniform in
    [0.5 %, 5 %] of the box side; equal weights, or Zipf weights w_k ~ k^-s."""
    cen = np.stack([unif(stream_key(seed, "mix_cx"), 0, k), unif(stream_key(seed, "mix_cy"), 0, k)], 1) * BOX
    sig = (sigma_frac[0] + (sigma_frac[1] - sigma_frac[0]) * unif(stream_key(seed, "mix_sig"), 0, k)) * BOX
    w = np.ones(k) if zipf_s is None else np.arange(1, k + 1, dtype=np.float64) ** (-zipf_s)
    cdf = np.cumsum(w) / w.sum()
    cdf[-1] = 1.0
    return Mixture(cen, sig, cdf, background)


def mixture_points(n: int, seed: int, mix: Mixture | None = None, start: int = 0) -> np.ndarray:
    """Points start .. start+n-1 of a clustered point table: with probability
    `background` uniform, else drawn from a mixture component; draws that leave
    [0, 2^30)^2 are redrawn from the next redraw sub-stream at the same index."""
    mix = mix or make_mixture(seed)
    out = np.empty((n, 2), dtype=np.int32)
    ksel, kcomp = stream_key(seed, "sel"), stream_key(seed, "comp")
    for s in range(0, n, _CHUNK):
        c = min(_CHUNK, n - s)
        g0 = start + s
        bg = unif(ksel, g0, c) < mix.background
        comp = np.searchsorted(mix.cdf, unif(kcomp, g0, c), side="right")
        comp = np.minimum(comp, len(mix.cdf) - 1)
        x = np.empty(c)
        y = np.empty(c)
        pending = np.arange(c)
        attempt = 0
        while pending.size:
            gi = g0 + pending  # global indices still to draw
            kn = stream_key(seed, "gauss", attempt)
            ku = stream_key(seed, "bgu", attempt)
            if attempt == 0:
                nx, ny = normal(kn, g0, c)
                ux, uy = unif(stream_key(int(ku), "x"), g0, c), unif(stream_key(int(ku), "y"), g0, c)
            else:
                nx, ny = normal(kn, 0, 0, gi)
                ux, uy = unif(stream_key(int(ku), "x"), 0, 0, gi), unif(stream_key(int(ku), "y"), 0, 0, gi)
            cm = comp[pending]
            gx = np.floor(mix.centers[cm, 0] + mix.sigmas[cm] * nx)
            gy = np.floor(mix.centers[cm, 1] + mix.sigmas[cm] * ny)
            b = bg[pending]
            gx = np.where(b, np.floor(ux * BOX), gx)
            gy = np.where(b, np.floor(uy * BOX), gy)
            ok = (gx >= 0) & (gx < BOX) & (gy >= 0) & (gy < BOX)
            x[pending[ok]] = gx[ok]
            y[pending[ok]] = gy[ok]
            pending = pending[~ok]
            attempt += 1
            if attempt > 200:  # never reached in practice; keeps the loop finite
                x[pending] = np.clip(gx[~ok], 0, BOX - 1)
                y[pending] = np.clip(gy[~ok], 0, BOX - 1)
                break
        out[s:s + c, 0] = x.astype(np.int32)
        out[s:s + c, 1] = y.astype(np.int32)
    return out


# ---------------------------------------------------------------------- polygons
def _mixture_chunk(args):
    # worker of mixture_points_parallel: fill rows [lo, hi) of the shared table
    from multiprocessing import shared_memory
    name, n, seed, mix, start, lo, hi = args
    shm = shared_memory.SharedMemory(name=name)
    try:
        out = np.ndarray((n, 2), dtype=np.int32, buffer=shm.buf)
        out[lo:hi] = mixture_points(hi - lo, seed, mix, start + lo)
        del out
    finally:
        shm.close()
    return hi - lo


def mixture_points_parallel(n: int, seed: int, mix: Mixture | None = None, start: int = 0,
                            workers: int | None = None) -> np.ndarray:
    """mixture_points(n, seed, mix, start), computed by a pool of spawned
    processes over chunks of the index range.  Every point depends only on its
    global index, so the result is the same array, byte for byte."""
    import multiprocessing as mp
    import os
    from multiprocessing import shared_memory
    mix = mix or make_mixture(seed)
    workers = workers or min(32, os.cpu_count() or 1)
    step = 1 << 23
    if workers <= 1 or n <= step:
        return mixture_points(n, seed, mix, start)
    shm = shared_memory.SharedMemory(create=True, size=max(n * 8, 8))
    try:
        jobs = [(shm.name, n, seed, mix, start, lo, min(n, lo + step)) for lo in range(0, n, step)]
        with mp.get_context("spawn").Pool(workers) as pool:
            done = sum(pool.imap_unordered(_mixture_chunk, jobs))
        assert done == n
        return np.ndarray((n, 2), dtype=np.int32, buffer=shm.buf).copy()
    finally:
        shm.close()
        shm.unlink()


def _rings(parts: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    off = np.zeros(len(parts) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(p) for p in parts])
    verts = np.concatenate(parts).astype(np.int32) if parts else np.zeros((0, 2), np.int32)
    return np.ascontiguousarray(verts), off


def star_polygons(seed: int, grid: int = 16, kmin: int = 16, kmax: int = 64,
                  rmin: float = 0.3, rmax: float = 0.45) -> tuple[np.ndarray, np.ndarray]:
    """One star-shaped polygon per cell of a grid x grid partition of the box:
    k ~ U{kmin..kmax} vertices at angles 2*pi*(m + U(-0.4, 0.4))/k and radii
    U(rmin, rmax) * cell around the cell centre.  The polygons never overlap."""
    cell = BOX // grid
    parts = []
    for q in range(grid * grid):
        cx = (q % grid) * cell + cell / 2
        cy = (q // grid) * cell + cell / 2
        k = kmin + int(u64(stream_key(seed, "star_k"), q, 1)[0] % np.uint64(kmax - kmin + 1))
        ka = stream_key(seed, "star_a", q)
        kr = stream_key(seed, "star_r", q)
        ang = 2 * math.pi * (np.arange(k) + 0.8 * (unif(ka, 0, k) - 0.5)) / k
        rad = (rmin + (rmax - rmin) * unif(kr, 0, k)) * cell
        parts.append(np.stack([np.rint(cx + rad * np.cos(ang)), np.rint(cy + rad * np.sin(ang))], 1))
    return _rings(parts)


def rect_polygon(x0: int, y0: int, x1: int, y1: int) -> np.ndarray:
    """Counter-clockwise ring of the axis-aligned rectangle [x0, x1] x [y0, y1]."""
    return np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], dtype=np.int32)


@dataclass
class Tessellation:
    verts: np.ndarray
    ring_off: np.ndarray
    nx: int
    ny: int
    lattice: np.ndarray = field(repr=False)  # (nx+1, ny+1, 2) int64 mesh corners


def _left_normal(d: np.ndarray) -> np.ndarray:
    return np.stack([-d[..., 1], d[..., 0]], -1)


def quad_tessellation(nx: int, ny: int, seed: int, kmin: int = 12, kmax: int = 499,
                      jitter: float = 0.2, amp: float = 0.35, white: float = 0.03) -> Tessellation:
    """A tessellation of the closed box [0, 2^30]^2 into nx * ny cells.

    The cell corners form a lattice jittered by up to `jitter` of the spacing
    (corners on the box border move only along it).  Every interior mesh edge is
    replaced by a polyline of k ~ logU[kmin, kmax] extra vertices that is a height
    function over the edge, kept strictly inside the edge's kite (the two
    triangles spanned by the edge and the centroids of its two cells) with a
    10 % margin; kites of different edges do not overlap, so no two cell
    boundaries cross.  The height profile is smooth like real boundaries: one
    or two slow waves of amplitude `amp` of the kite height plus a small
    vertex-to-vertex jitter (`white`).  Border edges get collinear extra
    vertices.  Each cell ring is counter-clockwise and has 4 + the sum of its
    sides' k vertices.
    """
    assert jitter <= 0.2 and nx >= 1 and ny >= 1
    sx, sy = BOX / nx, BOX / ny
    gx = np.rint(np.arange(nx + 1) * sx)
    gy = np.rint(np.arange(ny + 1) * sy)
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    nv = (nx + 1) * (ny + 1)
    vid = (ii * (ny + 1) + jj).ravel()
    jx = (2 * unif(stream_key(seed, "jit_x"), 0, nv) - 1)[vid].reshape(ii.shape) * jitter * sx
    jy = (2 * unif(stream_key(seed, "jit_y"), 0, nv) - 1)[vid].reshape(ii.shape) * jitter * sy
    jx[(ii == 0) | (ii == nx)] = 0
    jy[(jj == 0) | (jj == ny)] = 0
    L = np.stack([np.rint(gx[ii] + jx), np.rint(gy[jj] + jy)], -1)  # (nx+1, ny+1, 2) float exact ints
    L[..., 0] = np.clip(L[..., 0], 0, BOX)
    L[..., 1] = np.clip(L[..., 1], 0, BOX)
    # cell centroids (vertex average is inside a convex quad; it only has to be interior)
    C = 0.25 * (L[:-1, :-1] + L[1:, :-1] + L[1:, 1:] + L[:-1, 1:])  # (nx, ny, 2)

    def subdivide(A, B, cl, cr, eid, kind):
        """Extra vertices (k, 2) of edge A->B; cl / cr are the centroids of the
        cells on its left / right (None on the border)."""
        kk = stream_key(seed, kind, eid)
        k = int(np.floor(np.exp(math.log(kmin) + (math.log(kmax + 1) - math.log(kmin)) * unif(kk, 0, 1)[0])))
        k = min(max(k, kmin), kmax)
        d = B - A
        Ln = math.hypot(d[0], d[1])
        tmin = max(0.01, 10000.0 / Ln)
        m = np.arange(k)
        t = tmin + (1 - 2 * tmin) * (m + 0.5 + 0.8 * (unif(stream_key(int(kk), "t"), 0, k) - 0.5)) / k
        base = A[None, :] + t[:, None] * d[None, :]
        if cl is None or cr is None:
            return np.rint(base)
        nrm = _left_normal(d) / Ln

        def hmax(c):
            # Height limit of triangle (A, B, c) above position t of AB: a point
            # (s, h) of the edge frame lies inside iff h * sa <= h_c * s (side
            # Ac) and h * sb <= h_c * (L - s) (side Bc); a side whose base angle
            # is not acute imposes nothing.
            ac = c - A
            h_c = abs(np.dot(ac, nrm))
            sa = np.dot(ac, d) / Ln          # foot of c along AB, measured from A
            sb = Ln - sa                     # ... measured from B
            assert h_c > 0, "kite apex on the edge line"
            s = t * Ln
            lim = np.full_like(s, np.inf)
            if sa > 0:
                lim = np.minimum(lim, s * h_c / sa)
            if sb > 0:
                lim = np.minimum(lim, (Ln - s) * h_c / sb)
            return lim

        hl, hr = hmax(cl), hmax(cr)
        ks = stream_key(int(kk), "noise")
        w = unif(ks, 0, 8)
        amps = 0.2 + w[:2]
        ph = 2 * math.pi * w[2:4]
        nz = sum(amps[f] * np.sin(math.pi * (f + 1) * t + ph[f]) for f in range(2)) / amps.sum()
        nz = amp * nz + white * (2 * unif(stream_key(int(ks), "w"), 0, k) - 1)
        nz = np.clip(nz, -1.0, 1.0)
        h = 0.9 * np.where(nz >= 0, nz * hl, nz * hr)
        return np.rint(base + h[:, None] * nrm[None, :])

    # horizontal edges H(i, j): L[i, j] -> L[i+1, j]; left = cell (i, j), right = cell (i, j-1)
    H = {}
    for i in range(nx):
        for j in range(ny + 1):
            cl = C[i, j] if j < ny else None
            cr = C[i, j - 1] if j > 0 else None
            H[i, j] = subdivide(L[i, j], L[i + 1, j], cl, cr, i * (ny + 1) + j, "h")
    # vertical edges V(i, j): L[i, j] -> L[i, j+1]; left = cell (i-1, j), right = cell (i, j)
    Vt = {}
    for i in range(nx + 1):
        for j in range(ny):
            cl = C[i - 1, j] if i > 0 else None
            cr = C[i, j] if i < nx else None
            Vt[i, j] = subdivide(L[i, j], L[i, j + 1], cl, cr, i * ny + j, "v")
    parts = []
    for j in range(ny):
        for i in range(nx):
            ring = [L[i, j][None], H[i, j], L[i + 1, j][None], Vt[i + 1, j],
                    L[i + 1, j + 1][None], H[i, j + 1][::-1], L[i, j + 1][None], Vt[i, j][::-1]]
            parts.append(np.concatenate(ring, 0))
    verts, off = _rings(parts)
    assert verts.min() >= 0 and verts.max() <= BOX
    return Tessellation(verts, off, nx, ny, L.astype(np.int64))


def tessellation_shape(n_cells: int) -> tuple[int, int]:
    """nx, ny with nx * ny = n_cells and nx / ny as close to 1 as possible."""
    best = (n_cells, 1)
    for ny in range(1, int(math.isqrt(n_cells)) + 1):
        if n_cells % ny == 0:
            best = (n_cells // ny, ny)
    return best


def query_polygons(q: int, seed: int, mix: Mixture, vmin: int = 8, vmax: int = 5000,
                   mu_v: float = math.log(200.0), sig_v: float = 1.2,
                   r_med: float = 0.005, r_sig: float = 0.8, r_clip=(0.0005, 0.05),
                   notch: float = 0.2) -> tuple[np.ndarray, np.ndarray]:
    """q star-shaped query polygons: vertex count lognormal(mu_v, sig_v) clipped
    to [vmin, vmax]; centre drawn from the point mixture; mean radius lognormal
    with median r_med of the box side, clipped to r_clip; a `notch` share of the
    vertices pulled inwards to 30-60 % of the radius (concave).  The polygons
    overlap one another freely."""
    parts = []
    nv, _ = normal(stream_key(seed, "qv"), 0, q)
    nr, _ = normal(stream_key(seed, "qr"), 0, q)
    cen = mixture_points(q, seed ^ 0x5151, mix)
    for k in range(q):
        n = int(min(max(round(math.exp(mu_v + sig_v * nv[k])), vmin), vmax))
        R = min(max(r_med * math.exp(r_sig * nr[k]), r_clip[0]), r_clip[1]) * BOX
        ka = stream_key(seed, "qa", k)
        ang = 2 * math.pi * (np.arange(n) + 0.8 * (unif(ka, 0, n) - 0.5)) / n
        rad = R * (1 + 0.25 * (2 * unif(stream_key(int(ka), "r"), 0, n) - 1))
        pull = unif(stream_key(int(ka), "n"), 0, n) < notch
        rad = np.where(pull, rad * (0.3 + 0.3 * unif(stream_key(int(ka), "d"), 0, n)), rad)
        xy = np.stack([cen[k, 0] + rad * np.cos(ang), cen[k, 1] + rad * np.sin(ang)], 1)
        parts.append(np.clip(np.rint(xy), 0, BOX))
    return _rings(parts)


# ----------------------------------------------------------------------- configs
SEED_BASE = 0x2203143620


@dataclass
class Workload:
    name: str
    points: np.ndarray
    verts: np.ndarray
    ring_off: np.ndarray
    desc: str

    @property
    def n_points(self) -> int:
        return int(self.points.shape[0])

    @property
    def n_polys(self) -> int:
        return int(self.ring_off.shape[0] - 1)


def stars_join(n_points: int = 1_000_000, seed: int = SEED_BASE + 1) -> Workload:
    """Plain exact join: uniform points against 256 star polygons (16 x 16)."""
    v, o = star_polygons(seed)
    return Workload("stars256", uniform_points(n_points, seed), v, o,
                    f"{n_points} uniform points x 256 star polygons (16-64 vertices)")


def tessellation_join(n_points: int = 100_000_000, n_cells: int = 2000, seed: int = SEED_BASE + 2,
                      kmin: int = 12, kmax: int = 499, zipf_s: float | None = None) -> Workload:
    """Join at scale: mixture points against a jittered, noisily subdivided quad tessellation."""
    nx, ny = tessellation_shape(n_cells)
    t = quad_tessellation(nx, ny, seed, kmin=kmin, kmax=kmax)
    mix = make_mixture(seed, zipf_s=zipf_s)
    pts = mixture_points(n_points, seed, mix)
    return Workload(f"tess{n_cells}", pts, t.verts, t.ring_off,
                    f"{n_points} mixture points x {n_cells}-cell tessellation "
                    f"({4 + 4 * kmin}-{4 + 4 * kmax} vertices per cell)")


def batched_selection(n_points: int = 500_000_000, n_queries: int = 256, seed: int = SEED_BASE + 3) -> Workload:
    """Batched selection: mixture points queried by overlapping star polygons."""
    mix = make_mixture(seed)
    v, o = query_polygons(n_queries, seed, mix)
    return Workload(f"select{n_queries}", mixture_points(n_points, seed, mix), v, o,
                    f"{n_points} mixture points x {n_queries} query polygons (8-5000 vertices)")
