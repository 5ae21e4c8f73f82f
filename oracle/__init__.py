"""CPU oracle for the exact point-in-polygon join, selection and count.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg and reference arm may import this package.  The library never calls it, and it
shares no code with the CUDA path.  The arithmetic lives in `pip_oracle.c`
(plain C, exact int64); this module compiles it with gcc and marshals numpy
arrays.  See the header of `pip_oracle.c` for the definition it computes
(SPADE §5.2 selection / join / aggregation, §4.3 exact boundary tests, §7
intersection = containment for points), and of the distance join with disks
(§5.2 "Distance-Based Queries": distance(p, c) <= r, exact in int64).

Every function here is pinned by tests against facts that do not come from the
oracle itself (brute force with an independent formulation, closed forms for
rectangles, the tessellation invariant, additivity over triangulations).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pip_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pip_oracle.c into liboracle.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def load(path: str | None = None):
    """Load (building first if needed) the oracle shared library."""
    global _lib
    with _lock:
        if path is not None:
            return _bind(C.CDLL(path))
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
        return _lib


def _bind(lib):
    P = C.c_void_p
    lib.oracle_point_in_ring.argtypes = [C.c_int32, C.c_int32, P, C.c_uint64]
    lib.oracle_point_in_ring.restype = C.c_int
    lib.oracle_join_pure.argtypes = [P, C.c_uint64, P, P, C.c_uint32, P, C.c_uint64, P]
    lib.oracle_join_pure.restype = C.c_uint64
    lib.oracle_prepare.argtypes = [P, P, C.c_uint32]
    lib.oracle_prepare.restype = P
    lib.oracle_free.argtypes = [P]
    lib.oracle_free.restype = None
    lib.oracle_join_fast.argtypes = [P, P, C.c_uint64, P, C.c_uint64, P, C.c_int]
    lib.oracle_join_fast.restype = C.c_uint64
    lib.oracle_disk_join.argtypes = [P, C.c_uint64, P, P, C.c_uint32, P, C.c_uint64, P]
    lib.oracle_disk_join.restype = C.c_uint64
    lib.oracle_near_ring.argtypes = [C.c_int32, C.c_int32, P, C.c_uint64, C.c_int32]
    lib.oracle_near_ring.restype = C.c_int
    lib.oracle_buffer_join.argtypes = [P, C.c_uint64, P, P, C.c_uint32, P, P, C.c_uint64, P, C.c_int]
    lib.oracle_buffer_join.restype = C.c_uint64
    return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _prep(points, verts, ring_off):
    pts = np.ascontiguousarray(points, dtype=np.int32).reshape(-1, 2)
    xy = np.ascontiguousarray(verts, dtype=np.int32).reshape(-1, 2)
    off = np.ascontiguousarray(ring_off, dtype=np.uint64)
    return pts, xy, off


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def point_in_ring(px: int, py: int, ring: np.ndarray, lib=None) -> bool:
    """inside(p, R) for one ring, every edge (the definition itself)."""
    lib = lib or load()
    r = np.ascontiguousarray(ring, dtype=np.int32).reshape(-1, 2)
    return bool(lib.oracle_point_in_ring(int(px), int(py), _ptr(r), r.shape[0]))


def join_pure(points, verts, ring_off, lib=None):
    """(pairs (M, 2) uint32 sorted by (point id, polygon id), counts (P,) uint64),
    testing every edge of every polygon for every point."""
    lib = lib or load()
    pts, xy, off = _prep(points, verts, ring_off)
    P = off.shape[0] - 1
    counts = np.zeros(max(P, 1), dtype=np.uint64)
    total = lib.oracle_join_pure(_ptr(pts), pts.shape[0], _ptr(xy), _ptr(off), P, None, 0, _ptr(counts))
    pairs = np.zeros((max(total, 1), 2), dtype=np.uint32)
    lib.oracle_join_pure(_ptr(pts), pts.shape[0], _ptr(xy), _ptr(off), P, _ptr(pairs), total, _ptr(counts))
    return pairs[:total], counts[:P]


def disk_join(points, centers, radii, lib=None):
    """Distance join (SPADE §5.2 "Distance-Based Queries"): pairs (M, 2) uint32
    (point id, disk id) with (px - cx)^2 + (py - cy)^2 <= r^2, sorted, and
    counts (Q,) uint64.  Every disk is tested for every point."""
    lib = lib or load()
    pts = np.ascontiguousarray(points, dtype=np.int32).reshape(-1, 2)
    cxy = np.ascontiguousarray(centers, dtype=np.int32).reshape(-1, 2)
    r = np.ascontiguousarray(radii, dtype=np.int32).reshape(-1)
    Q = cxy.shape[0]
    assert r.shape[0] == Q and (Q == 0 or (r.min() >= 0 and r.max() < (1 << 30)))
    counts = np.zeros(max(Q, 1), dtype=np.uint64)
    total = lib.oracle_disk_join(_ptr(pts), pts.shape[0], _ptr(cxy), _ptr(r), Q, None, 0, _ptr(counts))
    pairs = np.zeros((max(total, 1), 2), dtype=np.uint32)
    lib.oracle_disk_join(_ptr(pts), pts.shape[0], _ptr(cxy), _ptr(r), Q, _ptr(pairs), total, _ptr(counts))
    return pairs[:total], counts[:Q]


def near_ring(px: int, py: int, ring: np.ndarray, r: int, lib=None) -> bool:
    """Is (px, py) within distance r of an edge (closed segment) of the ring?"""
    lib = lib or load()
    rg = np.ascontiguousarray(ring, dtype=np.int32).reshape(-1, 2)
    return bool(lib.oracle_near_ring(int(px), int(py), _ptr(rg), rg.shape[0], int(r)))


def buffer_join(points, verts, ring_off, radii, threads: int | None = None, lib=None):
    """Buffered-polygon join (SPADE §4.2 distance canvases, §5.2 distance
    queries): pairs (M, 2) uint32 (point id, polygon id), sorted, of the points
    inside polygon q or within distance radii[q] of one of its edges, and
    counts (P,) uint64.  Every edge of every polygon whose bbox grown by r
    reaches the point is tested."""
    lib = lib or load()
    pts, xy, off = _prep(points, verts, ring_off)
    P = off.shape[0] - 1
    r = np.ascontiguousarray(radii, dtype=np.int32).reshape(-1)
    assert r.shape[0] == P and (P == 0 or (r.min() >= 0 and r.max() < (1 << 30)))
    th = threads or default_threads()
    counts = np.zeros(max(P, 1), dtype=np.uint64)
    total = lib.oracle_buffer_join(_ptr(pts), pts.shape[0], _ptr(xy), _ptr(off), P, _ptr(r), None, 0, _ptr(counts), th)
    pairs = np.zeros((max(total, 1), 2), dtype=np.uint32)
    lib.oracle_buffer_join(_ptr(pts), pts.shape[0], _ptr(xy), _ptr(off), P, _ptr(r), _ptr(pairs), total,
                           _ptr(counts), th)
    return pairs[:total], counts[:P]


class Prepared:
    """Fast-mode structures (bbox, y-slabs, bucket grid) for one polygon set."""

    def __init__(self, verts, ring_off, lib=None):
        self.lib = lib or load()
        _, self.xy, self.off = _prep(np.zeros((0, 2), np.int32), verts, ring_off)
        self.P = self.off.shape[0] - 1
        self.h = self.lib.oracle_prepare(_ptr(self.xy), _ptr(self.off), self.P)
        if not self.h:
            raise MemoryError("oracle_prepare failed")

    def close(self):
        if self.h:
            self.lib.oracle_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def join(self, points, threads: int | None = None, want_pairs: bool = True):
        """(pairs, counts) like join_pure, through the exact shortcuts s1-s3."""
        pts = np.ascontiguousarray(points, dtype=np.int32).reshape(-1, 2)
        threads = threads or default_threads()
        counts = np.zeros(max(self.P, 1), dtype=np.uint64)
        if not want_pairs:
            total = self.lib.oracle_join_fast(self.h, _ptr(pts), pts.shape[0], None, 0, _ptr(counts), threads)
            return None, counts[:self.P], int(total)
        # size the pair buffer from the counts of a first pass (the oracle stays two-pass and simple)
        total = self.lib.oracle_join_fast(self.h, _ptr(pts), pts.shape[0], None, 0, _ptr(counts), threads)
        pairs = np.zeros((max(total, 1), 2), dtype=np.uint32)
        self.lib.oracle_join_fast(self.h, _ptr(pts), pts.shape[0], _ptr(pairs), total, _ptr(counts), threads)
        return pairs[:total], counts[:self.P]

    def counts(self, points, threads: int | None = None):
        """Per-polygon counts only (aggregation without materialising pairs)."""
        return self.join(points, threads, want_pairs=False)[1]

    def select(self, points, threads: int | None = None):
        """(ids, offsets): the ascending point-id list of query q is
        ids[offsets[q]:offsets[q + 1]]."""
        pairs, counts = self.join(points, threads)
        return group_by_polygon(pairs, counts)


def group_by_polygon(pairs: np.ndarray, counts: np.ndarray):
    """Selection lists from join pairs: a stable sort by polygon id keeps the
    ascending point-id order inside each list."""
    order = np.argsort(pairs[:, 1], kind="stable")
    offsets = np.zeros(counts.shape[0] + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(counts)
    return pairs[order, 0].copy(), offsets


def join_fast(points, verts, ring_off, threads: int | None = None):
    p = Prepared(verts, ring_off)
    try:
        return p.join(points, threads)
    finally:
        p.close()
