"""Thin ctypes binding of libspx (include/spx.h): argument marshalling only.

Every function of the C ABI is exposed under its own name; `Engine` wraps a
context for callers that hold torch tensors or numpy arrays.  All computation
runs in libspx's CUDA kernels; there is no CPU fallback, and a missing or
unloadable library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SPX_LIB: load another build of the library (the bounds-checked flavour,
# libspx_checked.so); there is no fallback when it is missing
LIB_PATH = os.environ.get("SPX_LIB") or os.path.join(_HERE, "libspx.so")

SPX_OK, SPX_EINVAL, SPX_ENOMEM, SPX_ECUDA, SPX_ECAPACITY, SPX_ETIMEOUT, SPX_EBUSY, SPX_EKERNEL = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "SPX_OK", -1: "SPX_EINVAL", -2: "SPX_ENOMEM", -3: "SPX_ECUDA", -4: "SPX_ECAPACITY",
                -5: "SPX_ETIMEOUT", -6: "SPX_EBUSY", -7: "SPX_EKERNEL"}

EXPORTS = [
    "spx_create", "spx_destroy", "spx_last_error", "spx_load_points", "spx_load_polygons", "spx_build_index",
    "spx_index_info_get", "spx_join", "spx_join_plain", "spx_aggregate", "spx_join_host", "spx_host_index_build",
    "spx_host_index_copy", "spx_host_index_free", "spx_stats", "spx_set_phase_timing", "spx_free",
    "spx_join_plain_static", "spx_select", "spx_autotune",
    "spx_server_create", "spx_server_submit", "spx_server_submit_polygons", "spx_server_poll", "spx_server_wait", "spx_server_release",
    "spx_server_stats", "spx_server_last_error", "spx_server_destroy", "spx_server_read",
    "spx_cluster_points", "spx_points_info", "spx_aggregate_host", "spx_set_host_streaming",
    "spx_build_disk_index", "spx_build_buffer_index", "spx_host_disk_index_build", "spx_host_disk_index_copy", "spx_host_disk_index_free", "spx_host_buffer_edges_build", "spx_host_buffer_edges_copy",
    "spx_host_buffer_edges_free",
    "spx_build_disk_index_device", "spx_disk_index_arrays", "spx_build_index_device", "spx_index_arrays", "spx_host_index_validate",
    "spx_check_bounded_wait",
]

SPX_REQ_SELECT, SPX_REQ_JOIN = 1, 2


class SpxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class IndexParams(C.Structure):
    _fields_ = [("grid_log2", C.c_int), ("fp32_filter", C.c_int), ("sub_log2", C.c_int), ("reserved", C.c_int * 5)]


class IndexInfo(C.Structure):
    _fields_ = [("grid_log2", C.c_int), ("sub_log2", C.c_int), ("n_polys", C.c_uint32), ("pad", C.c_uint32),
                ("n_cells", C.c_uint64), ("n_blocks", C.c_uint64), ("n_entries", C.c_uint64),
                ("n_inside", C.c_uint64), ("n_mixed", C.c_uint64), ("n_boundary", C.c_uint64),
                ("n_edge_refs", C.c_uint64), ("device_bytes", C.c_uint64), ("build_ms", C.c_double),
                ("sum_resolved", C.c_double), ("use_sum", C.c_int), ("pad2", C.c_int),
                ("edge_grid_log2", C.c_int), ("pad3", C.c_int), ("n_edge_items", C.c_uint64)]


class TuneParams(C.Structure):
    _fields_ = [("sample_points", C.c_uint64), ("grid_min", C.c_int), ("grid_max", C.c_int), ("reps", C.c_int),
                ("fp32_filter", C.c_int), ("max_index_bytes", C.c_uint64), ("reserved", C.c_int * 4)]


class TuneTrial(C.Structure):
    _fields_ = [("grid_log2", C.c_int), ("sub_log2", C.c_int), ("ms", C.c_double), ("build_ms", C.c_double),
                ("device_bytes", C.c_uint64)]


class ServerParams(C.Structure):
    _fields_ = [("max_batch", C.c_int), ("slots", C.c_int), ("plain", C.c_int), ("fused", C.c_int),
                ("output_budget", C.c_uint64), ("reserved", C.c_int * 4)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("index", C.c_uint32), ("tag", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("kind", C.c_int), ("tag", C.c_uint64), ("total", C.c_uint64),
                ("n_polys", C.c_uint32), ("batch_size", C.c_uint32), ("pairs_dev", C.c_void_p),
                ("counts_dev", C.c_void_p), ("ids_dev", C.c_void_p), ("offsets_dev", C.c_void_p),
                ("t_submit_ms", C.c_double), ("t_start_ms", C.c_double), ("t_done_ms", C.c_double),
                ("t_counted_ms", C.c_double), ("t_written_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("batches", C.c_uint64), ("batched_requests", C.c_uint64), ("bytes_in_use", C.c_uint64),
                ("peak_bytes_in_use", C.c_uint64), ("admission_waits", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("points_scanned", C.c_uint64), ("edge_tests", C.c_uint64),
                ("fp32_escalations", C.c_uint64), ("pairs_emitted", C.c_uint64),
                ("timed_joins", C.c_uint64), ("timed_aggregates", C.c_uint64),
                ("ms_resolve", C.c_double), ("ms_scan", C.c_double), ("ms_emit", C.c_double),
                ("ms_aggregate", C.c_double), ("ms_walk", C.c_double), ("points_from_directory", C.c_uint64)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libspx.so (built by paper_2203_14362_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libspx.so not found at {path}: run paper_2203_14362_gb300.build.build() first")
    lib = C.CDLL(path)
    V, U64, U32, I = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int
    P64 = C.POINTER(C.c_uint64)
    sig = {
        "spx_create": ([I, C.POINTER(V)], I),
        "spx_destroy": ([V], None),
        "spx_last_error": ([V], C.c_char_p),
        "spx_load_points": ([V, V, U64, I, P64], I),
        "spx_load_polygons": ([V, V, V, U32, P64], I),
        "spx_build_index": ([V, U64, C.POINTER(IndexParams), P64], I),
        "spx_index_info_get": ([V, U64, C.POINTER(IndexInfo)], I),
        "spx_join": ([V, U64, U64, V, U64, V, V, P64, V], I),
        "spx_join_plain": ([V, U64, U64, V, U64, V, V, P64, V], I),
        "spx_aggregate": ([V, U64, U64, V, V], I),
        "spx_join_host": ([V, V, U64, U64, V, U64, V, P64], I),
        "spx_host_index_build": ([V, V, U32, I, I, C.POINTER(V), P64], I),
        "spx_host_index_copy": ([V, V, V, V, V], I),
        "spx_host_index_free": ([V], None),
        "spx_stats": ([V, C.POINTER(Stats), I], I),
        "spx_set_phase_timing": ([V, I], I),
        "spx_join_plain_static": ([V, U64, U64, V, U64, V, V, V], I),
        "spx_select": ([V, U64, U64, V, U64, V, P64, V], I),
        "spx_autotune": ([V, U64, U64, C.POINTER(TuneParams), C.POINTER(IndexParams), C.POINTER(TuneTrial), U32,
                          C.POINTER(U32), P64, V], I),
        "spx_server_create": ([V, U64, V, U32, C.POINTER(ServerParams), C.POINTER(V)], I),
        "spx_server_submit": ([V, C.POINTER(Request), P64], I),
        "spx_server_submit_polygons": ([V, I, V, V, U32, U64, P64], I),
        "spx_server_poll": ([V, U64, C.POINTER(Result)], I),
        "spx_server_wait": ([V, U64, C.c_double, C.POINTER(Result)], I),
        "spx_server_release": ([V, U64], I),
        "spx_server_read": ([V, U64, V, U64, V, U64], I),
        "spx_server_stats": ([V, C.POINTER(ServerStats)], I),
        "spx_server_last_error": ([V], C.c_char_p),
        "spx_server_destroy": ([V], None),
        "spx_cluster_points": ([V, U64, I, P64], I),
        "spx_build_disk_index": ([V, V, V, U32, I, P64], I),
        "spx_build_buffer_index": ([V, U64, V, I, I, P64], I),
        "spx_host_disk_index_build": ([V, V, U32, I, C.POINTER(V), P64], I),
        "spx_host_disk_index_copy": ([V, V, V], I),
        "spx_host_disk_index_free": ([V], None),
        "spx_host_buffer_edges_build": ([V, V, U32, V, I, C.POINTER(V), P64], I),
        "spx_host_buffer_edges_copy": ([V, V, V, V], I),
        "spx_host_buffer_edges_free": ([V], None),
        "spx_build_disk_index_device": ([V, V, V, U32, I, P64], I),
        "spx_disk_index_arrays": ([V, U64, V, V, P64], I),
        "spx_build_index_device": ([V, U64, C.POINTER(IndexParams), C.POINTER(U64)], I),
        "spx_index_arrays": ([V, U64, V, V, V, V, P64], I),
        "spx_check_bounded_wait": ([V, U32, V], I),
        "spx_host_index_validate": ([V, U64, V, U64, V, U64, V, U64, I, I, U32, C.c_char_p, U64], I),
        "spx_aggregate_host": ([V, V, U64, U64, V], I),
        "spx_set_host_streaming": ([V, I, I], I),
        "spx_points_info": ([V, U64, C.POINTER(V), P64, C.POINTER(I)], I),
        "spx_free": ([V, U64], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dev_ptr(t):
    """Device pointer of a torch tensor (or an int address, or None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return C.c_void_p(t)
    return C.c_void_p(t.data_ptr())


# ------------------------------------------------------------- host index build
def host_index(verts: np.ndarray, ring_off: np.ndarray, grid_log2: int = 0, sub_log2: int = 0):
    """Build the grid index on the host only (spx_host_index_build); returns a
    dict with coarse (uint32), fine (uint32), entries (E, 4) uint32, edges
    (M, 4) int32, g and sub."""
    lib = load()
    xy = np.ascontiguousarray(verts, dtype=np.int32)
    off = np.ascontiguousarray(ring_off, dtype=np.uint64)
    h = C.c_void_p()
    sizes = (C.c_uint64 * 6)()
    st = lib.spx_host_index_build(_np_ptr(xy), _np_ptr(off), off.shape[0] - 1, grid_log2, sub_log2, C.byref(h),
                                  sizes)
    if st != SPX_OK:
        raise SpxError(st, "spx_host_index_build failed")
    try:
        coarse = np.zeros(sizes[0], np.uint32)
        fine = np.zeros(max(sizes[1], 1), np.uint32)
        ent = np.zeros((sizes[2], 4), np.uint32)
        edges = np.zeros((sizes[3], 4), np.int32)
        lib.spx_host_index_copy(h, _np_ptr(coarse), _np_ptr(fine), _np_ptr(ent), _np_ptr(edges))
    finally:
        lib.spx_host_index_free(h)
    return {"coarse": coarse, "fine": fine, "entries": ent, "edges": edges, "g": int(sizes[4]), "sub": int(sizes[5])}


def validate_index(ix: dict, n_polys: int):
    """spx_host_index_validate on a host_index dict: (True, "") or (False, the
    first violation)."""
    lib = load()
    coarse = np.ascontiguousarray(ix["coarse"], np.uint32)
    fine = np.ascontiguousarray(ix["fine"], np.uint32)
    ent = np.ascontiguousarray(ix["entries"], np.uint32).reshape(-1, 4)
    edges = np.ascontiguousarray(ix["edges"], np.int32).reshape(-1, 4)
    msg = C.create_string_buffer(256)
    st = lib.spx_host_index_validate(_np_ptr(coarse), coarse.shape[0], _np_ptr(fine), fine.shape[0], _np_ptr(ent),
                                     ent.shape[0], _np_ptr(edges), edges.shape[0], ix["g"], ix["sub"], n_polys, msg,
                                     256)
    return st == SPX_OK, msg.value.decode()


def host_disk_index(centers: np.ndarray, radii: np.ndarray, grid_log2: int = 0):
    """Build the disk index on the host only (spx_host_disk_index_build);
    returns a dict with cell (uint32), entries (uint32) and g."""
    lib = load()
    cxy = np.ascontiguousarray(centers, dtype=np.int32).reshape(-1, 2)
    r = np.ascontiguousarray(radii, dtype=np.int32)
    if r.shape[0] != cxy.shape[0]:
        raise ValueError("one radius per centre")
    h = C.c_void_p()
    sizes = (C.c_uint64 * 3)()
    st = lib.spx_host_disk_index_build(_np_ptr(cxy), _np_ptr(r), cxy.shape[0], grid_log2, C.byref(h), sizes)
    if st != SPX_OK:
        raise SpxError(st, "spx_host_disk_index_build failed")
    try:
        cell = np.zeros(sizes[0], np.uint32)
        ent = np.zeros(max(sizes[1], 1), np.uint32)
        lib.spx_host_disk_index_copy(h, _np_ptr(cell), _np_ptr(ent))
    finally:
        lib.spx_host_disk_index_free(h)
    return {"cell": cell, "entries": ent, "g": int(sizes[2])}


def host_buffer_edges(verts: np.ndarray, ring_off: np.ndarray, radii: np.ndarray, grid_log2: int = 0):
    """The edge grid of a buffered-polygon index, built on the host only
    (spx_host_buffer_edges_build); returns a dict with cell_off (uint32),
    item_q (uint32, bit 31: the polygon's r-region holds the whole cell),
    item_seg ((items, 4) int32) and g."""
    lib = load()
    xy = np.ascontiguousarray(verts, dtype=np.int32).reshape(-1, 2)
    off = np.ascontiguousarray(ring_off, dtype=np.uint64)
    r = np.ascontiguousarray(radii, dtype=np.int32)
    h = C.c_void_p()
    sizes = (C.c_uint64 * 3)()
    st = lib.spx_host_buffer_edges_build(_np_ptr(xy), _np_ptr(off), off.shape[0] - 1, _np_ptr(r), grid_log2,
                                         C.byref(h), sizes)
    if st != SPX_OK:
        raise SpxError(st, "spx_host_buffer_edges_build failed")
    try:
        cell_off = np.zeros(sizes[0], np.uint32)
        q = np.zeros(max(sizes[1], 1), np.uint32)
        seg = np.zeros((max(sizes[1], 1), 4), np.int32)
        lib.spx_host_buffer_edges_copy(h, _np_ptr(cell_off), _np_ptr(q), _np_ptr(seg))
    finally:
        lib.spx_host_buffer_edges_free(h)
    return {"cell_off": cell_off, "item_q": q[:sizes[1]], "item_seg": seg[:sizes[1]], "g": int(sizes[2])}


# ------------------------------------------------------------------- the engine
class Engine:
    """One libspx context on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.ctx = C.c_void_p()
        st = self.lib.spx_create(device, C.byref(self.ctx))
        if st != SPX_OK:
            raise SpxError(st, f"spx_create(device={device}) failed")
        self.device = device

    def close(self):
        if self.ctx:
            self.lib.spx_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != SPX_OK:
            raise SpxError(st, f"{what}: {self.lib.spx_last_error(self.ctx).decode()}")

    # -- loading
    def load_points(self, xy) -> int:
        """Host numpy (N, 2) int32 (copied) or a CUDA torch tensor (borrowed)."""
        h = C.c_uint64()
        if isinstance(xy, np.ndarray):
            a = np.ascontiguousarray(xy, dtype=np.int32)
            self._check(self.lib.spx_load_points(self.ctx, _np_ptr(a), a.shape[0], 0, C.byref(h)), "spx_load_points")
        else:
            assert xy.is_cuda and xy.is_contiguous() and str(xy.dtype) == "torch.int32"
            self._check(self.lib.spx_load_points(self.ctx, _dev_ptr(xy), xy.shape[0], 1, C.byref(h)),
                        "spx_load_points")
        return h.value

    def cluster_points(self, points: int, grid_log2: int = 0) -> int:
        """spx_cluster_points: a cell-clustered copy (aggregate only)."""
        h = C.c_uint64()
        self._check(self.lib.spx_cluster_points(self.ctx, points, grid_log2, C.byref(h)), "spx_cluster_points")
        return h.value

    def points_info(self, points: int) -> dict:
        """Device address, size and clustering grid of a point table."""
        ptr, n, c = C.c_void_p(), C.c_uint64(), C.c_int()
        self._check(self.lib.spx_points_info(self.ctx, points, C.byref(ptr), C.byref(n), C.byref(c)),
                    "spx_points_info")
        return {"ptr": ptr.value or 0, "n": n.value, "cluster_log2": c.value}

    def load_polygons(self, verts: np.ndarray, ring_off: np.ndarray) -> int:
        xy = np.ascontiguousarray(verts, dtype=np.int32)
        off = np.ascontiguousarray(ring_off, dtype=np.uint64)
        h = C.c_uint64()
        self._check(self.lib.spx_load_polygons(self.ctx, _np_ptr(xy), _np_ptr(off), off.shape[0] - 1, C.byref(h)),
                    "spx_load_polygons")
        return h.value

    def build_index(self, polys: int, grid_log2: int = 0, fp32_filter: bool = True, sub_log2: int = 0,
                    on_device: bool = False) -> int:
        """spx_build_index (or, on_device, spx_build_index_device: the same
        arrays built by kernels)."""
        p = IndexParams(grid_log2, 1 if fp32_filter else 0, sub_log2)
        h = C.c_uint64()
        fn = "spx_build_index_device" if on_device else "spx_build_index"
        self._check(getattr(self.lib, fn)(self.ctx, polys, C.byref(p), C.byref(h)), fn)
        return h.value

    def index_arrays(self, index: int) -> dict:
        """spx_index_arrays: a polygon index's arrays copied to the host (the
        layout of host_index, sentinels included)."""
        sizes = (C.c_uint64 * 4)()
        self._check(self.lib.spx_index_arrays(self.ctx, index, None, None, None, None, sizes), "spx_index_arrays")
        coarse = np.zeros(sizes[0], np.uint32)
        fine = np.zeros(sizes[1], np.uint32)
        ent = np.zeros((sizes[2], 4), np.uint32)
        edges = np.zeros((sizes[3], 4), np.int32)
        self._check(self.lib.spx_index_arrays(self.ctx, index, _np_ptr(coarse), _np_ptr(fine), _np_ptr(ent),
                                              _np_ptr(edges), sizes), "spx_index_arrays")
        return {"coarse": coarse, "fine": fine, "entries": ent, "edges": edges}

    def autotune(self, points: int, polys: int, sample_points: int = 0, grid_min: int = 0, grid_max: int = 0,
                 reps: int = 0, fp32_filter: bool = True, max_index_bytes: int = 0, keep_index: bool = True,
                 stream=None):
        """spx_autotune: returns (params dict, list of trial dicts, index handle or None)."""
        tp = TuneParams(sample_points, grid_min, grid_max, reps, 1 if fp32_filter else 0, max_index_bytes)
        best = IndexParams()
        trials = (TuneTrial * 64)()
        n = C.c_uint32()
        h = C.c_uint64()
        self._check(self.lib.spx_autotune(self.ctx, points, polys, C.byref(tp), C.byref(best), trials, 64,
                                          C.byref(n), C.byref(h) if keep_index else None, _stream(stream)),
                    "spx_autotune")
        params = {"grid_log2": best.grid_log2, "sub_log2": best.sub_log2, "fp32_filter": best.fp32_filter}
        rows = [{f: getattr(trials[i], f) for f, _ in TuneTrial._fields_} for i in range(min(n.value, 64))]
        return params, rows, (h.value if keep_index else None)

    def build_disk_index(self, centers: np.ndarray, radii: np.ndarray, grid_log2: int = 0,
                         on_device: bool = False) -> int:
        """spx_build_disk_index (or, on_device, spx_build_disk_index_device):
        an index of disks for distance joins / selections."""
        c = np.ascontiguousarray(centers, dtype=np.int32).reshape(-1, 2)
        r = np.ascontiguousarray(radii, dtype=np.int32).reshape(-1)
        assert c.shape[0] == r.shape[0]
        h = C.c_uint64()
        fn = "spx_build_disk_index_device" if on_device else "spx_build_disk_index"
        self._check(getattr(self.lib, fn)(self.ctx, _np_ptr(c), _np_ptr(r), c.shape[0], grid_log2, C.byref(h)), fn)
        return h.value

    def build_buffer_index(self, polys: int, radii: np.ndarray, grid_log2: int = 0, fp32_filter: bool = True) -> int:
        """spx_build_buffer_index: polygon set `polys`, polygon q buffered by
        radii[q], for distance joins / selections / counts."""
        r = np.ascontiguousarray(radii, dtype=np.int32).reshape(-1)
        h = C.c_uint64()
        self._check(self.lib.spx_build_buffer_index(self.ctx, polys, _np_ptr(r), grid_log2, 1 if fp32_filter else 0,
                                                    C.byref(h)), "spx_build_buffer_index")
        return h.value

    def disk_index_arrays(self, index: int) -> dict:
        """spx_disk_index_arrays: a disk index's cell words and entries, copied
        to the host (the layout of host_disk_index)."""
        sizes = (C.c_uint64 * 3)()
        self._check(self.lib.spx_disk_index_arrays(self.ctx, index, None, None, sizes), "spx_disk_index_arrays")
        cell = np.zeros(sizes[0], np.uint32)
        ent = np.zeros(max(sizes[1], 1), np.uint32)
        self._check(self.lib.spx_disk_index_arrays(self.ctx, index, _np_ptr(cell), _np_ptr(ent), sizes),
                    "spx_disk_index_arrays")
        return {"cell": cell, "entries": ent[:sizes[1]], "g": int(sizes[2])}

    def index_info(self, index: int) -> dict:
        inf = IndexInfo()
        self._check(self.lib.spx_index_info_get(self.ctx, index, C.byref(inf)), "spx_index_info_get")
        return {f: getattr(inf, f) for f, _ in IndexInfo._fields_}

    def free(self, handle: int):
        self._check(self.lib.spx_free(self.ctx, handle), "spx_free")

    # -- queries (device tensors)
    def join(self, points: int, index: int, pairs, counts=None, total=None, sync: bool = True, stream=None,
             plain: bool = False):
        """pairs: int32/uint32-compatible CUDA tensor of shape (cap, 2); counts: int64 (P,);
        total: int64 (1,).  Returns the total number of pairs when sync, else None."""
        cap = 0 if pairs is None else pairs.shape[0]
        n = C.c_uint64()
        f = self.lib.spx_join_plain if plain else self.lib.spx_join
        st = f(self.ctx, points, index, _dev_ptr(pairs), cap, _dev_ptr(counts), _dev_ptr(total),
               C.byref(n) if sync else None, _stream(stream))
        if st == SPX_ECAPACITY:
            raise SpxError(st, f"join needs {n.value} pairs, capacity {cap}")
        self._check(st, "spx_join")
        return n.value if sync else None

    def select(self, points: int, index: int, ids, offsets, sync: bool = True, stream=None):
        """Batched selection: ids (int32/uint32 CUDA tensor, cap entries), offsets
        (int64 CUDA tensor, P + 1 entries).  Returns the total when sync."""
        cap = 0 if ids is None else ids.shape[0]
        n = C.c_uint64()
        st = self.lib.spx_select(self.ctx, points, index, _dev_ptr(ids), cap, _dev_ptr(offsets),
                                 C.byref(n) if sync else None, _stream(stream))
        if st == SPX_ECAPACITY:
            raise SpxError(st, f"select needs {n.value} ids, capacity {cap}")
        self._check(st, "spx_select")
        return n.value if sync else None

    def join_plain_static(self, points: int, index: int, pairs, counts, total, stream=None, cap=None):
        """spx_join_plain_static: the plain join with its scratch in libspx's
        fixed device array (no allocation in the call); asynchronous.  cap
        (default: all rows of pairs) may be smaller than the tensor."""
        rows = 0 if pairs is None else pairs.shape[0]
        cap = rows if cap is None else int(cap)
        if cap > rows:
            raise ValueError(f"cap {cap} exceeds the {rows} rows of pairs")
        self._check(self.lib.spx_join_plain_static(self.ctx, points, index, _dev_ptr(pairs), cap, _dev_ptr(counts),
                                                   _dev_ptr(total), _stream(stream)), "spx_join_plain_static")

    def aggregate(self, points: int, index: int, counts, stream=None):
        self._check(self.lib.spx_aggregate(self.ctx, points, index, _dev_ptr(counts), _stream(stream)),
                    "spx_aggregate")

    def join_host(self, xy: np.ndarray, index: int, cap: int, n_polys: int, pairs_out=None, counts_out=None):
        """End-to-end join on host arrays; returns (pairs view, counts, total)."""
        a = np.ascontiguousarray(xy, dtype=np.int32)
        pairs = pairs_out if pairs_out is not None else np.zeros((cap, 2), np.uint32)
        counts = counts_out if counts_out is not None else np.zeros(max(n_polys, 1), np.uint64)
        n = C.c_uint64()
        st = self.lib.spx_join_host(self.ctx, _np_ptr(a), a.shape[0], index, _np_ptr(pairs), cap,
                                    _np_ptr(counts), C.byref(n))
        if st == SPX_ECAPACITY:
            raise SpxError(st, f"join needs {n.value} pairs, capacity {cap}")
        self._check(st, "spx_join_host")
        return pairs[:n.value], counts[:n_polys], n.value

    def aggregate_host(self, xy: np.ndarray, index: int, n_polys: int, counts_out=None):
        """Count-only aggregation over a host table, streamed through the device."""
        a = np.ascontiguousarray(xy, dtype=np.int32)
        counts = counts_out if counts_out is not None else np.zeros(max(n_polys, 1), np.uint64)
        self._check(self.lib.spx_aggregate_host(self.ctx, _np_ptr(a), a.shape[0], index, _np_ptr(counts)),
                    "spx_aggregate_host")
        return counts[:n_polys]

    def set_host_streaming(self, mode: int = 0, slice_log2: int = 0):
        self._check(self.lib.spx_set_host_streaming(self.ctx, mode, slice_log2), "spx_set_host_streaming")

    def check_bounded_wait(self, tries: int = 1000, stream=None) -> int:
        """spx_check_bounded_wait: the status of a bounded wait that runs out
        (SPX_ETIMEOUT expected)."""
        return self.lib.spx_check_bounded_wait(self.ctx, tries, _stream(stream))

    def set_phase_timing(self, on: bool):
        self._check(self.lib.spx_set_phase_timing(self.ctx, 1 if on else 0), "spx_set_phase_timing")

    def stats(self, reset: bool = False) -> dict:
        s = Stats()
        self._check(self.lib.spx_stats(self.ctx, C.byref(s), 1 if reset else 0), "spx_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}


class Server:
    """spx_server_*: a serving thread over one resident point table and a list
    of indexes (requests name an index by its position in that list)."""

    def __init__(self, eng: Engine, points: int, indexes, max_batch: int = 0, slots: int = 0, plain: bool = False,
                 output_budget: int = 0, fused: bool = False):
        self.lib = eng.lib
        arr = (C.c_uint64 * max(len(indexes), 1))(*indexes)
        prm = ServerParams(max_batch, slots, 1 if plain else 0, 1 if fused else 0, output_budget)
        h = C.c_void_p()
        st = self.lib.spx_server_create(eng.ctx, points, arr, len(indexes), C.byref(prm), C.byref(h))
        if st != SPX_OK:
            raise SpxError(st, f"spx_server_create: {self.lib.spx_last_error(eng.ctx).decode()}")
        self.h = h

    def _check(self, st: int, what: str):
        if st != SPX_OK:
            raise SpxError(st, f"{what}: {self.lib.spx_server_last_error(self.h).decode()}")

    def submit(self, kind: int, index: int, tag: int = 0) -> int:
        rid = C.c_uint64()
        self._check(self.lib.spx_server_submit(self.h, C.byref(Request(kind, index, tag)), C.byref(rid)),
                    "spx_server_submit")
        return rid.value

    def submit_polygons(self, kind: int, verts: np.ndarray, ring_off: np.ndarray, tag: int = 0) -> int:
        """A request with its own polygons: their index is built on the device
        when its batch starts."""
        xy = np.ascontiguousarray(verts, dtype=np.int32).reshape(-1, 2)
        off = np.ascontiguousarray(ring_off, dtype=np.uint64)
        rid = C.c_uint64()
        self._check(self.lib.spx_server_submit_polygons(self.h, kind, _np_ptr(xy), _np_ptr(off), off.shape[0] - 1, tag,
                                                        C.byref(rid)), "spx_server_submit_polygons")
        return rid.value

    def wait(self, rid: int, timeout_ms: float = -1.0):
        """Result dict, or None while the request is pending after timeout_ms."""
        r = Result()
        st = self.lib.spx_server_wait(self.h, rid, timeout_ms, C.byref(r))
        if st == SPX_EBUSY:
            return None
        self._check(st, "spx_server_wait")
        return {f: getattr(r, f) for f, _ in Result._fields_}

    def poll(self, rid: int):
        return self.wait(rid, 0.0)

    def release(self, rid: int):
        self._check(self.lib.spx_server_release(self.h, rid), "spx_server_release")

    def read(self, rid: int, result: dict):
        """Host copies of a finished result: (pairs (total, 2) uint32, counts) for
        a join, (ids, offsets) for a selection."""
        n, P = result["total"], result["n_polys"]
        if result["kind"] == SPX_REQ_JOIN:
            a, b = np.empty((n, 2), np.uint32), np.empty(P, np.uint64)
        else:
            a, b = np.empty(n, np.uint32), np.empty(P + 1, np.uint64)
        self._check(self.lib.spx_server_read(self.h, rid, _np_ptr(a), a.nbytes, _np_ptr(b), b.nbytes),
                    "spx_server_read")
        return a, b

    def stats(self) -> dict:
        s = ServerStats()
        self._check(self.lib.spx_server_stats(self.h, C.byref(s)), "spx_server_stats")
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            self.lib.spx_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream(stream):
    if stream is None:
        try:
            import torch
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)
