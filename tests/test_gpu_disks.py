"""GPU parity of the distance queries (spx_build_disk_index with spx_join,
spx_select, spx_aggregate) against the oracle's distance join, byte for byte."""
import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import datagen as g

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_14362_gb300 import spx  # noqa: E402

LATTICE_IN_DISC = [1, 5, 13, 29, 49, 81, 113, 149, 197, 253, 317]


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e = spx.Engine(0)
    yield e
    e.close()


@pytest.fixture(scope="module")
def data():
    seed = g.SEED_BASE + 95
    mix = g.make_mixture(seed)
    pts = g.mixture_points(1_500_000 + 77, seed, mix)
    bad = np.array([[-1, 3], [3, -1], [1 << 30, 0], [-(1 << 31), (1 << 31) - 1]], np.int32)
    pts = np.concatenate([pts[:500], bad, pts[500:]])  # unchecked device table: outside points in no disk
    rng = np.random.default_rng(seed)
    Q = 100
    centers = pts[rng.integers(0, pts.shape[0], Q)].astype(np.int64)
    centers = np.clip(centers, 0, 1 << 30)
    radii = np.exp(rng.normal(np.log(2e6), 1.0, Q)).astype(np.int64)
    radii[:3] = [0, (1 << 30) - 1, 5]
    centers[2] = [0, 0]  # a disk at the corner reaches outside the box
    centers = centers.astype(np.int32)
    radii = np.clip(radii, 0, (1 << 30) - 1).astype(np.int32)
    want_p, want_c = oracle.disk_join(pts, centers, radii)
    return pts, centers, radii, want_p, want_c


@pytest.mark.parametrize("grid,on_device", [(0, False), (6, False), (11, False), (13, False), (0, True), (11, True)])
def test_disk_join_select_aggregate(eng, data, grid, on_device):
    pts, centers, radii, want_p, want_c = data
    Q = centers.shape[0]
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    ph = eng.load_points(dpts)
    ih = eng.build_disk_index(centers, radii, grid, on_device=on_device)
    try:
        info = eng.index_info(ih)
        assert info["n_polys"] == Q and (grid == 0 or info["grid_log2"] == grid)
        pairs = torch.full((want_p.shape[0] + 7, 2), -1, dtype=torch.int32, device="cuda")
        counts = torch.zeros(Q, dtype=torch.int64, device="cuda")
        n = eng.join(ph, ih, pairs, counts)
        assert n == want_p.shape[0]
        assert np.array_equal(pairs[:n].cpu().numpy().view(np.uint32), want_p)
        assert np.array_equal(counts.cpu().numpy().view(np.uint64), want_c)
        ids = torch.empty(want_p.shape[0] + 1, dtype=torch.int32, device="cuda")
        offs = torch.zeros(Q + 1, dtype=torch.int64, device="cuda")
        assert eng.select(ph, ih, ids, offs) == want_p.shape[0]
        wi, wo = oracle.group_by_polygon(want_p, want_c)
        assert np.array_equal(ids[:n].cpu().numpy().view(np.uint32), wi)
        assert np.array_equal(offs.cpu().numpy().view(np.uint64), wo)
        c2 = torch.zeros(Q, dtype=torch.int64, device="cuda")
        eng.aggregate(ph, ih, c2)
        torch.cuda.synchronize()
        assert np.array_equal(c2.cpu().numpy().view(np.uint64), want_c)
        # capacity: the two-call pattern
        small = torch.empty((10, 2), dtype=torch.int32, device="cuda")
        with pytest.raises(spx.SpxError) as ei:
            eng.join(ph, ih, small)
        assert ei.value.status == spx.SPX_ECAPACITY
    finally:
        eng.free(ih)
        eng.free(ph)
        del dpts


def test_disk_lattice_counts(eng):
    h, c = 1024, 1 << 29
    ij = np.array([(i, j) for i in range(-12, 13) for j in range(-12, 13)], np.int64)
    pts = (c + h * ij).astype(np.int32)
    centers = np.array([[c, c]] * len(LATTICE_IN_DISC), np.int32)
    radii = np.array([h * r for r in range(len(LATTICE_IN_DISC))], np.int32)
    ph = eng.load_points(pts)
    for grid in (0, 13, 3):
        ih = eng.build_disk_index(centers, radii, grid)
        counts = torch.zeros(len(LATTICE_IN_DISC), dtype=torch.int64, device="cuda")
        eng.aggregate(ph, ih, counts)
        torch.cuda.synchronize()
        assert counts.cpu().tolist() == LATTICE_IN_DISC
        eng.free(ih)
    eng.free(ph)


def test_disk_index_errors(eng):
    c = np.array([[5, 5]], np.int32)
    with pytest.raises(spx.SpxError):
        eng.build_disk_index(np.array([[-1, 5]], np.int32), np.array([3], np.int32))
    with pytest.raises(spx.SpxError):
        eng.build_disk_index(c, np.array([1 << 30], np.int32))
    with pytest.raises(spx.SpxError):
        eng.build_disk_index(c, np.array([-2], np.int32))
    pts = g.uniform_points(1000, 3)
    ph = eng.load_points(pts)
    ih = eng.build_disk_index(c, np.array([100], np.int32))
    try:
        with pytest.raises(spx.SpxError):
            eng.join_host(pts, ih, cap=10, n_polys=1)
        with pytest.raises(spx.SpxError):
            spx.Server(eng, ph, [ih])
        many = eng.build_disk_index(np.repeat(c, 1025, axis=0), np.full(1025, 10, np.int32))
        ids = torch.empty(10, dtype=torch.int32, device="cuda")
        offs = torch.zeros(1026, dtype=torch.int64, device="cuda")
        with pytest.raises(spx.SpxError):
            eng.select(ph, many, ids, offs)
        eng.free(many)
    finally:
        eng.free(ih)
        eng.free(ph)


def test_disk_counts_in_global_memory_and_deep_overlaps(eng):
    # 12000 small disks (more than the 11776 counters kept in shared memory:
    # per-disk counts go to global memory) plus 1100 disks around one centre
    # (points near it lie in more than 1022 disks: the pass-1 result cannot
    # carry the count, so the write pass counts again)
    rng = np.random.default_rng(g.SEED_BASE + 96)
    c = 1 << 29
    pts = np.concatenate([rng.integers(0, 1 << 30, (60_000, 2)),
                          c + rng.integers(-(1 << 23), 1 << 23, (3000 + 13, 2))]).astype(np.int32)
    rng.shuffle(pts)
    n = pts.shape[0]
    deep = np.column_stack([c + rng.integers(-1000, 1000, 1100), c + rng.integers(-1000, 1000, 1100)])
    small = rng.integers(0, (1 << 30) + 1, (12000, 2))
    centers = np.concatenate([small[:6000], deep, small[6000:]]).astype(np.int32)
    radii = np.concatenate([rng.integers(1 << 20, 1 << 23, 6000), rng.integers(1 << 24, 1 << 25, 1100),
                            rng.integers(0, 1 << 23, 6000)]).astype(np.int32)
    Q = centers.shape[0]
    want_p, want_c = oracle.disk_join(pts, centers, radii)
    per_point = np.bincount(want_p[:, 0].astype(np.int64), minlength=n)
    assert per_point.max() > 1022  # the case is reached
    dpts = torch.from_numpy(pts).cuda()
    ph = eng.load_points(dpts)
    try:
        for grid in (0, 9):
            ih = eng.build_disk_index(centers, radii, grid)
            pairs = torch.empty((want_p.shape[0] + 3, 2), dtype=torch.int32, device="cuda")
            counts = torch.zeros(Q, dtype=torch.int64, device="cuda")
            m = eng.join(ph, ih, pairs, counts)
            assert m == want_p.shape[0]
            assert np.array_equal(pairs[:m].cpu().numpy().view(np.uint32), want_p)
            assert np.array_equal(counts.cpu().numpy().view(np.uint64), want_c)
            c2 = torch.zeros(Q, dtype=torch.int64, device="cuda")
            eng.aggregate(ph, ih, c2)
            torch.cuda.synchronize()
            assert np.array_equal(c2.cpu().numpy().view(np.uint64), want_c)
            eng.free(ih)
    finally:
        eng.free(ph)
        del dpts


def _same_index(eng, centers, radii, grid):
    """The device build's arrays and sizes equal the host build's, byte for byte."""
    host = spx.host_disk_index(centers, radii, grid)
    a = eng.build_disk_index(centers, radii, grid, on_device=False)
    b = eng.build_disk_index(centers, radii, grid, on_device=True)
    try:
        da, db = eng.disk_index_arrays(a), eng.disk_index_arrays(b)
        ia, ib = eng.index_info(a), eng.index_info(b)
    finally:
        eng.free(b)
        eng.free(a)
    assert da["g"] == db["g"] == host["g"]
    assert np.array_equal(da["cell"], host["cell"]) and np.array_equal(da["entries"], host["entries"])
    assert np.array_equal(db["cell"], host["cell"]), "device cell words differ"
    assert np.array_equal(db["entries"], host["entries"]), "device entries differ"
    for k in ("n_cells", "n_entries", "n_inside", "n_boundary", "device_bytes"):
        assert ia[k] == ib[k], k


@pytest.mark.parametrize("grid", [0, 1, 3, 8, 11, 13])
def test_device_disk_index_build_equals_host(eng, grid):
    from test_disk_index_host import crafted, disk_set
    centers, radii = disk_set(0xD15C0 + grid)
    if grid >= 3:
        cc, cr, _ = crafted(0xC0 + grid, grid)
        centers = np.concatenate([centers, cc.astype(np.int32)])
        radii = np.concatenate([radii, cr.astype(np.int32)])
    _same_index(eng, centers, radii, grid)


def test_device_disk_index_build_edge_cases(eng):
    # no disks; one zero-radius disk on the box's far corner (no cell); a disk
    # covering the whole box; 1100 deep overlaps plus 12000 small disks
    _same_index(eng, np.zeros((0, 2), np.int32), np.zeros(0, np.int32), 5)
    _same_index(eng, np.array([[1 << 30, 1 << 30]], np.int32), np.array([0], np.int32), 7)
    _same_index(eng, np.array([[1 << 29, 1 << 29]], np.int32), np.array([(1 << 30) - 1], np.int32), 6)
    rng = np.random.default_rng(g.SEED_BASE + 97)
    c = 1 << 29
    deep = np.column_stack([c + rng.integers(-1000, 1000, 1100), c + rng.integers(-1000, 1000, 1100)])
    small = rng.integers(0, (1 << 30) + 1, (12000, 2))
    centers = np.concatenate([small, deep]).astype(np.int32)
    radii = np.concatenate([rng.integers(0, 1 << 23, 12000), rng.integers(1 << 24, 1 << 25, 1100)]).astype(np.int32)
    _same_index(eng, centers, radii, 9)
    _same_index(eng, centers, radii, 0)

