"""GPU tests of the serving runtime (spx_server_*).

Every request's result must equal the oracle's, byte for byte, whatever the
batch it was answered in (alone, in a mix of selections and joins, through the
join's own passes per request, through the fused one-pass batch kernel,
through the plain one-request-per-launch path), with several batches in
flight, under an output budget that forces admission waits, and with requests
submitted from several threads at once.
"""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2203_14362_gb300 import datagen as g

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_14362_gb300 import spx  # noqa: E402

N_POINTS = 1_500_000 + 333  # ragged against every tile size


@pytest.fixture(scope="module")
def world():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    eng = spx.Engine(0)
    seed = g.SEED_BASE + 50
    mix = g.make_mixture(seed)
    pts = g.mixture_points(N_POINTS, seed, mix)
    dpts = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    ph = eng.load_points(dpts)
    # request index list: two tessellations (joins), four query sets (selections)
    sets = []
    for k, (nx, ny) in enumerate([(6, 5), (16, 12)]):
        t = g.quad_tessellation(nx, ny, seed + k, kmin=4, kmax=40)
        sets.append(("join", t.verts, t.ring_off))
    for k, q in enumerate([1, 5, 17, 64]):
        v, o = g.query_polygons(q, seed + 10 + k, mix, r_med=0.02, r_clip=(0.002, 0.1))
        sets.append(("select", v, o))
    handles, expect = [], []
    for kind, v, o in sets:
        gh = eng.load_polygons(v, o)
        ih = eng.build_index(gh)
        handles.append((gh, ih))
        ref = oracle.Prepared(v, o)
        pairs, counts = ref.join(pts)
        ref.close()
        if kind == "join":
            expect.append(("join", pairs, counts))
        else:
            ids, offs = oracle.group_by_polygon(pairs, counts)
            expect.append(("select", ids, offs))
    yield {"eng": eng, "ph": ph, "ix": [ih for _, ih in handles], "expect": expect, "sets": sets}
    for gh, ih in handles:
        eng.free(ih)
        eng.free(gh)
    eng.free(ph)
    eng.close()
    del dpts


def _kind(e):
    return spx.SPX_REQ_JOIN if e[0] == "join" else spx.SPX_REQ_SELECT


def _check(srv, rid, res, exp):
    assert res["status"] == spx.SPX_OK
    a, b = srv.read(rid, res)
    if exp[0] == "join":
        assert res["kind"] == spx.SPX_REQ_JOIN
        assert np.array_equal(a, exp[1])
        assert np.array_equal(b, exp[2])
    else:
        assert res["kind"] == spx.SPX_REQ_SELECT
        assert np.array_equal(a, exp[1])
        assert np.array_equal(b, exp[2])
    assert res["t_submit_ms"] <= res["t_start_ms"] <= res["t_counted_ms"] <= res["t_written_ms"] <= res["t_done_ms"]


# a fixed mixed sequence of index positions (joins are 0 and 1)
SEQ = [2, 0, 3, 4, 5, 1, 2, 2, 5, 0, 4, 3, 1, 5, 2, 0, 3, 3, 4, 1]


@pytest.mark.parametrize("cfg", [dict(max_batch=8, slots=2), dict(max_batch=3, slots=1),
                                 dict(max_batch=1, slots=3), dict(plain=True),
                                 dict(max_batch=8, slots=2, fused=True), dict(max_batch=3, slots=1, fused=True)])
def test_serve_burst_matches_oracle(world, cfg):
    srv = spx.Server(world["eng"], world["ph"], world["ix"], **cfg)
    try:
        ids = [srv.submit(_kind(world["expect"][k]), k, tag=100 + i) for i, k in enumerate(SEQ)]
        sizes = []
        for i, (rid, k) in enumerate(zip(ids, SEQ)):
            res = srv.wait(rid, 60_000)
            assert res is not None, "request did not finish"
            assert res["tag"] == 100 + i
            _check(srv, rid, res, world["expect"][k])
            sizes.append(res["batch_size"])
            srv.release(rid)
        st = srv.stats()
        assert st["completed"] == len(SEQ) and st["failed"] == 0
        assert st["batched_requests"] == len(SEQ)
        mb = 1 if cfg.get("plain") else cfg["max_batch"]
        assert max(sizes) <= mb
        if mb > 1:
            assert max(sizes) > 1  # a burst is batched
        assert st["bytes_in_use"] == 0
    finally:
        srv.close()


@pytest.mark.parametrize("fused", [False, True])
def test_serve_budget_forces_waits(world, fused):
    # a 1-byte budget: each batch runs only once nothing else is held
    srv = spx.Server(world["eng"], world["ph"], world["ix"], max_batch=1, slots=2, output_budget=1, fused=fused)
    try:
        ks = [0, 2, 1]
        ids = [srv.submit(_kind(world["expect"][k]), k) for k in ks]
        r0 = srv.wait(ids[0], 60_000)
        assert r0 is not None
        # while the first result is held, the others cannot be admitted
        assert srv.wait(ids[2], 300) is None
        _check(srv, ids[0], r0, world["expect"][ks[0]])
        srv.release(ids[0])
        # one result at a time: release each as it finishes
        pending = dict(zip(ids[1:], ks[1:]))
        for _ in range(1200):
            if not pending:
                break
            for rid in list(pending):
                res = srv.wait(rid, 50)
                if res is not None:
                    _check(srv, rid, res, world["expect"][pending.pop(rid)])
                    srv.release(rid)
        assert not pending, "requests did not finish"
        assert srv.stats()["admission_waits"] >= 1
    finally:
        srv.close()


def test_serve_threads(world):
    srv = spx.Server(world["eng"], world["ph"], world["ix"], max_batch=8, slots=2)
    errors = []

    def client(seed):
        rng = np.random.default_rng(seed)
        try:
            for _ in range(6):
                k = int(rng.integers(0, len(world["expect"])))
                rid = srv.submit(_kind(world["expect"][k]), k)
                res = srv.wait(rid, 60_000)
                assert res is not None
                _check(srv, rid, res, world["expect"][k])
                srv.release(rid)
        except Exception as e:  # reported in the main thread
            errors.append(e)

    try:
        th = [threading.Thread(target=client, args=(s,)) for s in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors, errors[0]
        assert srv.stats()["completed"] == 24
    finally:
        srv.close()


def test_serve_errors(world):
    eng = world["eng"]
    with pytest.raises(spx.SpxError):
        spx.Server(eng, world["ph"], world["ix"], max_batch=9)
    srv = spx.Server(eng, world["ph"], world["ix"])
    try:
        with pytest.raises(spx.SpxError) as ei:
            srv.submit(3, 0)
        assert ei.value.status == spx.SPX_EINVAL
        with pytest.raises(spx.SpxError) as ei:
            srv.submit(spx.SPX_REQ_JOIN, len(world["ix"]))
        assert ei.value.status == spx.SPX_EINVAL
        with pytest.raises(spx.SpxError) as ei:
            srv.wait(123456789, 0)
        assert ei.value.status == spx.SPX_EINVAL
        # destroy with work still queued finishes it first
        for k in (0, 2, 1):
            srv.submit(_kind(world["expect"][k]), k)
    finally:
        srv.close()


@pytest.mark.parametrize("fused", [False, True])
def test_serve_requests_with_their_own_polygons(world, fused):
    # every other request brings its polygons (the sets of the prebuilt
    # indexes), its index built on the device when its batch starts: the
    # results are the prebuilt ones, byte for byte
    srv = spx.Server(world["eng"], world["ph"], world["ix"], max_batch=8, slots=2, fused=fused)
    try:
        ids = []
        for i, k in enumerate(SEQ):
            kind = _kind(world["expect"][k])
            if i % 2:
                _, v, o = world["sets"][k]
                ids.append((srv.submit_polygons(kind, v, o, tag=i), k))
            else:
                ids.append((srv.submit(kind, k, tag=i), k))
        for i, (rid, k) in enumerate(ids):
            res = srv.wait(rid, 60_000)
            assert res is not None and res["tag"] == i
            _check(srv, rid, res, world["expect"][k])
            srv.release(rid)
        st = srv.stats()
        assert st["completed"] == len(SEQ) and st["failed"] == 0
        # the requests' own indexes are freed once no batch is in flight
        for _ in range(200):
            if srv.stats()["bytes_in_use"] == 0:
                break
            time.sleep(0.01)
        assert srv.stats()["bytes_in_use"] == 0
    finally:
        srv.close()


def test_serve_own_polygons_refused(world):
    srv = spx.Server(world["eng"], world["ph"], world["ix"])
    try:
        _, v, o = world["sets"][4]  # 17 query polygons
        bad = v.copy()
        bad[3, 0] = -1
        with pytest.raises(spx.SpxError) as ei:
            srv.submit_polygons(spx.SPX_REQ_SELECT, bad, o)
        assert ei.value.status == spx.SPX_EINVAL and "outside" in str(ei.value)
        off = o.copy()
        off[2], off[1] = off[1], off[2] + 1
        with pytest.raises(spx.SpxError):
            srv.submit_polygons(spx.SPX_REQ_JOIN, v, off)
        sq = np.array([[0, 0], [10, 0], [10, 10]], np.int32)
        many_v = np.tile(sq, (1025, 1))
        many_o = np.arange(0, 3 * 1026, 3, dtype=np.uint64)
        with pytest.raises(spx.SpxError):
            srv.submit_polygons(spx.SPX_REQ_SELECT, many_v, many_o)
        with pytest.raises(spx.SpxError):
            srv.submit_polygons(7, v, o)
    finally:
        srv.close()
