"""The multi-rank host logic of bench.py on CPU: two gloo ranks.

One process per GPU runs its own contiguous range of the point table
(weak scaling, index replicated); the only exchanges are the max-over-ranks
of the step time and the sum of the per-polygon counts.  Here two CPU ranks
check that the ranges partition the global table and that both reductions
give the global values.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch as t
    import torch.distributed as dist

    import bench
    from paper_2203_14362_gb300 import datagen as g
    try:
        w, r, loc = bench.dist_setup()
        assert (w, r) == (world, rank)
        bench.dist_init(w, loc, t)
        assert dist.get_backend() == "gloo"
        # max over ranks of a per-rank time
        got_max = bench.max_over_ranks(1.5 + rank, w, t)
        # sum of per-rank counts
        counts = t.tensor([rank + 1, 10 * (rank + 1), 0], dtype=t.int64)
        bench.sum_counts_over_ranks(counts, w)
        # the ranks' point ranges partition the global table
        n = 5000
        mix = g.make_mixture(123)
        mine = g.mixture_points(n, 123, mix, start=bench.shard_start(rank, n))
        parts = [t.zeros((n, 2), dtype=t.int32) for _ in range(w)]
        dist.all_gather(parts, t.from_numpy(mine))
        whole = t.cat(parts).numpy()
        ref = g.mixture_points(w * n, 123, mix)
        q.put((rank, got_max, counts.tolist(), bool(np.array_equal(whole, ref))))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent
        q.put((rank, "error", repr(e), False))


def test_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, got_max, counts, same = q.get(timeout=240)
        out[rank] = (got_max, counts, same)
    for p in procs:
        p.join(timeout=60)
    for r in range(2):
        got_max, counts, same = out[r]
        assert got_max == 2.5, out
        assert counts == [3, 30, 0], out
        assert same, out
