"""The multi-GPU run's host side with two gloo ranks on CPU: query sharding,
the max-over-ranks timing, and results gathered in rank order.  Each rank's
scan is stood in for by the oracle (the GPU is not needed for this logic);
the gathered result must equal one process over the whole batch."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1811_11076_gb300.shard import gather_results, max_over_ranks, query_shard
from synthdata import make_workload


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, per_rank, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        w = make_workload(n_series=150, n_queries=per_rank * world, d=2, length=24, n_classes=4,
                          seed=21)
        (p0, p1), q_off = query_shard(w.q_off, rank, world, per_rank)
        ids, dist_ = oracle.knn(w.db, w.db_off, w.q[p0:p1], q_off, band=0.2, kind=0, k=3)
        gi, gd = gather_results(ids, dist_)
        slowest = max_over_ranks(1.0 + rank)
        if rank == 0:
            out.put((gi, gd, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_gather():
    world, per_rank = 2, 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, per_rank, q)) for r in range(world)]
    for p in procs:
        p.start()
    gi, gd, slowest = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    w = make_workload(n_series=150, n_queries=per_rank * world, d=2, length=24, n_classes=4,
                      seed=21)
    ids, dist_ = oracle.knn(w.db, w.db_off, w.q, w.q_off, band=0.2, kind=0, k=3)
    assert (gi == ids).all() and np.allclose(gd, dist_)
    assert slowest == 2.0


def test_query_shard_covers_the_batch_once():
    q_off = np.concatenate([[0], np.cumsum(np.arange(1, 13))]).astype(np.int64)  # 12 queries
    seen = []
    for r in range(4):
        (p0, p1), off = query_shard(q_off, r, 4, 3)
        assert off[0] == 0 and off[-1] == p1 - p0
        seen.append((p0, p1))
    assert seen[0][0] == 0 and seen[-1][1] == q_off[-1]
    assert all(a[1] == b[0] for a, b in zip(seen, seen[1:]))
    with pytest.raises(ValueError):
        query_shard(q_off, 4, 4, 3)
    with pytest.raises(ValueError):
        query_shard(q_off, 0, 5, 3)
    assert max_over_ranks(3.5) == 3.5          # no process group: the value itself


def _rank_fails(rank, world, port, out):
    """Rank 1's step fails on the host (an exception before its collective);
    rank 0 must learn of it from its next host collective, which ends with an
    error within the process group's short timeout instead of waiting."""
    import datetime
    import time
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        # the failing step: no collective is in flight when the rank leaves
        raise SystemExit(3)
    t0 = time.time()
    try:
        max_over_ranks(1.0)
        out.put(("no error", time.time() - t0))
    except Exception as exc:  # the peer's exit surfaces here
        out.put((type(exc).__name__, time.time() - t0))


def test_a_failed_rank_is_reported_not_waited_for():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_fails, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    kind, waited = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert procs[1].exitcode == 3
    assert kind != "no error"
    assert waited < 60
