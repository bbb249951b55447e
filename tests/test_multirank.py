"""Host-side logic of the N > 1 path (replicas only): two gloo ranks on the CPU.

Each rank solves its own seeded instance, so the only exchange is the
aggregation of the timed region after it ends: the slowest rank's time and the
sum of the iterations of all ranks."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.timeout(300) if hasattr(pytest.mark, "timeout") else []


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        t, it = bench.aggregate(ws, 1.0 + 0.5 * rank, 100 * (rank + 1), "cpu")
        out.put((rank, t, it))
    finally:
        dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=240) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # max over ranks of the time, sum over ranks of the work
    assert res == [(0, 1.5, 300), (1, 1.5, 300)]


def test_aggregate_single_rank_is_identity():
    import bench
    assert bench.aggregate(1, 2.5, 7, "cpu") == (2.5, 7)


def test_replica_instances_are_distinct_and_reproducible():
    import argparse
    import bench
    a = argparse.Namespace(n=3000, m=1500)
    i0, i1, i0b = bench.make_instance(a, 0), bench.make_instance(a, 1), bench.make_instance(a, 0)
    assert i0["Q"].shape == (3000, 3000) and i0["A"].shape == (1500, 3000)
    assert np.array_equal(i0["Q"].data, i0b["Q"].data) and np.array_equal(i0["A"].indices, i0b["A"].indices)
    assert not np.array_equal(i0["c"], i1["c"])


def _batch_worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        from paper_2609_19557_gb300 import instances as I
        mine = bench.batch_shard(6, ws, rank)
        part = I.batched_set(2, count=6, n_lo=1000, n_hi=1400, n_median=1100, sigma=0.3, only=mine)
        sizes = [b["Q"].shape[0] for b in part]
        wall, solved, inner = bench.batch_totals(ws, 2.0 + rank, len(part) - rank, 1000 * (rank + 1), "cpu")
        out.put((rank, mine, sizes, wall, solved, inner))
    finally:
        dist.destroy_process_group()


def test_batch_sharded_by_problem_two_gloo_ranks():
    """The batched form shards by problem: the ranks' positions partition the
    batch, each rank builds exactly its positions of the whole batch, and the
    totals are the slowest rank's wall time and the sums of the counts."""
    import torch.multiprocessing as mp
    from paper_2609_19557_gb300 import instances as I
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_batch_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=240) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = [b["Q"].shape[0] for b in I.batched_set(2, count=6, n_lo=1000, n_hi=1400, n_median=1100, sigma=0.3)]
    assert sorted(res[0][1] + res[1][1]) == list(range(6))
    for rank, mine, sizes, wall, solved, inner in res:
        assert sizes == [whole[k] for k in mine]
        assert wall == 3.0 and solved == 3 + 2 and inner == 3000
