"""Host logic of bench.py's N > 1 path (replicas, one process per GPU), run
as two gloo ranks on CPU: the matrices are sharded without a collective, the
slowest rank's time is taken, and the whole-job rate counts every rank's
units."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = bench.shard(10, ws, rank)
        got = [None] * ws
        dist.all_gather_object(got, mine)
        slowest = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        out.put((rank, got, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, slowest in res:
        assert sorted(i for part in got for i in part) == list(range(10))   # every matrix once
        assert set(got[0]).isdisjoint(got[1])
        assert slowest == 2.5                                                # the slower rank's time


def test_whole_job_rate_and_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(1024, 65.0) == pytest.approx(1024 / 0.065)
    assert bench.shard(5, 1, 0) == [0, 1, 2, 3, 4]
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
