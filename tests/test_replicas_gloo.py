"""Host logic of bench.py's N > 1 path (replicas, one process per GPU), run
as two gloo ranks on CPU: the matrices are sharded without a collective,
balanced by their n^3 work, the slowest rank's time is taken, and the
whole-job rate counts every rank's units. This path is not measured on GPUs:
every run here has one GPU."""
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
        from paper_2203_10879_gb300 import inputs
        sizes = [int(x) for x in inputs.batch_sizes(1024)]
        mine = bench.shard(sizes, ws, rank)
        got = [None] * ws
        dist.all_gather_object(got, mine)
        slowest = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        out.put((rank, got, slowest, sizes))
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
    for rank, got, slowest, sizes in res:
        assert sorted(i for part in got for i in part) == list(range(1024))   # every matrix once
        assert set(got[0]).isdisjoint(got[1])
        assert slowest == 2.5                                                  # the slower rank's time
        # balanced by work: the ranks' sums of n^3 differ by at most one matrix's n^3
        work = [sum(float(sizes[i]) ** 3 for i in part) for part in got]
        assert abs(work[0] - work[1]) <= max(float(x) ** 3 for x in sizes)
        assert max(work) / min(work) <= 1.01


def test_whole_job_rate_and_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(1024, 65.0) == pytest.approx(1024 / 0.065)
    assert bench.shard(5, 1, 0) == [0, 1, 2, 3, 4]
    # equal sizes: dealt round-robin; unequal: the largest first, each to the lightest rank
    assert bench.shard(4, 2, 0) == [0, 2] and bench.shard(4, 2, 1) == [1, 3]
    assert bench.shard([512, 32, 32, 400, 300], 2, 0) == [0]
    assert bench.shard([512, 32, 32, 400, 300], 2, 1) == [1, 2, 3, 4]
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
