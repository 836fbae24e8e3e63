"""The multi-rank host logic of the benchmark on CPU: two gloo ranks, the
slowest rank's time taken by every rank, the whole-job rate of weak-scaled
replicas, and the reference arm, which runs on rank 0 only."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
        rate = bench.whole_job_rate(1000.0, world, got)
        # the reference arm does nothing on ranks other than 0
        ran = None
        if rank != 0:
            class A:
                steps, warmup = 1, 0
            bench.run_reference(A(), rank, world)
            ran = "skipped"
        dist.barrier()
        q.put((rank, got, rate, ran))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert [r[2] for r in res] == [2000.0 / 15.0] * 2
    assert res[1][3] == "skipped"


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.whole_job_rate(100.0, 1, 2.0) == 50.0
