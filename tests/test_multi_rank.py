"""World-size-2 CPU test (gloo) of the host side of the replicated benchmark: each rank works on its own
independent sequence, the step time is the maximum over ranks, and the whole-job rate counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t = bench.max_over_ranks(1.0 + 0.25 * rank, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(rank))
        q.put((rank, t, seeds, bench.whole_job_rate(world, 1000000, t)))
    finally:
        dist.destroy_process_group()


def test_replicas_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, seeds, rate in res:
        assert t == 1.25                      # the slowest rank's time
        assert len(set(seeds)) == world       # independent problems per rank
        assert rate == pytest.approx(world * 1.0 / 1.25)


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.replica_seed(0) != bench.replica_seed(1)
    assert bench.whole_job_rate(4, 2000000, 0.5) == pytest.approx(16.0)
