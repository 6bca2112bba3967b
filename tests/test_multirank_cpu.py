"""The benchmark's multi-rank logic with world_size-2 gloo ranks on the CPU:
the job time is the slowest rank's, the rate counts every rank's replica,
and every rank simulates its own seed (replicas, no exchange step)."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        slowest = bench.max_over_ranks(1.5 + rank, device="cpu")  # rank 1 is slower
        rate = bench.job_throughput(1000, world, slowest)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(42, rank))
        dist.barrier()
        q.put((rank, slowest, rate, seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate, seeds in out:
        assert slowest == 2.5
        assert rate == pytest.approx(2 * 1000 / 2.5)
        assert len(set(seeds)) == 2 and seeds[0] == 42


def test_single_process_defaults():
    import bench

    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.job_throughput(10, 1, 2.0) == 5.0
