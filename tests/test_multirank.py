"""The benchmark's multi-rank logic (one process per GPU, weak scaling, no
collective on the data path, time = the slowest rank) on two gloo ranks on
the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        value = bench.job_value(world, 2000, 7, ms / 1e3)
        q.put((rank, ms, value, bench.rank_seed(15060603901, rank)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_job_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(world))
    # every rank sees the slowest rank's time and the same whole-job value
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == res[1][2] == pytest.approx(2 * 2000 * 7 / 0.015)
    # each rank draws its own stack
    assert res[0][3] != res[1][3]


def test_single_rank_passthrough():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 2000, 10, 2.0) == 10000.0
