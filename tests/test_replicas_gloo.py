"""Replica placement across ranks, exercised with two gloo processes on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1412_8266_gb300.replicas import max_over_ranks, stream_range


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, per_rank, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = stream_range(rank, world, per_rank)
        t = max_over_ranks(1.5 + rank)  # each rank's "time"; the job takes the slowest
        got = [None] * world
        dist.all_gather_object(got, (first, count))
        q.put((rank, first, count, t, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_own_disjoint_ranges_and_take_the_max_time():
    world, per_rank = 2, 1 << 18
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, per_rank, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    ranges = res[0][4]
    assert ranges == [(0, per_rank), (per_rank, per_rank)]
    covered = sorted(x for f, c in ranges for x in (f, f + c))
    assert covered == [0, per_rank, per_rank, 2 * per_rank]
    assert all(r[3] == 2.5 for r in res)


def test_stream_range_rejects_bad_ranks():
    with pytest.raises(ValueError):
        stream_range(2, 2, 10)
    with pytest.raises(ValueError):
        stream_range(0, 1, 0)
    assert stream_range(0, 1, 7) == (0, 7)
    assert max_over_ranks(3.0) == 3.0
