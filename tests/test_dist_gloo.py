"""The multi-rank host path (replicas / independent-problem shards) on two
gloo ranks on the CPU: shards partition the problems, the timing reduction
takes the slowest rank and the job rate counts every rank's units."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1404_4161_gb300 import dist as D


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, lr = D.env()
        mine = D.shard(64, r, ws)
        got = [None] * ws
        dist.all_gather_object(got, mine)
        seconds = 1.0 + r  # rank 1 is slower
        spu, t, total = D.whole_job_seconds_per_unit(len(mine), seconds)
        dist.barrier()
        out[rank] = (got, t, total, spu)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        shards, t, total, spu = res[r]
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(64))
        assert t == 2.0 and total == 64.0
        assert abs(spu - 2.0 / 64) < 1e-15


def test_shard_single_rank_and_errors():
    assert D.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert D.shard(5, 1, 2) == [1, 3]
    with pytest.raises(ValueError):
        D.shard(5, 2, 2)
    assert D.max_over_ranks(3.5) == 3.5
