"""The multi-rank host logic on CPU: gloo, world size 2.

Ranks split a batch with no data-path collective (sharding by work), and the
benchmark reduces its per-rank timings with a max over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1909_13560_gb300 import sharding
from paper_1909_13560_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = W.config4(count=257)
    shares = sharding.shard_by_work(probs, world)
    mine = shares[rank]
    work = sum(sharding.problem_work(probs[i]) for i in mine)
    # each rank reports its share; rank 0 checks the union on the host
    got = [None] * world
    dist.all_gather_object(got, (rank, mine, work))
    import bench
    t = bench._max_over_ranks(dist, float(rank + 1) * 0.5)
    if rank == 0:
        out.put((got, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_a_batch_and_reduce_timings():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 1.0  # the max of 0.5 and 1.0
    idx = sorted(i for _, mine, _ in got for i in mine)
    assert idx == list(range(257))
    works = [w for _, _, w in got]
    probs = W.config4(count=257)
    biggest = max(sharding.problem_work(p) for p in probs)
    assert abs(works[0] - works[1]) <= biggest


def test_shard_by_work_single_and_many():
    probs = W.config4(count=50)
    assert sharding.shard_by_work(probs, 1) == [list(range(50))]
    shares = sharding.shard_by_work(probs, 8)
    assert sorted(i for s in shares for i in s) == list(range(50))
    with pytest.raises(ValueError):
        sharding.shard_by_work(probs, 0)
