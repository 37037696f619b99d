"""Replica sharding and cross-rank bookkeeping, on CPU with gloo, world size 2."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2206_01784_gb300 import replicas


def test_shard_round_robin_covers_once():
    units = list(range(11))
    parts = [replicas.shard_round_robin(units, r, 3) for r in range(3)]
    assert sorted(u for p in parts for u in p) == units


def test_shard_balanced():
    sizes = [5, 1, 9, 3, 3, 7, 2]
    parts = replicas.shard_balanced(sizes, 2)
    assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert abs(loads[0] - loads[1]) <= max(sizes)
    assert replicas.shard_balanced(sizes, 2) == parts  # deterministic


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.shard_round_robin(list(range(10)), rank, world)
        total = replicas.sum_over_ranks(sum(mine))
        slowest = replicas.max_over_ranks(1.5 + rank)
        lat = replicas.gather_lists([float(rank)] * (rank + 1))
        dist.barrier()
        q.put((rank, total, slowest, sorted(lat)))
    finally:
        dist.destroy_process_group()


def test_gloo_world_size_2():
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, slowest, lat in res:
        assert total == 45.0          # every unit counted once
        assert slowest == 2.5         # max over ranks
        assert lat == [0.0, 1.0, 1.0]
