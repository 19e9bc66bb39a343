"""Multi-process (replica) path of bench.py on CPU: world size 2 over gloo.
Each rank owns a disjoint share of independent realisations; the reported step
time is the maximum over ranks (no data-path collective)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.shard(64, rank, world)
    t = bench.max_over_ranks(10.0 + 5.0 * rank)  # this rank's step time
    dist.barrier()
    q.put((rank, mine, t))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_sharding_and_max_time(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    units = sorted(u for _, mine, _ in res for u in mine)
    assert units == list(range(64))  # every realisation exactly once
    assert all(len(mine) == 64 // world for _, mine, _ in res)
    assert all(t == 10.0 + 5.0 * (world - 1) for _, _, t in res)  # the slowest rank


def test_shard_uneven_and_single_rank():
    parts = [bench.shard(7, r, 3) for r in range(3)]
    assert parts == [[0, 1, 2], [3, 4], [5, 6]]
    assert bench.shard(5, 0, 1) == list(range(5))
    assert bench.max_over_ranks(3.5) == 3.5  # no process group
