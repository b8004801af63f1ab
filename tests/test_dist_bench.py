"""The multi-rank host logic of bench.py on the CPU: two gloo ranks, the
job's time as the maximum over ranks, points summed over ranks, and the
round-robin frame shards (frames are independent: no data-path exchange)."""

import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [7.5, 9.25][rank]  # rank 1 is the slower one
        t = bench.max_over_ranks(local_ms, world)
        pts = bench.sum_over_ranks([1000, 2500][rank], world)
        shard = bench.shard_frames(5, rank, world)
        q.put((rank, t, pts, shard))
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
    assert [o[1] for o in out] == [9.25, 9.25]
    assert [o[2] for o in out] == [3500.0, 3500.0]
    assert out[0][3] == [0, 2, 4] and out[1][3] == [1, 3]


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.sum_over_ranks(3.0, 1) == 3.0
    assert bench.shard_frames(4, 0, 1) == [0, 1, 2, 3]


@pytest.mark.parametrize("n,world", [(64, 2), (64, 8), (7, 3)])
def test_shards_partition_the_batch(n, world):
    shards = [bench.shard_frames(n, r, world) for r in range(world)]
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(n))
    assert max(len(s) for s in shards) - min(len(s) for s in shards) <= 1
