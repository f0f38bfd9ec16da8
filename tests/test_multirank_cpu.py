"""Host logic of the multi-rank benchmark on CPU: world_size-2 gloo ranks
(127.0.0.1).  Independent instances are shared out with no overlap and
nothing missing; the job's time is the slowest rank's; work adds up."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        for n in (256, 7, 1):
            lo, hi = bench.shard(n, rank, world)
            got = [None] * world
            dist.all_gather_object(got, (lo, hi))
            out[n] = got
        out["max"] = bench.max_over_ranks(10.0 + rank, dist)
        out["sum"] = bench.sum_over_ranks(3.0 * (rank + 1), dist)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_shard_partitions_without_overlap():
    for n in (0, 1, 5, 256, 257):
        for world in (1, 2, 3, 8):
            covered = []
            for r in range(world):
                lo, hi = bench.shard(n, r, world)
                assert 0 <= lo <= hi <= n
                covered.extend(range(lo, hi))
            assert covered == list(range(n))
            sizes = [bench.shard(n, r, world)[1] - bench.shard(n, r, world)[0] for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        out = res[r]
        assert out[256] == [(0, 128), (128, 256)]
        assert out[7] == [(0, 4), (4, 7)]
        assert out[1] == [(0, 1), (1, 1)]
        assert out["max"] == 11.0
        assert out["sum"] == 9.0
