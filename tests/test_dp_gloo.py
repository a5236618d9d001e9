"""Multi-process data-parallel host logic on CPU ranks (gloo, world size 2):
shards cover every signal once, per-rank seeds differ, and the benchmark's
aggregation takes the max time and the summed work over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_0809_1833_gb300 import dp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [0.5, 1.25][rank]
        units = [3, 4][rank]
        t, u = dp.aggregate(elapsed, units)
        q.put((rank, t, u, list(dp.shard(10, rank, world)), dp.rank_seed(0, rank)))
    finally:
        dist.destroy_process_group()


def test_shard_covers_each_item_once():
    for n in (0, 1, 7, 10, 1024):
        for world in (1, 2, 3, 8):
            got = [i for r in range(world) for i in dp.shard(n, r, world)]
            assert got == list(range(n))
            sizes = [len(dp.shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def test_aggregate_single_process():
    assert dp.aggregate(2.0, 5) == (2.0, 5.0)


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
    for rank, t, u, sh, seed in out:
        assert t == 1.25 and u == 7.0
    assert out[0][3] + out[1][3] == list(range(10))
    assert out[0][4] != out[1][4]
