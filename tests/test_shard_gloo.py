"""The sharded decode's exchange on CPU ranks (gloo, world size 2 and 3).

The driver (paper_0809_1833_gb300/sharded.py) only moves fixed-size records
between ranks and polls the stop flag; the per-rank arithmetic sits behind
an ``ops`` object, which on a GPU is the library (tests/test_shard_gpu.py).
Here a small CPU stand-in written in this test plays that role -- an FP64
restatement of the same record contract: the shard's best (|c|, global
index) key, the coefficient and the atom row; the winner is the largest
|c|, ties to the smaller global index -- so that the driver's all-gather,
record layout and stop polling are exercised across real process groups.
Each rank's x~ slice must equal the one-rank run on the whole dictionary.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_0809_1833_gb300.sharded import shard_range, sharded_recover


class CpuShardOps:
    """Record: float64 [|c|, -global index, c, global index, psi row (N)]."""

    def __init__(self, psi_shard, offset, y):
        self.P = np.asarray(psi_shard, dtype=np.float64)
        self.off = offset
        self.y = np.asarray(y, dtype=np.float64)
        self.N = self.y.size

    def init(self, eps, T):
        self.r = self.y.copy()
        self.x = np.zeros(self.P.shape[0])
        self.e0 = float(self.r @ self.r)
        self.e = self.e0
        self.thr2 = eps * eps * self.e0
        self.t, self.T = 0, T
        self.stop = not (self.e > self.thr2 and T > 0)

    def gather_buffer(self, world):
        return torch.zeros(world * (4 + self.N), dtype=torch.float64)

    def local(self):
        c = (self.P * self.r).sum(axis=1)      # per-row sums: the same bits in any shard
        i = int(np.argmax(np.abs(c)))          # first maximiser: the smallest index
        rec = np.concatenate([[abs(c[i]), -(self.off + i), c[i], self.off + i], self.P[i]])
        return torch.from_numpy(rec)

    def apply(self, recs, n):
        if self.stop:
            return
        R = recs.numpy().reshape(n, 4 + self.N)
        w = max(range(n), key=lambda k: (R[k, 0], R[k, 1]))
        c, m = R[w, 2], int(R[w, 3])
        self.r = self.r - c * R[w, 4:]
        if self.off <= m < self.off + self.P.shape[0]:
            self.x[m - self.off] += c
        self.e = float(self.r @ self.r)
        self.t += 1
        self.stop = not (self.e > self.thr2 and self.t < self.T)

    def stopped(self):
        return self.stop

    def result(self):
        return {"iters": self.t, "x_local": self.x}


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    g = np.random.default_rng(3)
    M, N = 40, 12
    P = g.standard_normal((M, N))
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    P[27] = P[5]                      # an exact tie between shards: atom 5 must win
    x = np.zeros(M)
    x[[5, 13, 31]] = [2.0, -1.5, 1.1]
    return P, x @ P


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P, y = _problem()
        off, cnt = shard_range(P.shape[0], world, rank)
        res = sharded_recover(CpuShardOps(P[off:off + cnt], off, y), 1e-9, 500, check_every=3)
        q.put((rank, off, res["iters"], res["x_local"].tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_match_one_rank(world):
    P, y = _problem()
    one = sharded_recover(CpuShardOps(P, 0, y), 1e-9, 500, check_every=3)
    assert one["x_local"][27] == 0.0 and one["x_local"][5] != 0.0
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x = np.concatenate([np.array(xl) for _, _, _, xl in out])
    assert all(it == one["iters"] for _, _, it, _ in out)
    assert np.array_equal(x, one["x_local"])


def test_shard_range_covers_every_atom_once():
    for M in (1, 7, 40, 16384):
        for world in (1, 2, 3, 8):
            got = []
            for r in range(world):
                off, cnt = shard_range(M, world, r)
                got += list(range(off, off + cnt))
            assert got == list(range(M))
