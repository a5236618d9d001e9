"""Data-parallel helpers: one process per GPU decodes its own signals.

Decodes of different signals are independent problems (Sec. 2: every signal
is encoded with the same dictionary and decoded on its own), so ranks share
no data during a run; the only communication is the timing and counting
done here after each timed region (max of the elapsed times, sum of the
work), never on the data path.
"""
from __future__ import annotations


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's signals: distinct per rank, same for a given rank."""
    return int(base) + 7919 * int(rank)


def shard(n: int, rank: int, world: int) -> range:
    """Contiguous share of n items for `rank` (sizes differ by at most 1)."""
    q, r = divmod(int(n), int(world))
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


def aggregate(elapsed_s: float, units: float, device=None):
    """Max of the ranks' elapsed times and sum of their units of work.

    Returns (max_elapsed_s, total_units); without an initialised process
    group it returns the local values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_s), float(units)
    t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
