"""One decode with the dictionary's atoms split across ranks, one GPU each.

Per MP iteration (Sec. 3, Eqs. 9-12) every rank computes its shard's best
candidate as a fixed-size record (packed key, global atom, coefficient, the
atom's row), the ranks exchange their records with one all-gather (NCCL on
GPUs), and every rank applies the same step: the largest |c| wins, ties to
the smallest global atom (Sec. 4); each rank updates its copy of r, the
energy and the stop test, and the owner adds c to its slice of x~.  The
arithmetic, the selection and the stop test run in the library's kernels
(``mp_shard_*``); this module only moves records between ranks and reads
the stop flag every ``check_every`` iterations (the kernels make the steps
after a stop no-ops, so the check interval never changes the result).
"""
from __future__ import annotations

import ctypes

from . import binding as B


def shard_range(M: int, world: int, rank: int) -> tuple[int, int]:
    """(first global atom, atom count) of ``rank``'s contiguous shard."""
    base, rem = divmod(int(M), int(world))
    return rank * base + min(rank, rem), base + (1 if rank < rem else 0)


class ShardOps:
    """The library's per-rank state for one sharded decode: residual copy,
    x~ slice, stop state and the record buffers, on the plan's device."""

    def __init__(self, plan, atom_offset: int, y, stream=None):
        import torch
        self.plan, self.offset = plan, int(atom_offset)
        self.dev = y.device
        self.stream = stream
        self.ld = B.mp_plan_query(plan, B.MP_Q_LD_FP32)
        self.rb = B.mp_shard_record_bytes(plan)
        m_local = int(B.mp_plan_query(plan, B.MP_Q_PLAN_M))
        self.y = y
        self.r = torch.empty(self.ld, dtype=torch.float32, device=self.dev)
        self.x = torch.empty(m_local, dtype=torch.float32, device=self.dev)
        self.state = torch.zeros(ctypes.sizeof(B.mp_shard_state), dtype=torch.uint8, device=self.dev)
        self.rec = torch.empty(self.rb, dtype=torch.uint8, device=self.dev)
        self.recs = None

    def record_bytes(self) -> int:
        return self.rb

    def init(self, eps: float, max_iters: int) -> None:
        B.mp_shard_init(self.plan, self.y.data_ptr(), self.r.data_ptr(), self.x.data_ptr(), eps, max_iters,
                        self.state.data_ptr(), self._s())

    def gather_buffer(self, world: int):
        import torch
        self.recs = torch.empty(world * self.rb, dtype=torch.uint8, device=self.dev)
        return self.recs

    def local(self):
        B.mp_shard_step_local(self.plan, self.offset, self.r.data_ptr(), self.rec.data_ptr(), self._s())
        return self.rec

    def apply(self, recs, n: int) -> None:
        B.mp_shard_step_apply(self.plan, self.offset, recs.data_ptr(), n, self.r.data_ptr(), self.x.data_ptr(),
                              self.state.data_ptr(), None, self._s())

    def host_state(self) -> B.mp_shard_state:
        raw = bytes(self.state.cpu().numpy().tobytes())
        return B.mp_shard_state.from_buffer_copy(raw)

    def stopped(self) -> bool:
        return bool(self.host_state().stopped)

    def result(self) -> dict:
        s = self.host_state()
        rel = (s.e / s.e0) ** 0.5 if s.e0 > 0 else 0.0
        return {"iters": s.t, "stop_reason": s.stop_reason, "status": s.status, "rel_residual": rel,
                "energy_audit_max": s.audit, "x_local": self.x}

    def _s(self):
        return self.stream


def sharded_recover(ops, eps: float, max_iters: int, group=None, check_every: int = 8) -> dict:
    """Run one sharded decode.  ``ops`` is this rank's ``ShardOps``; with
    torch.distributed initialised the records of all ranks of ``group`` are
    all-gathered every iteration, otherwise the decode runs on one shard."""
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    ops.init(eps, max_iters)
    if ops.stopped():
        return ops.result()
    recs = ops.gather_buffer(world)
    nccl = world > 1 and dist.get_backend(group) == "nccl"
    for it in range(int(max_iters)):
        rec = ops.local()
        if world == 1:
            ops.apply(rec, 1)
        else:
            if nccl:
                dist.all_gather_into_tensor(recs, rec, group=group)
            else:
                parts = list(recs.view(world, -1).unbind(0))
                dist.all_gather(parts, rec, group=group)
            ops.apply(recs, world)
        if (it + 1) % check_every == 0 and ops.stopped():
            break
    return ops.result()
