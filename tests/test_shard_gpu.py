"""The atom-sharded decode (mp_shard_*, paper_0809_1833_gb300/sharded.py) on
one GPU.  With one shard it must reproduce mp_recover bit for bit (the same
correlation, selection, update and energy orders).  With several shards of
one dictionary -- each its own plan, the records of all shards gathered by
hand every iteration, as the all-gather does across GPUs -- every shard's
residual stays identical, the winner is the global argmax with ties to the
smallest global index, and the concatenated x~ slices equal mp_recover's x~.
"""
import ctypes

import numpy as np
import pytest

import oracle_pins as P
from gpu_helpers import GpuPlan, cur_stream
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def B():
    from paper_0809_1833_gb300 import binding
    return binding


def run_shards(psi, y, eps, T, n_shards, cap=20000):
    """Decode with the dictionary split into n_shards plans on this GPU."""
    import torch
    from paper_0809_1833_gb300.sharded import shard_range
    b = B()
    M, N = psi.shape
    plans, states = [], []
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).cuda()
    for k in range(n_shards):
        off, cnt = shard_range(M, n_shards, k)
        pl = GpuPlan(psi[off:off + cnt])
        ld = pl.query(b.MP_Q_LD_FP32)
        st = dict(plan=pl, off=off, cnt=cnt,
                  r=torch.empty(ld, dtype=torch.float32, device="cuda"),
                  x=torch.full((cnt,), float("nan"), dtype=torch.float32, device="cuda"),
                  state=torch.zeros(ctypes.sizeof(b.mp_shard_state), dtype=torch.uint8, device="cuda"))
        b.mp_shard_init(pl.plan, yd.data_ptr(), st["r"].data_ptr(), st["x"].data_ptr(), eps, T,
                        st["state"].data_ptr(), cur_stream())
        states.append(st)
    rb = b.mp_shard_record_bytes(states[0]["plan"].plan)
    recs = torch.zeros(n_shards * rb, dtype=torch.uint8, device="cuda")
    atoms = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    tr = b.make_trace(atoms.data_ptr(), 0, 0, cap)

    def host_state(st):
        return b.mp_shard_state.from_buffer_copy(bytes(st["state"].cpu().numpy().tobytes()))

    for it in range(T):
        if host_state(states[0]).stopped:
            break
        for k, st in enumerate(states):
            b.mp_shard_step_local(st["plan"].plan, st["off"], st["r"].data_ptr(), recs.data_ptr() + k * rb,
                                  cur_stream())
        for k, st in enumerate(states):
            b.mp_shard_step_apply(st["plan"].plan, st["off"], recs.data_ptr(), n_shards, st["r"].data_ptr(),
                                  st["x"].data_ptr(), st["state"].data_ptr(), tr if k == 0 else None,
                                  cur_stream())
    torch.cuda.synchronize()
    ss = [host_state(st) for st in states]
    rs = [st["r"].cpu().numpy() for st in states]
    x = np.concatenate([st["x"].cpu().numpy() for st in states])
    for st in states:
        st["plan"].close()
    return dict(states=ss, r=rs, x=x, atoms=atoms.cpu().numpy()[:ss[0].t])


@pytest.mark.parametrize("n_shards", [1, 2, 3])
def test_shards_reproduce_the_single_device_decode(n_shards):
    prob = W.make_plain(256, 1500, 16, seed=4, eps=1e-6, T=3000)
    with GpuPlan(prob.psi) as pl:
        ref = pl.decode(prob.y[0], prob.eps, prob.T)
    out = run_shards(prob.psi, prob.y[0], prob.eps, prob.T, n_shards)
    s0 = out["states"][0]
    assert s0.t == ref["result"].iters and s0.stop_reason == ref["result"].stop_reason
    assert np.array_equal(out["atoms"], ref["atoms"])
    assert np.array_equal(out["x"], ref["x"])
    assert s0.e == ref["energies"][-1]
    for k in range(1, n_shards):
        assert np.array_equal(out["r"][k], out["r"][0])
        assert out["states"][k].e == s0.e and out["states"][k].t == s0.t
    assert np.array_equal(out["r"][0][:prob.N], ref["r"])


def test_tie_across_shards_goes_to_the_smallest_global_index():
    """The worked example split after atom 2: the step-1 tie is between atom
    0 (shard 0) and atom 4 (shard 1); the smaller index wins, and the run
    ends at t = 10 with the closed-form x~."""
    g = P.load_worked_example()
    ex = g["expected"]
    out = run_shards(np.array(g["psi_atoms"], dtype=np.float32), np.array(g["y"], dtype=np.float32),
                     g["eps"], g["T"], 2)
    assert out["states"][0].t == ex["iters"]
    assert list(out["atoms"]) == ex["atoms"]
    assert np.array_equal(out["x"].astype(np.float64), np.array(ex["x"]))


def test_sharded_driver_one_rank_and_edge_cases():
    import torch
    from paper_0809_1833_gb300.sharded import ShardOps, sharded_recover
    prob = W.make_plain(128, 700, 8, seed=6, eps=1e-6, T=2000)
    with GpuPlan(prob.psi) as pl:
        ref = pl.decode(prob.y[0], prob.eps, prob.T)
        y = torch.from_numpy(prob.y[0]).cuda()
        for every in (1, 8):
            res = sharded_recover(ShardOps(pl.plan, 0, y), prob.eps, prob.T, check_every=every)
            assert res["iters"] == ref["result"].iters
            assert np.array_equal(res["x_local"].cpu().numpy(), ref["x"])
        z = sharded_recover(ShardOps(pl.plan, 0, torch.zeros(128, device="cuda")), 1e-5, 100)
        assert z["iters"] == 0 and z["stop_reason"] == B().MP_STOP_ZERO_Y
        bad = y.clone()
        bad[3] = float("nan")
        nf = sharded_recover(ShardOps(pl.plan, 0, bad), 1e-5, 100)
        assert nf["iters"] == 0 and nf["status"] == B().MP_ERR_NONFINITE
        t0 = sharded_recover(ShardOps(pl.plan, 0, y), 1e-5, 0)
        assert t0["iters"] == 0 and t0["stop_reason"] == B().MP_STOP_MAX_ITERS
