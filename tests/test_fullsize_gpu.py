"""The batched and served workloads at their full sizes, in the launch
configuration the benchmark times (autotuned GEMM shape), checked on sampled
signals against the FP64 oracle and, where the oracle cannot finish in
seconds, on properties that hold at any size.

* BF16, N=2048, M=8192, 1024 signals: every signal converges and recovers
  its support; 6 sampled signals meet the oracle comparison rule.
* FP8, N=8192, M=32768, 256 signals: every signal converges and recovers its
  support; for 2 sampled signals the oracle replays the first 24 selected
  atoms (each must be an MP choice within the FP32 bound), and x~ equals the
  plain FP32 kernel's whenever the atom sequences agree.
* The served workload's four dictionaries: a request per dictionary through
  the server equals the same signal decoded by mp_recover_batched alone.
"""
import numpy as np
import pytest

from gpu_helpers import GpuPlan, compare_to_oracle, cur_stream, summation_depth, U32
from oracle import mp_oracle as orc
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def B():
    from paper_0809_1833_gb300 import binding
    return binding


def batched(pl, prec, prob, cap):
    import torch
    b = B()
    Y = torch.from_numpy(prob.y).cuda()
    X = torch.full((prob.B, prob.M), float("nan"), dtype=torch.float32, device="cuda")
    atoms = torch.full((prob.B, cap), -1, dtype=torch.int32, device="cuda")
    tr = b.make_trace(atoms.data_ptr(), 0, 0, cap)
    s, res = b.mp_recover_batched(pl.plan, prec, Y.data_ptr(), X.data_ptr(), prob.B, (prob.eps, prob.T), tr,
                                  cur_stream())
    torch.cuda.synchronize()
    return s, res, X.cpu().numpy(), atoms.cpu().numpy()


def test_batched_bf16_full_workload():
    prob = W.make_workload("batched_bf16_N2048_M8192_B1024", seed=0)
    p = B().MP_PREC_BF16
    with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
        s, res, X, atoms = batched(pl, p, prob, 4096)
        assert s == 0
        assert all(r.status == 0 and r.stop_reason == B().MP_STOP_CONVERGED for r in res)
        assert min(orc.support_score(X[b], prob.supports[b]) for b in range(prob.B)) == 1.0
        for b in (0, 170, 341, 512, 683, 1023):
            plain = pl.decode(prob.y[b], prob.eps, prob.T)
            r = res[b]
            same = r.iters == plain["result"].iters and np.array_equal(atoms[b, :r.iters], plain["atoms"])
            if same:
                assert np.array_equal(X[b], plain["x"]), b
            out = dict(result=r, x=X[b], atoms=atoms[b, :r.iters], r=plain["r"])
            compare_to_oracle(prob.psi, prob.y[b], prob.eps, prob.T, out, check_follow=not same)


def test_batched_fp8_full_workload():
    prob = W.make_workload("batched_fp8_N8192_M32768_B256", seed=0)
    p = B().MP_PREC_FP8E4M3
    with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
        s, res, X, atoms = batched(pl, p, prob, 10000)
        assert s == 0
        assert all(r.status == 0 and r.stop_reason == B().MP_STOP_CONVERGED for r in res)
        assert min(orc.support_score(X[b], prob.supports[b]) for b in range(prob.B)) == 1.0
        for b in (0, 255):
            plain = pl.decode(prob.y[b], prob.eps, prob.T)
            r = res[b]
            if r.iters == plain["result"].iters and np.array_equal(atoms[b, :r.iters], plain["atoms"]):
                assert np.array_equal(X[b], plain["x"]), b
            # the first 24 selections are MP choices of the FP64 oracle, within
            # the FP32 rounding bound of one correlation (no drift yet)
            f = orc.follow(prob.psi, prob.y[b], atoms[b, :24])
            tol = np.maximum(1e-5, 2 * summation_depth(prob.N) * U32 * f["rnorm"] / f["cmax"])
            assert np.all(f["ratio"] >= 1 - tol), f["ratio"].min()


def test_served_full_dictionaries_equal_lone_batched_decodes():
    b = B()
    w = W.WORKLOADS["served_4dict_poisson2000"]
    p = b.MP_PREC_BF16
    srv = b.mp_server_create(64 << 30, 64, 256)
    plans, probs, tickets = [], [], []
    try:
        dids = []
        for k, (N, M) in enumerate(w["dicts"]):       # every dictionary before the first submit
            psi = W.gaussian_dictionary(N, M, seed=k)
            pl = GpuPlan(psi, prec_mask=1 << p)
            plans.append(pl)
            dids.append(b.mp_server_add_dictionary(srv, pl.plan, p))
            probs.append(W.make_plain(N, M, max(4, N // 16), seed=50 + k, eps=w["eps"], T=w["T"], psi=psi))
        for did, prob in zip(dids, probs):
            st, tk = b.mp_server_submit(srv, did, np.ascontiguousarray(prob.y[0]), w["eps"], w["T"])
            assert st == b.MP_OK
            tickets.append((did, tk))
        for k, (did, tk) in enumerate(tickets):
            prob = probs[k]
            x = np.empty(prob.M, np.float32)
            while True:
                st, res = b.mp_server_poll(srv, tk, x)
                if st == b.MP_OK:
                    break
                assert st == b.MP_PENDING
            s, lone, Xl, _ = batched(plans[k], p, prob, 16)
            assert s == 0 and res.iters == lone[0].iters and np.array_equal(x, Xl[0]), k
            assert orc.support_score(x, prob.supports[0]) == 1.0
    finally:
        b.mp_server_destroy(srv)
        for pl in plans:
            pl.close()
