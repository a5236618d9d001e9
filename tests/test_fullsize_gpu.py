"""The batched and served workloads at their full sizes, in the launch
configuration the benchmark times (autotuned GEMM shape), checked against
the full FP64 oracle on sampled signals, each compared with the batched
path's own final residual (its drift) and atom sequence.

* BF16, N=2048, M=8192, 1024 signals: every signal converges and recovers
  its support; 16 sampled signals meet the oracle rule (the literal atom
  sequence up to the first oracle gap <= 1e-5, x~ within 1e-4 relative).
* FP8, N=8192, M=32768, 256 signals: every signal converges and recovers its
  support; 4 sampled signals meet the same rule against full FP64 oracle
  decodes (each about half a minute on the host cores).
* The served workload's four dictionaries: a request per dictionary through
  the server equals the same signal decoded by mp_recover_batched alone.
"""
import numpy as np
import pytest

from gpu_helpers import GpuPlan, batched_decode, batched_signal, compare_to_oracle
from oracle import mp_oracle as orc
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def B():
    from paper_0809_1833_gb300 import binding
    return binding


def batched(pl, prec, prob, cap):
    out = batched_decode(pl, prec, prob.y, (prob.eps, prob.T), cap)
    return out["status"], out["results"], out["X"], out["atoms"]


def _full_workload(name, prec, cap, sample):
    prob = W.make_workload(name, seed=0)
    with GpuPlan(prob.psi, prec_mask=1 << prec) as pl:
        out = batched_decode(pl, prec, prob.y, (prob.eps, prob.T), cap)
    assert out["status"] == 0
    res, X = out["results"], out["X"]
    assert all(r.status == 0 and r.stop_reason == B().MP_STOP_CONVERGED for r in res)
    assert min(orc.support_score(X[b], prob.supports[b]) for b in range(prob.B)) == 1.0
    diag = []
    for b in sample:
        ora = orc.mp(prob.psi, prob.y[b], prob.eps, prob.T)
        d = compare_to_oracle(prob.psi, prob.y[b], prob.eps, prob.T, batched_signal(out, b), ora=ora,
                              check_follow=False, label=f"{name}[{b}]")
        assert d["x_rel_err"] <= 1e-4
        diag.append(d)
    return diag


def test_batched_bf16_full_workload():
    sample = [int(b) for b in np.linspace(0, 1023, 16)]
    _full_workload("batched_bf16_N2048_M8192_B1024", B().MP_PREC_BF16, 4096, sample)


def test_batched_fp8_full_workload():
    _full_workload("batched_fp8_N8192_M32768_B256", B().MP_PREC_FP8E4M3, 10000, [0, 85, 170, 255])


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
