"""Continuous-batching server (include/mpgb_server.h).

Requests for two resident dictionaries are submitted while others run; each
result must equal the lone decode of the same request (mp_recover_batched
with B = 1) bit for bit, since a signal's arithmetic does not depend on its
batch row or its neighbours.  Faults are injected on the host.
"""
import threading
import time

import numpy as np
import pytest

from gpu_helpers import GpuPlan, compare_to_oracle, cur_stream
from oracle import mp_oracle as orc
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def B():
    from paper_0809_1833_gb300 import binding
    return binding


def lone(pl, prec, y, eps, T):
    import torch
    Yd = torch.from_numpy(np.ascontiguousarray(y[None, :], dtype=np.float32)).cuda()
    X = torch.empty((1, pl.M), dtype=torch.float32, device="cuda")
    s, res = B().mp_recover_batched(pl.plan, prec, Yd.data_ptr(), X.data_ptr(), 1, (eps, T), None, cur_stream(),
                                    raise_on_error=False)
    torch.cuda.synchronize()
    return s, res[0], X.cpu().numpy()[0]


def wait_all(srv, tickets, M_of, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            x = np.empty(M_of[t], dtype=np.float32)
            s, res = B().mp_server_poll(srv, t, x)
            if s == B().MP_OK:
                out[t] = (res, x)
            else:
                assert s == B().MP_PENDING, s
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.001)
    return out


def test_mixed_requests_equal_lone_decodes():
    prec = B().MP_PREC_BF16
    dicts = [(256, 1024), (512, 2048)]
    psis = [W.gaussian_dictionary(N, M, seed=20 + i) for i, (N, M) in enumerate(dicts)]
    plans = [GpuPlan(p, prec_mask=1 << prec) for p in psis]
    srv = B().mp_server_create(4 << 30, 64, 10000)
    try:
        ids = [B().mp_server_add_dictionary(srv, pl.plan, prec) for pl in plans]
        assert all(B().mp_server_dictionary_slots(srv, i) == 64 for i in ids)
        rng = np.random.default_rng(5)
        reqs = []
        for k in range(160):
            d = int(rng.integers(0, 2))
            N, M = dicts[d]
            K = int(rng.integers(4, N // 16 + 1))
            prob = W.make_plain(N, M, K, seed=1000 + k, eps=1e-5, T=4000, psi=psis[d])
            reqs.append((d, prob))
        tickets, M_of = [], {}
        for i, (d, prob) in enumerate(reqs):
            s, t = B().mp_server_submit(srv, ids[d], np.ascontiguousarray(prob.y[0]), prob.eps, prob.T)
            assert s == 0
            tickets.append(t)
            M_of[t] = prob.M
            if i % 20 == 19:
                time.sleep(0.002)   # later requests arrive while earlier ones run
        out = wait_all(srv, tickets, M_of)
        st = B().mp_server_get_stats(srv)
        assert st.completed == len(reqs) and st.rejected == 0 and st.active == 0 and st.queued == 0
        assert 0 < st.latency_p50_s <= st.latency_p99_s
        for i, ((d, prob), t) in enumerate(zip(reqs, tickets)):
            res, x = out[t]
            s, r1, x1 = lone(plans[d], prec, prob.y[0], prob.eps, prob.T)
            assert res.status == 0 and res.iters == r1.iters and res.stop_reason == r1.stop_reason
            assert np.array_equal(x, x1), i
            if i % 16 == 0:
                ora = orc.mp(prob.psi, prob.y[0], prob.eps, prob.T)
                assert np.linalg.norm(x - ora["x"]) <= 1e-4 * np.linalg.norm(ora["x"])
                assert orc.support_score(x, prob.supports[0]) == 1.0
    finally:
        B().mp_server_destroy(srv)
        for pl in plans:
            pl.close()


def test_server_faults_injected_on_host():
    prec = B().MP_PREC_BF16
    psi = W.gaussian_dictionary(128, 512, seed=3)
    with GpuPlan(psi, prec_mask=1 << prec) as pl:
        # budget too small for even one slot
        small = B().mp_server_create(1024, 8, 4)
        with pytest.raises(B().MpError) as ei:
            B().mp_server_add_dictionary(small, pl.plan, prec)
        assert ei.value.status == B().MP_ERR_BUSY
        B().mp_server_destroy(small)
        srv = B().mp_server_create(1 << 30, 4, 3)
        try:
            d = B().mp_server_add_dictionary(srv, pl.plan, prec)
            prob = W.make_plain(128, 512, 6, seed=9, psi=psi)
            bad = prob.y[0].copy()
            bad[3] = np.nan
            s1, t_nan = B().mp_server_submit(srv, d, bad, 1e-5, 1000)
            s2, t_zero = B().mp_server_submit(srv, d, np.zeros(128, np.float32), 1e-5, 1000)
            s3, t_ok = B().mp_server_submit(srv, d, np.ascontiguousarray(prob.y[0]), 1e-5, 1000)
            assert s1 == s2 == s3 == 0
            # flood the queue: beyond max_queue waiting requests are refused
            statuses = [B().mp_server_submit(srv, d, np.ascontiguousarray(prob.y[0]), 1e-5, 1000) for _ in range(40)]
            assert any(s == B().MP_ERR_BUSY for s, _ in statuses)
            accepted = [t for s, t in statuses if s == 0]
            out = wait_all(srv, [t_nan, t_zero, t_ok] + accepted, {t: 512 for t in [t_nan, t_zero, t_ok] + accepted})
            assert out[t_nan][0].status == B().MP_ERR_NONFINITE and out[t_nan][0].iters == 0
            assert out[t_zero][0].stop_reason == B().MP_STOP_ZERO_Y and not np.any(out[t_zero][1])
            assert out[t_ok][0].status == 0
            for t in accepted:
                assert np.array_equal(out[t][1], out[t_ok][1])
            s, _ = B().mp_server_poll(srv, t_ok)
            assert s == B().MP_ERR_NOT_FOUND        # released by the successful poll
            st = B().mp_server_get_stats(srv)
            assert st.rejected == sum(1 for s, _ in statuses if s == B().MP_ERR_BUSY)
        finally:
            B().mp_server_destroy(srv)


def test_concurrent_submitters():
    prec = B().MP_PREC_BF16
    psi = W.gaussian_dictionary(256, 1024, seed=8)
    with GpuPlan(psi, prec_mask=1 << prec) as pl:
        srv = B().mp_server_create(1 << 30, 32, 1000)
        try:
            d = B().mp_server_add_dictionary(srv, pl.plan, prec)
            probs = [W.make_plain(256, 1024, 10, seed=300 + k, psi=psi) for k in range(48)]
            tickets = [None] * len(probs)

            def worker(lo, hi):
                for k in range(lo, hi):
                    s, t = B().mp_server_submit(srv, d, np.ascontiguousarray(probs[k].y[0]), 1e-5, 2000)
                    assert s == 0
                    tickets[k] = t

            th = [threading.Thread(target=worker, args=(i * 12, (i + 1) * 12)) for i in range(4)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            out = wait_all(srv, tickets, {t: 1024 for t in tickets})
            for k, t in enumerate(tickets):
                _, r1, x1 = lone(pl, prec, probs[k].y[0], 1e-5, 2000)
                assert np.array_equal(out[t][1], x1)
        finally:
            B().mp_server_destroy(srv)
