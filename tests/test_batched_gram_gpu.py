"""Batched and served decodes with Gram-updated correlations
(MP_OPT_BATCH_GRAM, refresh period R).

Not in the paper: from Eqs. 9 and 11, after r <- r - c psi_m every
correlation moves by -c <psi_m, psi_j> = -c G[m][j].  Each signal keeps its
FP32 correlations, computed directly from the FP32 atoms at admission and
every R of its own steps; a step takes the 8 largest |c|, rescores them in
FP32 from the FP32 atoms exactly as the direct batched step does, commits
the best and updates the row from one row of G.  The selection is the FP32
rescore's, so whenever the FP32 argmax is among the 8 candidates the decode
equals the plain FP32 kernel's bit for bit; the tests check that (for every
signal here), the literal oracle rule on sampled signals, the server's
alone-equals-in-the-mix property in this mode, and the option's argument
checks.

The switched mode (MP_OPT_BATCH_GRAM_BELOW = S) runs direct steps while more
than S signals are active and Gram steps after, with every active signal's
correlations computed directly at the switch; since both kinds of step
select by the same FP32 rescore, its decodes must equal the direct decode's
bit for bit here too, on a small batch at several thresholds and on the full
1024-signal BF16 workload at the threshold the benchmark uses.
"""
import time

import numpy as np
import pytest

from gpu_helpers import GpuPlan, batched_decode, batched_signal, compare_to_oracle, cur_stream
from oracle import mp_oracle as orc
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def B():
    from paper_0809_1833_gb300 import binding
    return binding


@pytest.mark.parametrize("R", [16, 64, 4096])
def test_gram_batched_matches_plain_and_oracle(R):
    prob = W.make_batched(256, 1024, 300, 2, 16, seed=5, eps=1e-5, T=3000)
    p = B().MP_PREC_BF16
    with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
        pl.set(B().MP_OPT_BATCH_GRAM, R)
        out = batched_decode(pl, p, prob.y, (prob.eps, prob.T), 3000)
        assert out["status"] == 0
        assert pl.query(B().MP_Q_BATCH_GRAM) == R
        assert pl.query(B().MP_Q_GRAM_BYTES) == 1024 * 1024 * 4
        n_same = 0
        for b in range(prob.B):
            r = out["results"][b]
            assert r.status == 0 and r.stop_reason == B().MP_STOP_CONVERGED
            plain = pl.decode(prob.y[b], prob.eps, prob.T)
            if r.iters == plain["result"].iters and np.array_equal(out["atoms"][b, :r.iters], plain["atoms"]):
                # the same atoms: the same FP32 coefficients, update and energies
                assert np.array_equal(out["X"][b], plain["x"]), b
                assert np.array_equal(out["R"][b], plain["r"]), b
                assert np.array_equal(out["energies"][b, :r.iters], plain["energies"]), b
                n_same += 1
            if b % 15 == 0:
                compare_to_oracle(prob.psi, prob.y[b], prob.eps, prob.T, batched_signal(out, b), check_follow=False)
                assert orc.support_score(out["X"][b], prob.supports[b]) == 1.0
        assert n_same == prob.B, n_same


def test_gram_batched_largest_served_dictionary():
    """The 4096 x 16384 dictionary of the served workload (1 GiB Gram
    matrix), 12 signals with K ~ U{4..256}, R = 64: every signal converges,
    recovers its support, equals the plain decode bit for bit, and 3 of them
    meet the literal oracle rule."""
    wl = W.WORKLOADS["served_4dict_poisson2000"]
    N, M = wl["dicts"][3]
    psi = W.gaussian_dictionary(N, M, seed=13)
    g = np.random.default_rng([1, 2])
    ys, sups = [], []
    for _ in range(12):
        K = int(g.integers(4, N // 16 + 1))
        x, supp = W.sparse_signal(M, K, g, wl["values"])
        ys.append(W.encode(psi, x))
        sups.append(supp)
    Y = np.stack(ys)
    p = B().MP_PREC_BF16
    with GpuPlan(psi, prec_mask=1 << p) as pl:
        pl.set(B().MP_OPT_BATCH_GRAM, 64)
        out = batched_decode(pl, p, Y, (wl["eps"], wl["T"]), wl["T"])
        assert out["status"] == 0
        n_same = 0
        for b in range(len(ys)):
            r = out["results"][b]
            assert r.status == 0 and r.stop_reason == B().MP_STOP_CONVERGED, b
            assert orc.support_score(out["X"][b], sups[b]) == 1.0, b
            plain = pl.decode(Y[b], wl["eps"], wl["T"])
            if r.iters == plain["result"].iters and np.array_equal(out["atoms"][b, :r.iters], plain["atoms"]):
                assert np.array_equal(out["X"][b], plain["x"]), b
                n_same += 1
        assert n_same == len(ys), n_same
    for b in (0, 5, 11):
        compare_to_oracle(psi, Y[b], wl["eps"], wl["T"], batched_signal(out, b), check_follow=False)


def test_gram_server_mixed_requests_equal_lone_decodes():
    """Requests for two Gram-mode dictionaries (R = 32) submitted while
    others run: each result equals the same signal decoded alone by
    mp_recover_batched in the same mode, bit for bit."""
    from test_server_gpu import lone, wait_all
    prec = B().MP_PREC_BF16
    dicts = [(256, 1024), (512, 2048)]
    psis = [W.gaussian_dictionary(N, M, seed=30 + i) for i, (N, M) in enumerate(dicts)]
    plans = [GpuPlan(p, prec_mask=1 << prec) for p in psis]
    for pl in plans:
        pl.set(B().MP_OPT_BATCH_GRAM, 32)
    srv = B().mp_server_create(4 << 30, 64, 10000)
    try:
        ids = [B().mp_server_add_dictionary(srv, pl.plan, prec) for pl in plans]
        rng = np.random.default_rng(9)
        reqs = []
        for k in range(120):
            d = int(rng.integers(0, 2))
            N, M = dicts[d]
            K = int(rng.integers(4, N // 16 + 1))
            reqs.append((d, W.make_plain(N, M, K, seed=3000 + k, eps=1e-5, T=4000, psi=psis[d])))
        tickets, M_of = [], {}
        for i, (d, prob) in enumerate(reqs):
            s, t = B().mp_server_submit(srv, ids[d], np.ascontiguousarray(prob.y[0]), prob.eps, prob.T)
            assert s == 0
            tickets.append(t)
            M_of[t] = prob.M
            if i % 20 == 19:
                time.sleep(0.002)
        out = wait_all(srv, tickets, M_of)
    finally:
        B().mp_server_destroy(srv)
    try:
        for t, (d, prob) in zip(tickets, reqs):
            res, x = out[t]
            s, r1, x1 = lone(plans[d], prec, prob.y[0], prob.eps, prob.T)
            assert s == 0 and res.status == 0
            assert res.iters == r1.iters and np.array_equal(x, x1), t
            assert orc.support_score(x, prob.supports[0]) == 1.0
    finally:
        for pl in plans:
            pl.close()


def test_gram_option_checks():
    psi = W.gaussian_dictionary(64, 300, seed=3)
    with GpuPlan(psi, prec_mask=(1 << B().MP_PREC_BF16) | (1 << B().MP_PREC_FP8E4M3)) as pl:
        for bad in (1, 8, 17, 40, -16):
            with pytest.raises(B().MpError) as ei:
                pl.set(B().MP_OPT_BATCH_GRAM, bad)
            assert ei.value.status == B().MP_ERR_INVALID
        # Gram steps read the FP32 atoms only: an FP8 plan runs them too, and
        # each signal equals its plain FP32 decode
        pl.set(B().MP_OPT_BATCH_GRAM, 32)
        prob = W.make_batched(64, 300, 4, 1, 3, seed=2, psi=psi, eps=1e-5, T=500)
        out = batched_decode(pl, B().MP_PREC_FP8E4M3, prob.y, (prob.eps, prob.T), 500)
        assert out["status"] == 0
        for b in range(prob.B):
            plain = pl.decode(prob.y[b], prob.eps, prob.T)
            assert np.array_equal(out["X"][b], plain["x"]), b
        pl.set(B().MP_OPT_BATCH_GRAM, 0)
        out = batched_decode(pl, B().MP_PREC_FP8E4M3, prob.y, (prob.eps, prob.T), 500)
        assert out["status"] == 0


def _same_decodes(out, ref, n):
    for b in range(n):
        r, r0 = out["results"][b], ref["results"][b]
        assert (r.status, r.stop_reason, r.iters) == (r0.status, r0.stop_reason, r0.iters), b
        assert r.rel_residual == r0.rel_residual and r.energy_audit_max == r0.energy_audit_max, b
    for k in ("X", "atoms", "coefs", "energies", "R"):
        assert np.array_equal(out[k], ref[k], equal_nan=True), k


@pytest.mark.parametrize("S", [1, 64, 299, 300])
def test_switched_batched_equals_direct(S):
    """300 signals, R = 64: S = 300 (the whole batch) starts with Gram steps,
    S = 299 switches after the first replay, S = 64 part-way, S = 1 at the
    tail.  Every signal equals the direct decode bit for bit; sampled
    signals meet the oracle rule on their own atoms and residual."""
    prob = W.make_batched(256, 1024, 300, 2, 16, seed=5, eps=1e-5, T=3000)
    p = B().MP_PREC_BF16
    with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
        l0 = pl.query(B().MP_Q_KERNEL_LAUNCHES)
        ref = batched_decode(pl, p, prob.y, (prob.eps, prob.T), 3000)
        l1 = pl.query(B().MP_Q_KERNEL_LAUNCHES)
        assert ref["status"] == 0
        pl.set(B().MP_OPT_BATCH_GRAM, 64)
        pl.set(B().MP_OPT_BATCH_GRAM_BELOW, S)
        out = batched_decode(pl, p, prob.y, (prob.eps, prob.T), 3000)
        l2 = pl.query(B().MP_Q_KERNEL_LAUNCHES)
        assert out["status"] == 0
        assert pl.query(B().MP_Q_BATCH_GRAM_BELOW) == S and pl.query(B().MP_Q_BATCH_GRAM) == 64
        _same_decodes(out, ref, prob.B)
        if S >= 64:
            # Gram steps are one launch, direct steps two: the switch happened
            assert l2 - l1 < l1 - l0, (l1 - l0, l2 - l1)
        for b in range(0, prob.B, 60):
            compare_to_oracle(prob.psi, prob.y[b], prob.eps, prob.T, batched_signal(out, b), check_follow=False,
                              gram_period=64, gram_rescored=True)
            assert orc.support_score(out["X"][b], prob.supports[b]) == 1.0


@pytest.mark.parametrize("R,S", [(256, 0), (512, 896), (256, 512)], ids=["gram_R256", "switch896_R512", "switch512_R256"])
def test_gram_full_bf16_workload_equals_direct(R, S):
    """The 1024-signal BF16 workload (N = 2048, M = 8192) in the benchmark's
    Gram settings (every step a Gram step with R = 256; direct steps down to
    896 active signals, then Gram steps with R = 512) and one more switch
    point: all 1024 decodes equal the direct decodes bit for bit, and 4
    sampled signals meet the oracle rule."""
    name = "batched_bf16_N2048_M8192_B1024"
    prob = W.make_workload(name, seed=0)
    p = B().MP_PREC_BF16
    with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
        ref = batched_decode(pl, p, prob.y, (prob.eps, prob.T), 1024)
        assert ref["status"] == 0
        pl.set(B().MP_OPT_BATCH_GRAM, R)
        pl.set(B().MP_OPT_BATCH_GRAM_BELOW, S)
        out = batched_decode(pl, p, prob.y, (prob.eps, prob.T), 1024)
        assert out["status"] == 0
    _same_decodes(out, ref, prob.B)
    for b in (0, 341, 682, 1023):
        d = compare_to_oracle(prob.psi, prob.y[b], prob.eps, prob.T, batched_signal(out, b), check_follow=False,
                              gram_period=R, gram_rescored=True,
                              label=f"{name}[{b}] R={R} S={S}")
        assert d["x_rel_err"] <= 1e-4


def test_switched_option_checks():
    psi = W.gaussian_dictionary(64, 300, seed=3)
    p = B().MP_PREC_BF16
    with GpuPlan(psi, prec_mask=1 << p) as pl:
        with pytest.raises(B().MpError) as ei:
            pl.set(B().MP_OPT_BATCH_GRAM_BELOW, -1)
        assert ei.value.status == B().MP_ERR_INVALID
        # without a Gram period the threshold has no effect: direct steps
        pl.set(B().MP_OPT_BATCH_GRAM_BELOW, 8)
        prob = W.make_batched(64, 300, 4, 1, 3, seed=2, psi=psi, eps=1e-5, T=500)
        out = batched_decode(pl, p, prob.y, (prob.eps, prob.T), 500)
        assert out["status"] == 0
        assert pl.query(B().MP_Q_BATCH_GRAM_BELOW) == 0 and pl.query(B().MP_Q_BATCH_GRAM) == 0


def test_gram_fp8_full_workload():
    """The FP8 workload's dictionary (N = 8192, M = 32768, 4 GiB Gram
    matrix), its 256 signals decoded with Gram steps (R = 512) on an FP8
    plan: every signal converges and recovers its support, 8 sampled signals
    equal the plain FP32 decode bit for bit, and one meets the oracle rule
    against a full FP64 oracle decode."""
    name = "batched_fp8_N8192_M32768_B256"
    prob = W.make_workload(name, seed=0)
    p = B().MP_PREC_FP8E4M3
    with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
        pl.set(B().MP_OPT_BATCH_GRAM, 512)
        out = batched_decode(pl, p, prob.y, (prob.eps, prob.T), 4096)
        assert out["status"] == 0
        assert pl.query(B().MP_Q_GRAM_BYTES) == prob.M * prob.M * 4
        res = out["results"]
        assert all(r.status == 0 and r.stop_reason == B().MP_STOP_CONVERGED for r in res)
        assert min(orc.support_score(out["X"][b], prob.supports[b]) for b in range(prob.B)) == 1.0
        for b in range(0, prob.B, 32):
            plain = pl.decode(prob.y[b], prob.eps, prob.T)
            assert res[b].iters == plain["result"].iters, b
            assert np.array_equal(out["X"][b], plain["x"]), b
    d = compare_to_oracle(prob.psi, prob.y[128], prob.eps, prob.T, batched_signal(out, 128), check_follow=False,
                          gram_period=512, gram_rescored=True,
                          label=f"{name}[128] Gram R=512")
    assert d["x_rel_err"] <= 1e-4


@pytest.mark.parametrize("R,S", [(32, 0), (32, 4), (16, 1)], ids=["gram", "switch4", "switch1"])
def test_gram_edge_cases(R, S):
    """The edge cases of the direct batched decode in the Gram and switched
    modes: y = 0, T = 0, a non-finite signal, eps above 1 and eps = 0 beside a
    normal signal; every signal's result equals the direct decode's, and a
    second call with one signal on the same plan equals its first decode."""
    psi = W.gaussian_dictionary(64, 300, seed=2)
    prob = W.make_batched(64, 300, 6, 1, 3, seed=2, psi=psi, eps=1e-5, T=500)
    Y = prob.y.copy()
    Y[1] = 0.0                  # y = 0
    Y[3, 7] = np.nan            # non-finite signal
    stops = [(1e-5, 500), (1e-5, 500), (1e-5, 0), (1e-5, 500), (2.0, 500), (0.0, 9)]
    p = B().MP_PREC_BF16
    with GpuPlan(psi, prec_mask=1 << p) as pl:
        ref = batched_decode(pl, p, Y, stops, 500)
        pl.set(B().MP_OPT_BATCH_GRAM, R)
        pl.set(B().MP_OPT_BATCH_GRAM_BELOW, S)
        out = batched_decode(pl, p, Y, stops, 500)
        assert ref["status"] == out["status"] == B().MP_ERR_NONFINITE
        for b in range(6):
            r, r0 = out["results"][b], ref["results"][b]
            assert (r.status, r.stop_reason, r.iters) == (r0.status, r0.stop_reason, r0.iters), b
        for b in (0, 1, 2, 4, 5):
            assert np.array_equal(out["X"][b], ref["X"][b]), b
            n = out["results"][b].iters
            assert np.array_equal(out["atoms"][b, :n], ref["atoms"][b, :n]), b
        assert out["results"][5].iters == 9 and out["results"][1].stop_reason == B().MP_STOP_ZERO_Y
        one = batched_decode(pl, p, prob.y[:1], (1e-5, 500), 500)
        assert one["status"] == 0 and one["results"][0].iters == out["results"][0].iters
        assert np.array_equal(one["X"][0], out["X"][0])
