"""Parity of the persistent FP32 kernel (mp_recover) with the FP64 oracle.

Every case goes through the C ABI.  The three launch shapes (one resident
cluster, grid-resident, grid-streaming) are forced in turn on the same
inputs; they share one per-atom summation order, so they must agree bit for
bit with each other, and each must meet the oracle comparison rule.
"""
import numpy as np
import pytest

import oracle_pins as P
from gpu_helpers import GpuPlan, compare_to_oracle
from oracle import mp_oracle as orc
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MODES = [1, 2, 3]


def B():
    from paper_0809_1833_gb300 import binding
    return binding


@pytest.mark.parametrize("mode", MODES)
def test_worked_example_bit_exact(mode):
    """Closed-form instance: every value is dyadic, so FP32 must reproduce
    the atoms, coefficients, energies and x~ exactly, including the
    smallest-index tie at step 1 and the stop at the equality e = eps^2 e0."""
    g = P.load_worked_example()
    ex = g["expected"]
    psi = np.array(g["psi_atoms"], dtype=np.float32)
    with GpuPlan(psi, mode=mode) as pl:
        out = pl.decode(np.array(g["y"], dtype=np.float32), g["eps"], g["T"])
    assert out["result"].iters == ex["iters"]
    assert out["result"].stop_reason == ex["stop_reason"]
    assert list(out["atoms"]) == ex["atoms"]
    assert np.array_equal(out["coefs"].astype(np.float64), np.array(ex["coefs"]))
    assert np.array_equal(out["energies"], np.array(ex["energies"]))
    assert np.array_equal(out["x"].astype(np.float64), np.array(ex["x"]))
    assert out["result"].energy_audit_max == 0.0


SHAPES = [
    # (N, M, K, eps, T, seed): several tiles, ragged tails, tiny and degenerate sizes
    (256, 1024, 16, 1e-6, 20000, 0),      # small plain workload, full size
    (100, 333, 6, 1e-5, 5000, 1),         # N not a multiple of 32, M ragged over CTAs
    (37, 1000, 2, 1e-4, 2000, 2),
    (1000, 3001, 40, 1e-5, 5000, 3),
    (64, 5, 1, 1e-6, 100, 4),             # fewer atoms than CTAs
    (1, 1, 1, 1e-6, 10, 5),               # N = M = 1
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"N{s[0]}_M{s[1]}_K{s[2]}")
def test_parity_with_oracle(shape, mode):
    N, M, K, eps, T, seed = shape
    prob = W.make_plain(N, M, K, seed=seed, eps=eps, T=T)
    with GpuPlan(prob.psi, mode=mode) as pl:
        if pl.query(B().MP_Q_PLAIN_MODE) != mode:
            pytest.skip(f"launch shape {mode} cannot hold N={N}, M={M}")
        out = pl.decode(prob.y[0], eps, T)
    assert out["status"] == 0
    d = compare_to_oracle(prob.psi, prob.y[0], eps, T, out)
    # the device's FP64 energy audit: e_k = e_{k-1} - c_k^2 up to FP32 drift
    assert out["result"].energy_audit_max <= 1e-5
    assert d["x_rel_err"] <= 1e-4


@pytest.mark.parametrize("shape", [(300, 1500, 12), (1000, 1200, 20)], ids=["N300", "N1000"])
def test_modes_agree_bitwise(shape):
    """Every launch shape computes each correlation in one order and the FP64
    energy in one order (128 chains, whatever the shape's thread count), so
    atoms, x~ and the energies agree bit for bit."""
    N, M, K = shape
    prob = W.make_plain(N, M, K, seed=9, eps=1e-5, T=3000)
    outs = []
    for mode in MODES:
        with GpuPlan(prob.psi, mode=mode) as pl:
            if pl.query(B().MP_Q_PLAIN_MODE) != mode:
                continue
            outs.append(pl.decode(prob.y[0], prob.eps, prob.T))
    assert len(outs) >= 2
    for o in outs[1:]:
        assert np.array_equal(o["atoms"], outs[0]["atoms"])
        assert np.array_equal(o["x"], outs[0]["x"])
        assert np.array_equal(o["energies"], outs[0]["energies"])


@pytest.mark.parametrize("mode", MODES)
def test_deterministic(mode):
    prob = W.make_plain(256, 2048, 24, seed=6, eps=1e-5, T=4000)
    with GpuPlan(prob.psi, mode=mode) as pl:
        assert pl.query(B().MP_Q_PLAIN_MODE) == mode
        a = pl.decode(prob.y[0], prob.eps, prob.T)
        b = pl.decode(prob.y[0], prob.eps, prob.T)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["atoms"], b["atoms"])


@pytest.mark.parametrize("mode", MODES)
def test_edge_cases(mode):
    prob = W.make_plain(128, 512, 8, seed=7)
    with GpuPlan(prob.psi, mode=mode) as pl:
        z = pl.decode(np.zeros(128, np.float32), 1e-5, 100)
        assert z["result"].iters == 0 and z["result"].stop_reason == B().MP_STOP_ZERO_Y
        assert not np.any(z["x"])
        t0 = pl.decode(prob.y[0], 1e-5, 0)
        assert t0["result"].iters == 0 and t0["result"].stop_reason == B().MP_STOP_MAX_ITERS
        assert not np.any(t0["x"]) and t0["result"].rel_residual == 1.0
        one = pl.decode(prob.y[0], 1.0, 100)
        assert one["result"].iters == 0 and one["result"].stop_reason == B().MP_STOP_CONVERGED
        capped = pl.decode(prob.y[0], 0.0, 7)
        assert capped["result"].iters == 7 and capped["result"].stop_reason == B().MP_STOP_MAX_ITERS
        ora = orc.mp(prob.psi, prob.y[0], 0.0, 7)
        assert list(capped["atoms"]) == list(ora["atoms"])
        bad = prob.y[0].copy()
        bad[5] = np.nan
        nf = pl.decode(bad, 1e-5, 100, raise_on_error=False)
        assert nf["status"] == B().MP_ERR_NONFINITE and nf["result"].iters == 0
        # the plan still works after the rejected input
        ok = pl.decode(prob.y[0], 1e-5, 1000)
        # this signal's last steps run at |c| ~ 2e-5 ||y||, where the FP32
        # residual's drift (~4e-8 ||y||) decides near ties: step 24 of 28
        # (oracle gap 7.9e-5) goes either way, so the FP32-bound rule
        compare_to_oracle(prob.psi, prob.y[0], 1e-5, 1000, ok, strict=False)


@pytest.mark.parametrize("mode", [2, 3])
def test_watchdog_times_out_and_context_survives(mode):
    """One CTA never arrives at the first grid barrier: every other CTA's
    bounded wait runs out, the call returns MP_ERR_TIMEOUT, and the next
    decode on the same context is correct."""
    prob = W.make_plain(256, 4096, 10, seed=8, eps=1e-5, T=1000)
    with GpuPlan(prob.psi, mode=mode) as pl:
        pl.set(B().MP_OPT_WATCHDOG_NS, 50_000_000)       # 50 ms
        pl.set(B().MP_OPT_DEBUG_SKIP_ARRIVE, 1)
        bad = pl.decode(prob.y[0], prob.eps, prob.T, raise_on_error=False)
        assert bad["status"] == B().MP_ERR_TIMEOUT
        pl.set(B().MP_OPT_DEBUG_SKIP_ARRIVE, -1)
        good = pl.decode(prob.y[0], prob.eps, prob.T)
    compare_to_oracle(prob.psi, prob.y[0], prob.eps, prob.T, good)


def test_plan_layouts_and_normalisation():
    prob = W.make_plain(96, 400, 5, seed=10, eps=1e-5, T=2000)
    with GpuPlan(prob.psi) as a, GpuPlan(prob.psi, layout_row_major=True) as b:
        oa, ob = a.decode(prob.y[0], prob.eps, prob.T), b.decode(prob.y[0], prob.eps, prob.T)
    assert np.array_equal(oa["x"], ob["x"])
    scaled = prob.psi * np.linspace(0.5, 3.0, prob.M, dtype=np.float32)[:, None]
    with pytest.raises(Exception) as ei:
        GpuPlan(scaled)
    assert getattr(ei.value, "status", None) == B().MP_ERR_INVALID
    with GpuPlan(scaled, normalize=True) as c:
        oc = c.decode(prob.y[0], prob.eps, prob.T)
    compare_to_oracle(prob.psi, prob.y[0], prob.eps, prob.T, oc, x_tol=1e-4)
    nanpsi = prob.psi.copy()
    nanpsi[3, 4] = np.inf
    with pytest.raises(Exception) as ei:
        GpuPlan(nanpsi)
    assert getattr(ei.value, "status", None) == B().MP_ERR_NONFINITE


def test_host_buffer_entry_point():
    prob = W.make_plain(256, 1024, 16, seed=0, eps=1e-6, T=20000)
    with GpuPlan(prob.psi) as pl:
        dev = pl.decode(prob.y[0], prob.eps, prob.T)
        xh = np.full(prob.M, np.nan, np.float32)
        s, res = B().mp_recover_host(pl.plan, np.ascontiguousarray(prob.y[0]), xh, prob.eps, prob.T)
    assert s == 0 and res.iters == dev["result"].iters
    assert np.array_equal(xh, dev["x"])


def test_large_streamed_workload_full_size():
    """The 256 MiB dictionary (N=4096, M=16384, K=256) in the launch shape
    the benchmark times (grid streaming), against the full FP64 oracle."""
    prob = W.make_workload("plain_fp32_N4096_M16384_K256", seed=0)
    with GpuPlan(prob.psi) as pl:
        assert pl.query(B().MP_Q_PLAIN_MODE) == 3
        out = pl.decode(prob.y[0], prob.eps, prob.T)
    d = compare_to_oracle(prob.psi, prob.y[0], prob.eps, prob.T, out, check_follow=False)
    assert out["result"].stop_reason == B().MP_STOP_CONVERGED
    assert orc.support_score(out["x"], prob.supports[0]) == 1.0
    # FP32 atom sequence equals FP64's over the whole decode at this size
    assert d["first_divergence"] is None


def test_cache_policies_do_not_change_results():
    """The streaming shape's L2 hints (evict-first stream, an evict-last
    resident part) and its stage size only move bytes differently: the
    decode is bit for bit the same."""
    prob = W.make_plain(512, 6000, 20, seed=12, eps=1e-6, T=3000)
    outs = []
    for opts in ({}, {B().MP_OPT_PLAIN_EVICT_FIRST: 0}, {B().MP_OPT_PLAIN_L2_KEEP_BYTES: 4 << 20},
                 {B().MP_OPT_PLAIN_STAGE_BYTES: 8192}):
        with GpuPlan(prob.psi, mode=3) as pl:
            for k, v in opts.items():
                pl.set(k, v)
            outs.append(pl.decode(prob.y[0], prob.eps, prob.T))
    for o in outs[1:]:
        for k in ("atoms", "x", "energies", "r"):
            assert np.array_equal(o[k], outs[0][k]), k
