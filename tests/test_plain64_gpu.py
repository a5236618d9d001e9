"""Parity of the FP64 persistent decode (mp_recover_f64) with the FP64 oracle.

The FP64 decode is the FP32 kernel instantiated for double: the same three
launch shapes, with a 128-bit argmax key and a per-CTA slot exchange instead
of the 64-bit atomic max.  Both it and the oracle compute in FP64, so the
comparison rule runs with gamma_d = d 2^-53 and a near-tie floor of 1e-13:
the atom sequence must equal the oracle's except at ties within FP64
rounding, and x~ must agree to 1e-9 relative.
"""
import numpy as np
import pytest

import oracle_pins as P
from gpu_helpers import GpuPlan, compare_to_oracle
from oracle import mp_oracle as orc
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MODES = [1, 2, 3]
X_TOL64 = 1e-9


def B():
    from paper_0809_1833_gb300 import binding
    return binding


def plan64(psi, mode=0, master64=False):
    pl = GpuPlan(psi, prec_mask=1 << B().MP_PREC_FP64, master64=master64)
    if mode:
        pl.set(B().MP_OPT_PLAIN_MODE, mode)
        if pl.query(B().MP_Q_PLAIN64_MODE) != mode:
            pl.close()
            pytest.skip(f"launch shape {mode} does not fit this FP64 dictionary")
    return pl


@pytest.mark.parametrize("mode", MODES)
def test_worked_example_bit_exact_fp64(mode):
    """The dyadic closed-form instance is exact in FP64 too: atoms, the
    step-1 tie to the smaller index, coefficients, energies, x~ and t = 10
    at the equality e = eps^2 e0."""
    g = P.load_worked_example()
    ex = g["expected"]
    with plan64(np.array(g["psi_atoms"], dtype=np.float32), mode) as pl:
        out = pl.decode64(np.array(g["y"], dtype=np.float64), g["eps"], g["T"])
    assert out["result"].iters == ex["iters"]
    assert out["result"].stop_reason == ex["stop_reason"]
    assert list(out["atoms"]) == ex["atoms"]
    assert np.array_equal(out["coefs"], np.array(ex["coefs"]))
    assert np.array_equal(out["energies"], np.array(ex["energies"]))
    assert np.array_equal(out["x"], np.array(ex["x"]))
    assert out["result"].energy_audit_max == 0.0


SHAPES = [
    # (N, M, K, eps, T, seed)
    (256, 1024, 16, 1e-9, 20000, 0),
    (100, 333, 6, 1e-9, 5000, 1),         # N not a multiple of 32, M ragged over CTAs
    (1000, 3001, 40, 1e-10, 5000, 3),
    (64, 5, 1, 1e-12, 100, 4),            # fewer atoms than CTAs
    (1, 1, 1, 1e-12, 10, 5),              # N = M = 1
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"N{s[0]}_M{s[1]}_K{s[2]}")
def test_fp64_parity_with_oracle(shape, mode):
    """FP32-stored dictionary widened exactly (the oracle's input), y widened
    from FP32: both sides see the same numbers."""
    N, M, K, eps, T, seed = shape
    prob = W.make_plain(N, M, K, seed=seed, eps=eps, T=T)
    y = prob.y[0].astype(np.float64)
    with plan64(prob.psi, mode) as pl:
        out = pl.decode64(y, eps, T)
    # (64, 5, 1): eps = 1e-12 with 5 atoms in R^64 is past what FP64
    # resolves; the run ends at T with r at the rounding floor, where
    # rounding decides the later selections: the FP64-bound rule there
    d = compare_to_oracle(prob.psi, y, eps, T, out, x_tol=X_TOL64, fp64=True, strict=(N, M) != (64, 5))
    assert out["result"].status == 0
    assert d["first_divergence"] is None or d["first_near_tie"] is not None


def test_fp64_modes_agree_bitwise():
    prob = W.make_plain(128, 700, 10, seed=11, eps=1e-10, T=3000)
    y = prob.y[0].astype(np.float64)
    outs = []
    for mode in MODES:
        with plan64(prob.psi, mode) as pl:
            outs.append(pl.decode64(y, prob.eps, prob.T))
    for o in outs[1:]:
        assert np.array_equal(o["atoms"], outs[0]["atoms"])
        assert np.array_equal(o["x"], outs[0]["x"])
        assert np.array_equal(o["energies"], outs[0]["energies"])


@pytest.mark.parametrize("case", [(1500, 600, 1), (3500, 600, 1), (4500, 600, 2), (7500, 300, 2), (9000, 150, 3)],
                         ids=lambda c: f"N{c[0]}_pieces{c[2]}")
def test_fp64_cooperative_stream_matches_resident_bitwise(case):
    """FP64 atoms of 8 KB and more (12, 28, 36, 60 and 72 KB here): 4 warps
    share every stage, each summing one class of
    segments (the FP64 correlation order is defined by those classes),
    atoms above 32 KB stream as pieces of whole 4-segment groups, the
    warps' chains running on across the pieces, and where the ring holds
    two atoms two such groups of warps take alternate atoms.  The
    grid-resident shape computes the same sums with one warp per atom: the
    two must agree bit for bit, and both meet the oracle rule."""
    N, M, pieces = case
    prob = W.make_plain(N, M, 10, seed=13, eps=1e-10, T=3000)
    y = prob.y[0].astype(np.float64)
    outs = []
    for mode in (2, 3):
        with plan64(prob.psi, mode) as pl:
            if mode == 3:
                assert pl.query(B().MP_Q_PLAIN64_PIECES) == pieces
                assert pl.query(B().MP_Q_PLAIN64_STAGES) >= 4
            outs.append(pl.decode64(y, prob.eps, prob.T))
    for k in ("atoms", "x", "energies", "r"):
        assert np.array_equal(outs[0][k], outs[1][k]), k
    # with M < N the FP32-rounded y keeps a part outside the atoms' span:
    # ||r|| stays far above eps ||y|| while the correlations decay to the
    # rounding floor, and the run ends at T with rounding deciding near ties
    compare_to_oracle(prob.psi, y, prob.eps, prob.T, outs[1], x_tol=X_TOL64, fp64=True, strict=M >= N)


def test_fp64_master_paper_timing_instance():
    """Sec. 4's double-precision workload at its smallest size (M = 1000,
    N = 500, K = 70, Bernoulli Psi drawn in FP64, eps = 1e-7, T = N), from an
    FP64 master dictionary, against the oracle on the same FP64 numbers."""
    prob = W.paper_timing_problem(1000, seed=0, fp64=True)
    with plan64(prob.psi, master64=True) as pl:
        out = pl.decode64(prob.y[0], prob.eps, prob.T)
    compare_to_oracle(prob.psi, prob.y[0], prob.eps, prob.T, out, x_tol=X_TOL64, fp64=True)


def test_fp64_orthonormal_recovers_in_k_steps():
    """Orthonormal Psi: c = x, so MP picks the K nonzeros in order of
    decreasing |x_m| and stops after exactly K steps with x~ = x."""
    N, K = 96, 7
    Q = W.orthonormal_dictionary(N, seed=3)
    g = np.random.default_rng(12)
    supp = g.choice(N, size=K, replace=False)
    x = np.zeros(N)
    x[supp] = (np.arange(K) + 1.0) * np.where(g.random(K) < 0.5, -1, 1) * 0.37
    y = x @ Q
    with plan64(Q, master64=True) as pl:
        out = pl.decode64(y, 1e-12, 100)
    assert out["result"].iters == K
    assert list(out["atoms"]) == list(supp[np.argsort(-np.abs(x[supp]), kind="stable")])
    assert np.max(np.abs(out["x"] - x)) <= 1e-13


@pytest.mark.parametrize("mode", MODES)
def test_fp64_edge_cases(mode):
    prob = W.make_plain(128, 512, 8, seed=7)
    y = prob.y[0].astype(np.float64)
    with plan64(prob.psi, mode) as pl:
        z = pl.decode64(np.zeros(128), 1e-5, 100)
        assert z["result"].iters == 0 and z["result"].stop_reason == B().MP_STOP_ZERO_Y
        assert not np.any(z["x"])
        t0 = pl.decode64(y, 1e-5, 0)
        assert t0["result"].iters == 0 and t0["result"].stop_reason == B().MP_STOP_MAX_ITERS
        capped = pl.decode64(y, 0.0, 7, trace_cap=3)
        assert capped["result"].iters == 7 and len(capped["atoms"]) == 3
        ora = orc.mp(prob.psi, y, 0.0, 7)
        assert list(capped["atoms"]) == list(ora["atoms"][:3])
        bad = y.copy()
        bad[5] = np.inf
        nf = pl.decode64(bad, 1e-5, 100, raise_on_error=False)
        assert nf["status"] == B().MP_ERR_NONFINITE and nf["result"].iters == 0
        ok = pl.decode64(y, 1e-9, 1000)
        compare_to_oracle(prob.psi, y, 1e-9, 1000, ok, x_tol=X_TOL64, fp64=True)


def test_fp64_needs_the_fp64_copy():
    import torch
    prob = W.make_plain(64, 200, 3, seed=9)
    with GpuPlan(prob.psi) as pl:                       # FP32 only
        assert pl.query(B().MP_Q_PLAIN64_MODE) == 0
        y = torch.zeros(64, dtype=torch.float64, device="cuda")
        x = torch.zeros(200, dtype=torch.float64, device="cuda")
        s, _ = B().mp_recover_f64(pl.plan, y.data_ptr(), x.data_ptr(), 1e-5, 10, raise_on_error=False)
        assert s == B().MP_ERR_UNSUPPORTED
    with plan64(prob.psi) as pl:
        Y = torch.zeros((2, 64), dtype=torch.float32, device="cuda")
        X = torch.zeros((2, 200), dtype=torch.float32, device="cuda")
        s, _ = B().mp_recover_batched(pl.plan, B().MP_PREC_FP64, Y.data_ptr(), X.data_ptr(), 2, (1e-5, 10),
                                      raise_on_error=False)
        assert s == B().MP_ERR_UNSUPPORTED


@pytest.mark.parametrize("case", [(256, 2), (256, 3), (4500, 3)], ids=lambda c: f"N{c[0]}_mode{c[1]}")
def test_fp64_watchdog_times_out_and_context_survives(case):
    """One CTA skips its first grid-barrier arrival: every other CTA's bounded
    wait expires, the call returns MP_ERR_TIMEOUT and the next call on the
    same plan decodes normally.  N = 4500 runs the shared-stage shape (two
    groups of 4 warps, atoms in 2 pieces), whose producer and consumers must
    leave cleanly too."""
    N, mode = case
    prob = W.make_plain(N, 4096 if N <= 256 else 600, 10, seed=8, eps=1e-9, T=1000)
    y = prob.y[0].astype(np.float64)
    with plan64(prob.psi, mode) as pl:
        pl.set(B().MP_OPT_WATCHDOG_NS, 50_000_000)
        pl.set(B().MP_OPT_DEBUG_SKIP_ARRIVE, 1)
        bad = pl.decode64(y, prob.eps, prob.T, raise_on_error=False)
        assert bad["status"] == B().MP_ERR_TIMEOUT
        pl.set(B().MP_OPT_DEBUG_SKIP_ARRIVE, -1)
        good = pl.decode64(y, prob.eps, prob.T)
    compare_to_oracle(prob.psi, y, prob.eps, prob.T, good, x_tol=X_TOL64, fp64=True)


def test_fp64_largest_paper_timing_size_properties():
    """M = 15000, N = 7500 (900 MB FP64 dictionary, grid streaming): at full
    size the oracle cannot replay all N steps in seconds, so check what holds
    at any size -- the identity y = Psi x~ + r in FP64, energy conservation,
    the stop rule -- and replay the first 40 selected atoms in the oracle's
    follow mode (each must be an FP64 MP choice)."""
    prob = W.paper_timing_problem(15000, seed=0, fp64=True)
    psi, y = prob.psi, prob.y[0]
    with plan64(psi, master64=True) as pl:
        assert pl.query(B().MP_Q_PLAIN64_MODE) == 3
        out = pl.decode64(y, prob.eps, prob.T)
    res = out["result"]
    assert res.status == 0 and 0 < res.iters <= prob.T
    assert (res.stop_reason == B().MP_STOP_CONVERGED) == (res.rel_residual <= prob.eps)
    ident = np.linalg.norm(y - out["x"] @ psi - out["r"]) / np.linalg.norm(y)
    assert ident <= 1e-12, ident
    assert res.energy_audit_max <= 1e-12
    f = orc.follow(psi, y, out["atoms"][:40])
    assert np.all(f["ratio"] >= 1 - 1e-12), f["ratio"].min()
