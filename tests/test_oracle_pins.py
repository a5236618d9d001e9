"""The FP64 oracle against facts fixed by the paper and the mathematics."""
import numpy as np
import pytest

import oracle_pins as P
from oracle import mp_oracle as orc
from oracle.brute import l0_supports, mp_loops
from paper_0809_1833_gb300 import workloads as W


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda f: f.__name__)
def test_pin(check):
    check(orc)


def test_worked_example_loops_agree():
    g = P.load_worked_example()
    b = mp_loops(g["psi_atoms"], g["y"], g["eps"], g["T"])
    assert b["atoms"] == g["expected"]["atoms"]
    assert list(b["x"]) == g["expected"]["x"]


def test_follow_mode():
    prob = W.make_plain(64, 256, 6, seed=4, eps=1e-6, T=300)
    out = orc.mp(prob.psi, prob.y[0], prob.eps, prob.T)
    f = orc.follow(prob.psi, prob.y[0], out["atoms"])
    assert np.all(f["ratio"] == 1.0)
    assert np.array_equal(f["x"], out["x"])
    bad = out["atoms"].copy()
    bad[2] = (bad[2] + 1) % prob.M
    g = orc.follow(prob.psi, prob.y[0], bad)
    assert g["ratio"][2] < 1.0 and np.all(g["ratio"][:2] == 1.0)


def test_l0_unique_support_two_sparse():
    """Eq. 6 by enumeration: a 2-sparse instance on a 6x10 Gaussian
    dictionary has a unique sparsest support, the generator's."""
    prob = W.make_plain(6, 10, 2, seed=1, eps=1e-6, T=50)
    k, sup = l0_supports(prob.psi, prob.y[0].astype(np.float64), 3, tol=1e-6)
    assert k == 2 and sup == [tuple(prob.supports[0].tolist())]


def test_recovery_regime_small_workload():
    """K/N = 1/16 (the paper's exact-recovery regime, Sec. 3): the FP64
    oracle recovers the support and E(sigma, rho) is tiny."""
    prob = W.make_workload("plain_fp32_N256_M1024_K16", seed=0)
    out = orc.mp(prob.psi, prob.y[0], prob.eps, prob.T)
    assert out["stop_reason"] == 0
    assert orc.support_score(out["x"], prob.supports[0]) == 1.0
    assert orc.reconstruction_error(out["x"], prob.x_true[0]) < 1e-6


def test_error_metrics():
    x = np.array([0.0, 1.0, -2.0, 0.0])
    assert orc.reconstruction_error(x, x) == 0.0
    assert orc.reconstruction_error(np.zeros(4), x) == 100.0
    assert orc.support_score(np.array([0, 5.0, -1, 0]), np.array([1, 2])) == 1.0
    assert orc.support_score(np.array([3.0, 5.0, 0, 0]), np.array([1, 2])) == 0.5


def test_generators_unit_columns():
    for psi in (W.gaussian_dictionary(100, 300, 0), W.bernoulli_dictionary(64, 100, 0)):
        n = np.linalg.norm(psi.astype(np.float64), axis=1)
        assert np.max(np.abs(n - 1.0)) < 1e-6
    b = W.bernoulli_dictionary(256, 50, 0).astype(np.float64)
    assert np.array_equal(np.einsum("mn,mn->m", b, b), np.ones(50))
    prob = W.make_batched(64, 256, 5, 2, 6, seed=0)
    for bi in range(prob.B):
        assert 2 <= len(prob.supports[bi]) <= 6
        assert np.all(np.abs(prob.x_true[bi][prob.supports[bi]]) >= 1.0)
