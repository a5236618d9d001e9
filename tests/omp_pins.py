"""Checks that pin the FP64 OMP oracle (oracle/omp_oracle.py) to facts the
method's definition fixes; each takes the oracle module so a planted
mistake can be run through the same checks."""
import json
import os

import numpy as np

from paper_0809_1833_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "omp_worked_example_N2_M3.json")


def load_worked_example():
    with open(GOLDEN) as f:
        return json.load(f)


def check_worked_example(orc):
    """Hand-derived instance where the least-squares fit differs from MP's
    update at step 2 (x~_2 moves from 36/25 to 9/8)."""
    g = load_worked_example()
    ex = g["expected"]
    out = orc.omp(g["psi_atoms"], g["y"], g["eps"], g["T"])
    assert out["iters"] == ex["iters"] and out["stop_reason"] == ex["stop_reason"]
    assert list(out["atoms"]) == ex["atoms"]
    assert np.allclose(out["coefs"], ex["coefs"], rtol=0, atol=1e-14)
    assert np.allclose(out["x"], ex["x"], rtol=0, atol=1e-14)
    assert np.linalg.norm(out["r"]) <= 1e-14
    # top-two gaps before each selection, by hand: 1/6, then 1/4
    assert np.allclose(out["gaps"], ex["gaps"], rtol=0, atol=1e-14)


def check_follow_worked_example(orc):
    """Follow mode with the imposed order 0, 2 (the reverse of OMP's):
    ratios 5/6 and 4/5, max|c| and ||r|| before each step, the final fit."""
    g = load_worked_example()
    fx = g["follow"]
    f = orc.follow(g["psi_atoms"], g["y"], fx["atoms"])
    assert np.allclose(f["ratio"], fx["ratio"], rtol=0, atol=1e-14)
    assert np.allclose(f["cmax"], fx["cmax"], rtol=0, atol=1e-14)
    assert np.allclose(f["rnorm"], fx["rnorm"], rtol=0, atol=1e-14)
    assert np.allclose(f["x"], fx["x"], rtol=0, atol=1e-14)
    assert np.linalg.norm(f["r"]) <= 1e-14


def check_orthonormal_equals_mp(orc):
    """Orthonormal Psi: the fit of step 3 equals MP's one-coefficient update,
    so OMP recovers x in exactly K steps in decreasing-|x| order."""
    N, K = 48, 6
    Q = W.orthonormal_dictionary(N, seed=2)
    g = np.random.default_rng(3)
    supp = g.choice(N, size=K, replace=False)
    x = np.zeros(N)
    x[supp] = (np.arange(K) + 1.0) * 0.3 * np.where(g.random(K) < 0.5, -1, 1)
    out = orc.omp(Q, x @ Q, 1e-12, 100)
    assert out["iters"] == K and out["stop_reason"] == orc.STOP_CONVERGED
    assert list(out["atoms"]) == list(supp[np.argsort(-np.abs(x[supp]), kind="stable")])
    assert np.max(np.abs(out["x"] - x)) <= 1e-12
    # correlations before step k are the unselected entries of x: gap
    # (m_k - m_{k+1}) / m_k with m the sorted magnitudes, 1 at the last step;
    # follow along OMP's own order gives ratio 1, max|c| = m_k (whatever the
    # sign of that entry; here some are negative) and ||r|| = the norm of the
    # unselected entries
    m = np.sort(np.abs(x[supp]))[::-1]
    assert np.max(np.abs(out["gaps"] - np.append((m[:-1] - m[1:]) / m[:-1], 1.0))) <= 1e-12
    f = orc.follow(Q, x @ Q, out["atoms"])
    assert np.all(np.abs(f["ratio"] - 1.0) <= 1e-12)
    assert np.max(np.abs(f["cmax"] - m)) <= 1e-12
    assert np.max(np.abs(f["rnorm"] - np.sqrt(np.cumsum((m ** 2)[::-1])[::-1]))) <= 1e-12


def check_residual_orthogonal_to_selected(orc):
    """After every step r is orthogonal to each selected atom, and no atom
    is selected twice."""
    prob = W.make_plain(40, 120, 8, seed=5)
    psi = prob.psi.astype(np.float64)
    y = prob.y[0].astype(np.float64)
    full = orc.omp(psi, y, 1e-9, 30)
    assert len(set(full["atoms"].tolist())) == len(full["atoms"])
    for k in range(1, full["iters"] + 1):
        o = orc.omp(psi, y, 0.0, k)
        S = o["support"]
        assert np.max(np.abs(psi[S] @ o["r"])) <= 1e-12 * np.linalg.norm(y)
        assert np.allclose(o["x"][S] @ psi[S] + o["r"], y, atol=1e-12)


def check_exact_recovery_in_k_steps(orc):
    """A K-sparse signal with K much smaller than N: once the K support atoms
    are selected, y lies in their span and r = 0, so OMP stops after exactly
    K steps with x~ = x (MP needs many more steps)."""
    prob = W.make_plain(64, 200, 5, seed=9)
    psi = prob.psi.astype(np.float64)
    x = prob.x_true[0]
    y = x @ psi
    out = orc.omp(psi, y, 1e-10, 100)
    assert out["iters"] == 5 and out["stop_reason"] == orc.STOP_CONVERGED
    assert sorted(out["atoms"].tolist()) == sorted(prob.supports[0].tolist())
    assert np.max(np.abs(out["x"] - x)) <= 1e-10


def check_rank_stop(orc):
    """eps = 0 in R^4 with atoms in general position: after 4 steps the
    selected atoms span R^4, r = 0, and the next selection lies in their span."""
    g = np.random.default_rng(7)
    P = g.standard_normal((10, 4))
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    y = g.standard_normal(4)
    out = orc.omp(P, y, 0.0, 50)
    assert out["iters"] == 4
    assert out["stop_reason"] in (orc.STOP_RANK, orc.STOP_CONVERGED)
    assert np.linalg.norm(out["r"]) <= 1e-12 * np.linalg.norm(y)


def check_first_step_is_mp(orc):
    """Step 1 is MP's step: same atom, and for one unit atom the fit equals
    <y, psi_i> (Bernoulli atoms with N = 64 are exactly unit norm)."""
    from oracle import mp_oracle
    prob = W.make_plain(64, 90, 3, seed=11, dictionary="bernoulli")
    a = orc.omp(prob.psi, prob.y[0], 0.0, 1)
    b = mp_oracle.mp(prob.psi, prob.y[0], 0.0, 1)
    assert list(a["atoms"]) == list(b["atoms"])
    assert np.allclose(a["x"], b["x"], rtol=0, atol=1e-15)


def check_stop_reasons(orc):
    P = np.eye(3)
    z = orc.omp(P, np.zeros(3), 1e-6, 5)
    assert z["iters"] == 0 and z["stop_reason"] == orc.STOP_ZERO_Y
    c = orc.omp(P, np.array([3.0, 2.0, 1.0]), 0.0, 2)
    assert c["iters"] == 2 and c["stop_reason"] == orc.STOP_MAX_ITERS
    d = orc.omp(P, np.array([3.0, 2.0, 1.0]), 0.5, 10)
    # e0 = 14, thr2 = 3.5: after atom 0 e = 5, after atom 1 e = 1 <= 3.5
    assert d["iters"] == 2 and d["stop_reason"] == orc.STOP_CONVERGED


def check_tie_goes_to_smallest_index(orc):
    """|c_0| = |c_1| exactly (orthonormal atoms, y = (2, -2, 1)): the smaller
    index is selected first."""
    out = orc.omp(np.eye(3), np.array([2.0, -2.0, 1.0]), 0.0, 3)
    assert list(out["atoms"]) == [0, 1, 2]
    # gaps: |c| = (2, 2, 1) is a tie (0); then (0, 2, 1) gives 1/2; then
    # (0, 0, 1) gives 1
    assert list(out["gaps"]) == [0.0, 0.5, 1.0]


ALL_CHECKS = [check_tie_goes_to_smallest_index, check_worked_example, check_follow_worked_example,
              check_orthonormal_equals_mp, check_residual_orthogonal_to_selected,
              check_exact_recovery_in_k_steps, check_rank_stop, check_first_step_is_mp, check_stop_reasons]
