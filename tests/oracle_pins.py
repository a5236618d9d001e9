"""Checks that pin the FP64 oracle to facts the paper and the mathematics fix.

Each ``check_*`` takes an oracle module (anything exposing ``mp`` with the
signature of ``oracle.mp_oracle.mp``) and raises AssertionError when the
module disagrees with the pinned fact.  ``test_oracle_pins.py`` runs them on
the real oracle; ``test_oracle_mutations.py`` runs them on copies of the
oracle with planted mistakes and requires that every mistake is caught.
"""
import json
import os

import numpy as np

from paper_0809_1833_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_worked_example():
    with open(os.path.join(GOLDEN, "worked_example_N4_M6.json")) as f:
        return json.load(f)


def check_worked_example(orc):
    """Closed-form instance: tie-break, sign handling, stop equality case."""
    g = load_worked_example()
    ex = g["expected"]
    out = orc.mp(np.array(g["psi_atoms"]), np.array(g["y"]), g["eps"], g["T"])
    assert out["iters"] == ex["iters"], out["iters"]
    assert out["stop_reason"] == ex["stop_reason"]
    assert list(out["atoms"]) == ex["atoms"]
    assert np.array_equal(out["coefs"], np.array(ex["coefs"]))
    assert np.array_equal(out["x"], np.array(ex["x"]))
    assert np.array_equal(out["energies"], np.array(ex["energies"]))
    # the same values follow from the closed form e_t = 3 * 4^-t
    t = np.arange(1, ex["iters"] + 1)
    assert np.array_equal(out["energies"], 3.0 * 4.0 ** (-t))
    # top-two gaps before each update: the exact tie of step 1 gives 0, every
    # later step 1/3 (1/3 rounded once: 1/4 over 3/4 and its power-of-two
    # scalings are correctly rounded divisions of the same ratio)
    assert np.array_equal(out["gaps"], np.array(ex["gaps"]))
    assert out["gaps"][0] == 0.0 and np.all(out["gaps"][1:] == 1.0 / 3.0)


def check_follow_worked_example(orc):
    """Follow mode on the worked example with an imposed non-MP sequence
    (5, 0, 5), values derived by hand: ratio |c_i| / max|c| before each
    step, max|c| (largest magnitude, whatever its sign), ||r|| before each
    step, and the final x~ and r."""
    g = load_worked_example()
    fx = g["follow"]
    f = orc.follow(np.array(g["psi_atoms"]), np.array(g["y"]), fx["atoms"])
    assert np.allclose(f["ratio"], fx["ratio"], rtol=1e-15, atol=0)
    assert np.array_equal(f["cmax"], np.array(fx["cmax"]))
    assert np.allclose(f["rnorm"] ** 2, fx["rnorm2"], rtol=1e-15, atol=0)
    assert np.array_equal(f["x"], np.array(fx["x"]))
    assert np.array_equal(f["r"], np.array(fx["r"]))


def check_energy_conservation(orc):
    """||r_{k+1}||^2 = ||r_k||^2 - c_k^2 when atoms have unit norm exactly
    (Eq. 11 with Eq. 4: <r - c psi, r - c psi> = e - 2c^2 + c^2)."""
    prob = W.make_plain(64, 256, 6, seed=3, eps=1e-9, T=300, values="pm12",
                        dictionary="bernoulli")
    out = orc.mp(prob.psi, prob.y[0], prob.eps, prob.T)
    e = np.concatenate([[out["e0"]], out["energies"]])
    c = out["coefs"]
    assert out["iters"] > 20
    assert np.max(np.abs(e[1:] - (e[:-1] - c ** 2))) <= 1e-12 * out["e0"]


def check_energy_identity_general(orc):
    """For any atom norm: e_{k+1} = e_k - c^2 (2 - ||psi_i||^2)."""
    prob = W.make_plain(48, 160, 5, seed=11, eps=1e-9, T=200)
    P = prob.psi.astype(np.float64)
    out = orc.mp(prob.psi, prob.y[0], prob.eps, prob.T)
    nrm2 = np.einsum("mn,mn->m", P, P)[out["atoms"]]
    e = np.concatenate([[out["e0"]], out["energies"]])
    c = out["coefs"]
    assert np.max(np.abs(e[1:] - (e[:-1] - c ** 2 * (2.0 - nrm2)))) <= 1e-12 * out["e0"]


def check_monotone_residual(orc):
    prob = W.make_plain(96, 384, 8, seed=5, eps=1e-8, T=400)
    out = orc.mp(prob.psi, prob.y[0], prob.eps, prob.T)
    e = np.concatenate([[out["e0"]], out["energies"]])
    assert out["iters"] > 10
    assert np.all(np.diff(e) <= 1e-15 * out["e0"])


def check_reconstruction_identity(orc):
    """y = Psi x~ + r at the end, x~ summed atom by atom in FP64."""
    prob = W.make_plain(80, 300, 7, seed=2, eps=1e-6, T=500)
    out = orc.mp(prob.psi, prob.y[0], prob.eps, prob.T)
    P = prob.psi.astype(np.float64)
    acc = np.zeros(prob.N)
    for m in np.nonzero(out["x"])[0]:
        acc += out["x"][m] * P[m]
    y = prob.y[0].astype(np.float64)
    assert np.linalg.norm(y - acc - out["r"]) <= 1e-13 * np.linalg.norm(y)
    # and the loop test holds at exit: ||r|| <= eps ||y||
    assert out["stop_reason"] == 0
    assert np.linalg.norm(out["r"]) <= prob.eps * np.linalg.norm(y) * (1 + 1e-12)


def check_orthonormal_exact(orc):
    """Orthonormal Psi (N = M): correlations equal x, so MP recovers x in
    exactly K steps, largest |x_m| first."""
    N, K = 64, 8
    Q = W.orthonormal_dictionary(N, seed=7)
    x = np.zeros(N)
    supp = np.array([3, 9, 17, 22, 40, 41, 55, 63])
    mags = np.linspace(2.0, 1.0, K)
    x[supp] = mags * np.array([1, -1, 1, 1, -1, 1, -1, -1])
    y = x @ Q
    out = orc.mp(Q, y, 1e-10, 1000)
    assert out["iters"] == K
    assert list(out["atoms"]) == list(supp[np.argsort(-mags, kind="stable")])
    assert np.max(np.abs(out["x"] - x)) <= 1e-12
    # before step k the correlations are the not yet selected entries of x
    # (selected ones are 0 up to rounding), so the top-two gap is
    # (m_k - m_{k+1}) / m_k with m sorted by decreasing magnitude, and 1 at
    # the last step
    m = np.sort(mags)[::-1]
    gap = np.append((m[:-1] - m[1:]) / m[:-1], 1.0)
    assert np.max(np.abs(out["gaps"] - gap)) <= 1e-12
    # follow mode along MP's own sequence: ratio 1, max|c| = m_k whatever
    # the sign of that entry, ||r|| = the norm of the entries still unselected
    f = orc.follow(Q, y, out["atoms"])
    assert np.all(np.abs(f["ratio"] - 1.0) <= 1e-12)
    assert np.max(np.abs(f["cmax"] - m)) <= 1e-12
    tail = np.sqrt(np.cumsum((m ** 2)[::-1])[::-1])
    assert np.max(np.abs(f["rnorm"] - tail)) <= 1e-12


def check_against_loops(orc):
    """Same iterates as the explicit-loop version on tiny random inputs."""
    from oracle.brute import mp_loops
    for seed in range(4):
        prob = W.make_plain(5, 9, 2, seed=seed, eps=1e-4, T=60)
        a = orc.mp(prob.psi, prob.y[0], prob.eps, prob.T)
        b = mp_loops(prob.psi, prob.y[0], prob.eps, prob.T)
        assert a["iters"] == b["iters"]
        assert list(a["atoms"]) == list(b["atoms"])
        assert np.allclose(a["x"], b["x"], rtol=0, atol=1e-12)
        assert np.allclose(a["energies"], b["energies"], rtol=1e-10, atol=1e-14)


def check_one_sparse(orc):
    """K = 1: y = x_j psi_j, and |<psi_i, psi_j>| < 1 for i != j, so MP
    selects j first with coefficient x_j and stops after one step."""
    from oracle.brute import l0_supports
    for seed in range(3):
        prob = W.make_plain(6, 10, 1, seed=seed, eps=1e-6, T=50)
        j = int(prob.supports[0][0])
        y = prob.psi[j].astype(np.float64) * prob.x_true[0, j]
        out = orc.mp(prob.psi, y, 1e-6, 50)
        assert out["iters"] == 1 and out["atoms"][0] == j
        assert abs(out["x"][j] - prob.x_true[0, j]) <= 1e-6 * abs(prob.x_true[0, j])
        k, sup = l0_supports(prob.psi, y, 2)
        assert k == 1 and sup == [(j,)]


def check_stop_reasons(orc):
    psi = W.gaussian_dictionary(8, 20, seed=1)
    z = orc.mp(psi, np.zeros(8), 1e-5, 100)
    assert z["iters"] == 0 and z["stop_reason"] == 2 and not np.any(z["x"])
    y = psi[3] * 2.0 + psi[7]
    capped = orc.mp(psi, y, 1e-12, 3)
    assert capped["iters"] == 3 and capped["stop_reason"] == 1
    loose = orc.mp(psi, y, 1.0, 100)                # ||y|| <= 1 * ||y|| at t = 0
    assert loose["iters"] == 0 and loose["stop_reason"] == 0


ALL_CHECKS = [check_worked_example, check_follow_worked_example, check_energy_conservation,
              check_energy_identity_general, check_monotone_residual,
              check_reconstruction_identity, check_orthonormal_exact,
              check_against_loops, check_one_sparse, check_stop_reasons]
