"""The FP64 OMP oracle against facts its definition fixes, and planted
mistakes in an in-memory copy of it that those checks must catch."""
import os
import types

import numpy as np
import pytest

import omp_pins as P
from oracle import omp_oracle as orc
from paper_0809_1833_gb300 import workloads as W

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "omp_oracle.py")

MUTATIONS = {
    "mp_update_instead_of_fit": ("        xs = np.linalg.lstsq(A, y, rcond=None)[0]   # step 3\n"
                                 "        r = y - A @ xs                              # step 4\n",
                                 "        xs = np.append(xs, c[i])\n        r = r - c[i] * P[i]\n"),
    "argmax_signed": ("        a = np.abs(c)\n        i = int(np.argmax(a))\n        if S:",
                      "        a = c\n        i = int(np.argmax(a))\n        if S:"),
    "ties_to_largest_index": ("        i = int(np.argmax(a))\n        if S:",
                              "        i = int(len(a) - 1 - np.argmax(a[::-1]))\n        if S:"),
    "residual_from_previous_r": ("        r = y - A @ xs                              # step 4",
                                 "        r = r - A @ xs"),
    "fit_on_last_atom_only": ("        A = P[S].T\n        xs = np.linalg.lstsq(A, y, rcond=None)[0]   # step 3",
                              "        A = P[S[-1:]].T\n        xs = np.linalg.lstsq(A, y, rcond=None)[0]   # step 3"),
    "stale_energy": ("        e = float(np.dot(r, r))\n        t += 1", "        t += 1"),
    "stop_strict": ("    while e > thr2 and t < T:", "    while e >= thr2 and t < T:"),
    "x_scattered_to_wrong_atoms": ("        x[S] = xs", "        x[np.sort(S)] = xs"),
    # the top-two gap behind the parity tests' near-tie window
    "gap_absolute": ("gaps.append((float(a[i]) - second) / float(a[i]) if a[i] > 0 else 0.0)",
                     "gaps.append(float(a[i]) - second)"),
    "gap_after_update": ("second = float(np.partition(a, M - 2)[M - 2])",
                         "a = np.abs(P @ r); second = float(np.partition(a, M - 2)[M - 2])"),
    "gap_second_distinct_value": ("second = float(np.partition(a, M - 2)[M - 2])",
                                  "second = float(np.max(a[a < a[i]])) if np.any(a < a[i]) else 0.0"),
    "gap_second_is_max": ("second = float(np.partition(a, M - 2)[M - 2])",
                          "second = float(np.partition(a, M - 1)[M - 1])"),
    # follow mode
    "follow_ratio_of_cmax_signed": ("        cmax = float(np.max(np.abs(c)))\n        ratio[k]",
                                    "        cmax = float(np.max(c))\n        ratio[k]"),
    "follow_rnorm_after_fit": ("        rnorm[k] = float(np.sqrt(np.dot(r, r)))\n        S.append(int(i))\n"
                               "        A = P[S].T\n        xs = np.linalg.lstsq(A, y, rcond=None)[0]\n"
                               "        r = y - A @ xs\n",
                               "        S.append(int(i))\n        A = P[S].T\n"
                               "        xs = np.linalg.lstsq(A, y, rcond=None)[0]\n        r = y - A @ xs\n"
                               "        rnorm[k] = float(np.sqrt(np.dot(r, r)))\n"),
}


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda f: f.__name__)
def test_pin(check):
    check(orc)


def _mutant(old, new):
    with open(SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation anchor {old!r} not unique"
    mod = types.ModuleType("mutant_omp_oracle")
    exec(compile(src.replace(old, new), "mutant_omp_oracle", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name):
    mod = _mutant(*MUTATIONS[name])
    caught = []
    for check in P.ALL_CHECKS:
        try:
            check(mod)
        except Exception:
            caught.append(check.__name__)
    assert caught, f"planted mistake {name} passed every pin"


def test_follow_mode():
    prob = W.make_plain(48, 160, 6, seed=4)
    out = orc.omp(prob.psi, prob.y[0], 1e-7, 100)
    f = orc.follow(prob.psi, prob.y[0], out["atoms"])
    assert np.all(f["ratio"] == 1.0)
    assert np.allclose(f["x"], out["x"], atol=1e-14)
    bad = out["atoms"].copy()
    bad[1] = (bad[1] + 1) % prob.M
    assert orc.follow(prob.psi, prob.y[0], bad)["ratio"][1] < 1.0
