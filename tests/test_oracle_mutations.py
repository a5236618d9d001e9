"""Plants plausible mistakes in an in-memory copy of the oracle and checks
that the pins catch every one of them (the oracle file itself is untouched).
"""
import os
import types

import pytest

import oracle_pins as P

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "mp_oracle.py")

MUTATIONS = {
    "argmax_signed": ("a = np.abs(c)", "a = c"),
    "ties_to_largest_index": ("i = int(np.argmax(a))",
                              "i = int(len(a) - 1 - np.argmax(a[::-1]))"),
    "x_overwrite": ("x[i] += ci", "x[i] = ci"),
    "x_wrong_sign": ("x[i] += ci", "x[i] -= ci"),
    "residual_wrong_sign": ("r -= ci * P[i]", "r += ci * P[i]"),
    "residual_not_updated": ("r -= ci * P[i]", "pass"),
    "transposed_operand": ("c = P @ r ", "c = P.T @ r "),
    "wrong_atom_row": ("r -= ci * P[i]", "r -= ci * P[(i + 1) % M]"),
    "stop_strict": ("while e > thr2 and t < T", "while e >= thr2 and t < T"),
    "listing_threshold": ("thr2 = float(eps) * float(eps) * e0",
                          "thr2 = float(eps) * float(np.sqrt(e0))"),
    "stale_energy": ("e = float(np.dot(r, r))", "e = e"),
    "double_count_t": ("t += 1  ", "t += 2  "),
    "dropped_cap": ("while e > thr2 and t < T", "while e > thr2"),
    # the top-two gap that sets every parity test's near-tie window
    "gap_absolute": ("gaps.append((float(a[i]) - second) / float(a[i]) if a[i] > 0 else 0.0)",
                     "gaps.append(float(a[i]) - second)"),
    "gap_after_update": ("second = float(np.partition(a, M - 2)[M - 2])",
                         "a = np.abs(P @ r); second = float(np.partition(a, M - 2)[M - 2])"),
    "gap_second_distinct_value": ("second = float(np.partition(a, M - 2)[M - 2])",
                                  "second = float(np.max(a[a < a[i]])) if np.any(a < a[i]) else 0.0"),
    "gap_second_signed": ("second = float(np.partition(a, M - 2)[M - 2])",
                          "second = float(np.max(np.delete(c, i)))"),
    "gap_second_is_max": ("second = float(np.partition(a, M - 2)[M - 2])",
                          "second = float(np.partition(a, M - 1)[M - 1])"),
    # follow mode, whose max|c| and ||r|| set the tolerance of rule (iii)
    "follow_ratio_signed": ("ratio[k] = abs(float(c[i])) / cmax if cmax > 0 else 1.0",
                            "ratio[k] = float(c[i]) / cmax if cmax > 0 else 1.0"),
    "follow_cmax_signed": ("cmax = float(np.max(np.abs(c)))", "cmax = float(np.max(c))"),
    "follow_rnorm_after_update": ("        rnorm[k] = float(np.sqrt(np.dot(r, r)))\n        x[i] += float(c[i])\n"
                                  "        r -= float(c[i]) * P[i]\n",
                                  "        x[i] += float(c[i])\n        r -= float(c[i]) * P[i]\n"
                                  "        rnorm[k] = float(np.sqrt(np.dot(r, r)))\n"),
    "follow_x_overwrite": ("x[i] += float(c[i])", "x[i] = float(c[i])"),
}


def _mutant(old, new):
    with open(SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation anchor {old!r} not unique"
    mod = types.ModuleType("mutant_oracle")
    exec(compile(src.replace(old, new), "mutant_oracle", "exec"), mod.__dict__)
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
