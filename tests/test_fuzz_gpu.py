"""Seeded random shapes against the FP64 oracle: sizes that are not multiples
of anything (ragged atom slices, partial 32/64/128-element rows, partial
atom tiles and row tiles), every launch shape that fits, both batched
precisions.  Each case must meet the comparison rule of the fixed-shape
tests."""
import numpy as np
import pytest

from gpu_helpers import GpuPlan, batched_decode, batched_signal, compare_to_oracle
from oracle import mp_oracle as orc
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def B():
    from paper_0809_1833_gb300 import binding
    return binding


def _shapes(n, seed):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        N = int(g.integers(3, 1500))
        M = int(g.integers(2, 6000))
        K = int(max(1, min(M, N // 16 + int(g.integers(0, 3)))))
        out.append((N, M, K, int(g.integers(0, 1 << 30))))
    return out


@pytest.mark.parametrize("shape", _shapes(30, 2024), ids=lambda s: f"N{s[0]}_M{s[1]}_K{s[2]}")
def test_plain_random_shapes_all_launch_shapes(shape):
    N, M, K, seed = shape
    prob = W.make_plain(N, M, K, seed=seed % 1000, eps=1e-5, T=4000)
    ora = orc.mp(prob.psi, prob.y[0], prob.eps, prob.T)
    ran = 0
    for mode in (0, 1, 2, 3):
        with GpuPlan(prob.psi) as pl:
            if mode:
                pl.set(B().MP_OPT_PLAIN_MODE, mode)
                if pl.query(B().MP_Q_PLAIN_MODE) != mode:
                    continue
            out = pl.decode(prob.y[0], prob.eps, prob.T)
        assert out["result"].status == 0
        compare_to_oracle(prob.psi, prob.y[0], prob.eps, prob.T, out, ora=ora)
        ran += 1
    assert ran >= 2


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("case", [(150, 2100, 77), (700, 1300, 300), (33, 4100, 5)],
                         ids=lambda c: f"N{c[0]}_M{c[1]}_B{c[2]}")
def test_batched_random_shapes(case, prec):
    N, M, Bn = case
    prob = W.make_batched(N, M, Bn, 1, max(2, N // 16), seed=N + M, eps=1e-5, T=3000)
    p = B().MP_PREC_BF16 if prec == "bf16" else B().MP_PREC_FP8E4M3
    with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
        out = batched_decode(pl, p, prob.y, (prob.eps, prob.T), 3000)
        X, atoms, res = out["X"], out["atoms"], out["results"]
        assert out["status"] == 0
        for b in sorted({0, Bn // 2, Bn - 1}):
            plain = pl.decode(prob.y[b], prob.eps, prob.T)
            r = res[b]
            same = r.iters == plain["result"].iters and np.array_equal(atoms[b, :r.iters], plain["atoms"])
            if same:
                assert np.array_equal(X[b], plain["x"]), b
                assert np.array_equal(out["R"][b], plain["r"]), b
            compare_to_oracle(prob.psi, prob.y[b], prob.eps, prob.T, batched_signal(out, b), check_follow=not same)


@pytest.mark.parametrize("shape", _shapes(8, 77), ids=lambda s: f"N{s[0]}_M{s[1]}_K{s[2]}")
def test_fp64_gram_omp_random_shapes(shape):
    """The FP64 decode, MP with Gram-updated correlations (R = 16) and OMP on
    the same random shapes."""
    from test_omp_gpu import compare_omp, decode_omp
    N, M, K, seed = shape
    prob = W.make_plain(N, M, K, seed=seed % 1000, eps=1e-5, T=4000)
    y64 = prob.y[0].astype(np.float64)
    with GpuPlan(prob.psi, prec_mask=1 << B().MP_PREC_FP64) as pl:
        out64 = pl.decode64(y64, 1e-9, 4000)
        compare_to_oracle(prob.psi, y64, 1e-9, 4000, out64, x_tol=1e-9, fp64=True)
        omp = decode_omp(pl, prob.y[0], prob.eps, prob.T)
        compare_omp(prob.psi, prob.y[0], prob.eps, prob.T, omp)
        pl.set(B().MP_OPT_PLAIN_GRAM, 16)
        gram = pl.decode(prob.y[0], prob.eps, prob.T)
        compare_to_oracle(prob.psi, prob.y[0], prob.eps, prob.T, gram, gram_period=16, strict=False)
