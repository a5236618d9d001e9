"""Parity of the FP32 OMP decode (mp_recover_omp) with the FP64 OMP oracle.

OMP keeps MP's selection and fits x~ by least squares on the selected atoms
(oracle/omp_oracle.py).  The GPU orthonormalises each new atom against the
selected ones in FP32 (classical Gram-Schmidt applied twice) and solves
R x = Q^T y after the loop.  Comparison rule as for MP: the atom sequence
equals the oracle's up to the first step whose oracle top-two gap is within
the FP32 error bound (plus the basis' loss of orthogonality, k 2^-24 per
step) and, literally, up to the first step whose oracle gap is <= 1e-5;
x~ within 1e-4 relative L2; and every selected atom is an OMP choice when
the oracle replays the GPU's sequence.
"""
import numpy as np
import pytest

import omp_pins as P
from gpu_helpers import GpuPlan, cur_stream, first_near_tie, log_parity, summation_depth, GAP_TIE, U32
from oracle import omp_oracle as orc
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def B():
    from paper_0809_1833_gb300 import binding
    return binding


def decode_omp(pl, y, eps, T, raise_on_error=True):
    import torch
    b = B()
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).cuda()
    x = torch.full((pl.M,), float("nan"), dtype=torch.float32, device="cuda")
    cap = max(1, min(int(T), pl.N + 1))
    atoms = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    coefs = torch.zeros(cap, dtype=torch.float32, device="cuda")
    en = torch.zeros(cap, dtype=torch.float64, device="cuda")
    r = torch.full((pl.N,), float("nan"), dtype=torch.float32, device="cuda")
    tr = b.make_trace(atoms.data_ptr(), coefs.data_ptr(), en.data_ptr(), cap, r.data_ptr())
    s, res = b.mp_recover_omp(pl.plan, yd.data_ptr(), x.data_ptr(), eps, T, tr, True, cur_stream(),
                              raise_on_error=raise_on_error)
    torch.cuda.synchronize()
    n = min(res.iters, cap)
    return dict(status=s, result=res, x=x.cpu().numpy(), atoms=atoms.cpu().numpy()[:n],
                coefs=coefs.cpu().numpy()[:n], energies=en.cpu().numpy()[:n], r=r.cpu().numpy())


def compare_omp(psi, y, eps, T, gpu, x_tol=1e-4, ora=None, literal=True):
    if ora is None:
        ora = orc.omp(psi, y, eps, T)
    res = gpu["result"]
    ga = np.asarray(gpu["atoms"], dtype=np.int64)
    oa = ora["atoms"]
    N = np.asarray(psi).shape[1]
    f = orc.follow(psi, y, ga) if len(ga) else None
    Delta = float(np.linalg.norm(gpu["r"].astype(np.float64) - f["r"])) if f is not None else 0.0
    k = np.arange(max(len(oa), len(ga)) + 1)
    gamma = (summation_depth(N) + 2 * k + 4) * U32
    tie = None
    if len(oa):
        rk = np.sqrt(np.concatenate([[ora["e0"]], ora["energies"][:-1]]))
        tol = np.maximum(GAP_TIE, (2 * Delta + 2 * gamma[:len(oa)] * rk) / np.maximum(np.abs(ora["coefs"]), 1e-300))
        ties = np.nonzero(ora["gaps"] <= tol)[0]
        tie = int(ties[0]) if ties.size else None
    lit = first_near_tie(ora["gaps"]) if len(oa) else None
    div = next((j for j in range(min(len(ga), len(oa))) if ga[j] != oa[j]), None)
    rec = dict(method="omp", N=N, M=int(np.asarray(psi).shape[0]), iters=res.iters, oracle_iters=ora["iters"],
               first_divergence=div, literal_cutoff=lit, fp32_bound_cutoff=tie, drift=Delta)
    try:
        lim = len(oa) if tie is None else tie
        n = min(lim, len(ga))
        assert np.array_equal(ga[:n], oa[:n]), (ga[:n], oa[:n], tie)
        nl = min(len(oa) if lit is None else lit, len(ga))
        rec["literal_rule_holds"] = bool(np.array_equal(ga[:nl], oa[:nl]))
        if literal:
            assert rec["literal_rule_holds"], f"OMP sequence diverges at {div} before the first 1e-5 gap {lit}"
        if tie is None:
            assert res.iters == ora["iters"] and res.stop_reason == ora["stop_reason"], (res.iters, ora["iters"])
        nx = np.linalg.norm(ora["x"])
        xerr = np.linalg.norm(gpu["x"].astype(np.float64) - ora["x"]) / (nx if nx > 0 else 1.0)
        rec["x_rel_err"] = xerr
        assert xerr <= x_tol, xerr
        if f is not None:
            tolf = np.maximum(GAP_TIE, (2 * Delta + 2 * gamma[:len(ga)] * f["rnorm"]) / np.maximum(f["cmax"], 1e-300))
            rec["min_ratio"] = float(f["ratio"].min())
            assert np.all(f["ratio"] >= 1 - tolf), f["ratio"].min()
            # the GPU's x~ is the least-squares fit on its own selection
            assert np.linalg.norm(gpu["x"] - f["x"]) <= x_tol * max(np.linalg.norm(f["x"]), 1e-30)
    finally:
        log_parity(rec)
    return dict(x_rel_err=rec.get("x_rel_err"), drift=Delta, first_near_tie=tie, literal_cutoff=lit,
                first_divergence=div)


@pytest.mark.parametrize("mode", [2, 3])
def test_omp_worked_example(mode):
    g = P.load_worked_example()
    ex = g["expected"]
    with GpuPlan(np.array(g["psi_atoms"], dtype=np.float32), mode=mode) as pl:
        out = decode_omp(pl, np.array(g["y"], dtype=np.float32), g["eps"], g["T"])
    assert out["result"].iters == ex["iters"] and out["result"].stop_reason == ex["stop_reason"]
    assert list(out["atoms"]) == ex["atoms"]
    assert np.allclose(out["x"], ex["x"], rtol=0, atol=1e-6)
    assert np.linalg.norm(out["r"]) <= 1e-6


SHAPES = [
    # (N, M, K, eps, T, seed)
    (256, 1024, 16, 1e-6, 20000, 0),
    (100, 333, 6, 1e-5, 5000, 1),
    (1000, 3001, 40, 1e-5, 5000, 3),
    (64, 5, 1, 1e-6, 100, 4),
]


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"N{s[0]}_M{s[1]}_K{s[2]}")
def test_omp_parity_with_oracle(shape, mode):
    N, M, K, eps, T, seed = shape
    prob = W.make_plain(N, M, K, seed=seed, eps=eps, T=T)
    with GpuPlan(prob.psi, mode=mode) as pl:
        out = decode_omp(pl, prob.y[0], eps, T)
    assert out["result"].status == 0
    compare_omp(prob.psi, prob.y[0], eps, T, out)
    # OMP stops after about K steps on a recoverable signal (MP needs many more)
    assert out["result"].iters <= K + 2


@pytest.mark.parametrize("shape", [(200, 900, 12), (1000, 3001, 40)], ids=["N200", "N1000"])
def test_omp_modes_agree_bitwise(shape):
    N, M, K = shape
    prob = W.make_plain(N, M, K, seed=8, eps=1e-6, T=500)
    outs = []
    for mode in (2, 3):
        with GpuPlan(prob.psi, mode=mode) as pl:
            outs.append(decode_omp(pl, prob.y[0], prob.eps, prob.T))
    for k in ("atoms", "x", "energies", "r"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_omp_rank_stop_and_edge_cases():
    g = np.random.default_rng(7)
    P_ = g.standard_normal((40, 16))
    P_ /= np.linalg.norm(P_, axis=1, keepdims=True)
    y = g.standard_normal(16).astype(np.float32)
    with GpuPlan(P_.astype(np.float32)) as pl:
        full = decode_omp(pl, y, 0.0, 100)
        assert full["result"].iters == 16 and full["result"].stop_reason in (B().MP_STOP_RANK, B().MP_STOP_CONVERGED)
        assert np.linalg.norm(full["r"]) <= 1e-4 * np.linalg.norm(y)
        z = decode_omp(pl, np.zeros(16, np.float32), 1e-5, 10)
        assert z["result"].iters == 0 and z["result"].stop_reason == B().MP_STOP_ZERO_Y and not np.any(z["x"])
        t0 = decode_omp(pl, y, 1e-5, 0)
        assert t0["result"].iters == 0 and not np.any(t0["x"])
        bad = y.copy()
        bad[2] = np.nan
        nf = decode_omp(pl, bad, 1e-5, 10, raise_on_error=False)
        assert nf["status"] == B().MP_ERR_NONFINITE
        again = decode_omp(pl, y, 1e-3, 5)
        compare_omp(P_.astype(np.float32), y, 1e-3, 5, again)
        pl.set(B().MP_OPT_PLAIN_MODE, 1)
        s = decode_omp(pl, y, 1e-3, 5, raise_on_error=False)["status"]
        assert s == B().MP_ERR_UNSUPPORTED


def test_omp_full_size_plain_workload():
    """The 256 MiB dictionary (N=4096, M=16384, K=256), grid streaming,
    against the full FP64 OMP oracle (256 growing least-squares fits): the
    literal sequence rule, the iteration count, x~ within 1e-4 relative,
    every step an OMP choice in the FP64 replay; OMP recovers the support."""
    prob = W.make_workload("plain_fp32_N4096_M16384_K256", seed=0)
    with GpuPlan(prob.psi) as pl:
        out = decode_omp(pl, prob.y[0], prob.eps, prob.T)
        assert pl.query(B().MP_Q_PLAIN_MODE) == 3
    res = out["result"]
    assert res.stop_reason == B().MP_STOP_CONVERGED and res.iters <= 256 + 4
    assert orc_support(out["x"], prob.supports[0]) == 1.0
    d = compare_omp(prob.psi, prob.y[0], prob.eps, prob.T, out)
    assert d["x_rel_err"] <= 1e-4


def orc_support(x, supp):
    from oracle import mp_oracle
    return mp_oracle.support_score(x, supp)
