"""Sec. 3's phase-diagram experiment (E(sigma, rho), Eq. 14) through the
batched decode, signal by signal against the FP64 oracle on a few cells of
the diagram: one cell deep in the recovery region, one at its edge, one with
more nonzeros than measurements (K > N, no recovery possible).

Per signal: the selected atoms equal the oracle's up to the oracle's first
near tie (relative top-two gap <= 1e-4; beyond it either atom is an MP step
and FP32 drift may decide), and the experiment's output agrees -- a signal
the oracle recovers (E <= 1e-6 %) is recovered by the GPU to the FP32 rule
(x~ within 1e-4 relative L2, i.e. E <= 1e-6 %), and a signal the oracle
fails on (E >= 1 %) fails on the GPU too.
"""
import numpy as np
import pytest

from gpu_helpers import cur_stream, GpuPlan
from oracle import mp_oracle as orc
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TIE = 1e-4


def B():
    from paper_0809_1833_gb300 import binding
    return binding


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("rho,sigmas", [(0.3, [0.01, 0.05, 0.4]), (0.7, [0.1, 0.25])],
                         ids=["rho0.3", "rho0.7"])
def test_phase_diagram_cells_match_oracle(rho, sigmas, prec):
    import torch
    trials = 3
    prob = W.phase_diagram_batch(rho, sigmas, trials, seed=4)
    p = B().MP_PREC_BF16 if prec == "bf16" else B().MP_PREC_FP8E4M3
    cap = prob.T
    with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
        Y = torch.from_numpy(prob.y).cuda()
        X = torch.full((prob.B, prob.M), float("nan"), dtype=torch.float32, device="cuda")
        atoms = torch.full((prob.B, cap), -1, dtype=torch.int32, device="cuda")
        tr = B().make_trace(atoms.data_ptr(), 0, 0, cap)
        s, res = B().mp_recover_batched(pl.plan, p, Y.data_ptr(), X.data_ptr(), prob.B, (prob.eps, prob.T), tr,
                                        cur_stream())
        torch.cuda.synchronize()
        X = X.cpu().numpy()
        atoms = atoms.cpu().numpy()
    assert s == 0
    kinds = set()
    for b in range(prob.B):
        ora = orc.mp(prob.psi, prob.y[b], prob.eps, prob.T)
        Eo = orc.reconstruction_error(ora["x"], prob.x_true[b])
        Eg = orc.reconstruction_error(X[b], prob.x_true[b])
        ties = np.nonzero(ora["gaps"] <= TIE)[0]
        n = min(int(ties[0]) if ties.size else len(ora["atoms"]), res[b].iters)
        assert np.array_equal(atoms[b, :n], ora["atoms"][:n]), (b, n)
        if Eo <= 1e-6:
            kinds.add("recovered")
            assert Eg <= 1e-6, (b, Eg, Eo)
        elif Eo >= 1.0:
            kinds.add("failed")
            assert Eg >= 1.0, (b, Eg, Eo)
    if rho == 0.3:
        assert kinds == {"recovered", "failed"}   # the cells straddle the transition
