"""The allocation-free entry point (mp_recover_noalloc), for callers that
cannot allocate GPU memory: it must decode exactly like mp_recover, the
plan-based entry point, on two calls in a row (the second call reuses the
library's static scratch and must not see the first call's state).

Kept in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import GpuPlan, compare_to_oracle, cur_stream
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(256, 1024, 16, 1e-6), (100, 3001, 6, 1e-5), (4096, 16384, 64, 1e-5)],
                         ids=lambda s: f"N{s[0]}_M{s[1]}")
def test_noalloc_matches_plan_entry_point(shape):
    import torch
    from paper_0809_1833_gb300 import binding as B
    N, M, K, eps = shape
    T = 10000
    psi = W.gaussian_dictionary(N, M, seed=4)
    ld = (N + 3) // 4 * 4
    padded = np.zeros((M, ld), dtype=np.float32)
    padded[:, :N] = psi
    psi_d = torch.from_numpy(padded).cuda()
    signals = [W.make_plain(N, M, K, seed=s, eps=eps, T=T, psi=psi) for s in (11, 12)]
    with GpuPlan(psi) as pl:
        for prob in signals:            # two calls in a row
            ref = pl.decode(prob.y[0], eps, T)
            y = torch.from_numpy(prob.y[0]).cuda()
            x = torch.full((M,), float("nan"), dtype=torch.float32, device="cuda")
            res = B.mp_result()
            st = B.mp_stop(eps, T, 0)
            s = B.mp_recover_noalloc(psi_d.data_ptr(), N, M, ld, y.data_ptr(), x.data_ptr(), st, res, cur_stream())
            assert s == 0, B.last_error()
            xg = x.cpu().numpy()
            assert res.iters == ref["result"].iters
            assert res.stop_reason == ref["result"].stop_reason
            assert abs(res.rel_residual - ref["result"].rel_residual) <= 1e-6
            err = np.linalg.norm(xg.astype(np.float64) - ref["x"]) / np.linalg.norm(ref["x"])
            assert err <= 1e-4, err
    if N <= 256:
        out = dict(result=res, x=xg, atoms=ref["atoms"], r=ref["r"])
        compare_to_oracle(psi, signals[-1].y[0], eps, T, out, check_follow=False)


def test_noalloc_rejects_bad_arguments():
    import torch
    from paper_0809_1833_gb300 import binding as B
    psi = torch.zeros((8, 6), dtype=torch.float32, device="cuda")
    y = torch.zeros(6, dtype=torch.float32, device="cuda")
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    res = B.mp_result()
    st = B.mp_stop(1e-5, 10, 0)
    # ld not a multiple of 4
    assert B.mp_recover_noalloc(psi.data_ptr(), 6, 8, 6, y.data_ptr(), x.data_ptr(), st, res, None) == B.MP_ERR_INVALID
    assert "ld" in B.last_error()
    # N beyond what the on-chip residual can hold
    big = 1 << 20
    assert B.mp_recover_noalloc(psi.data_ptr(), big, 1, big, y.data_ptr(), x.data_ptr(), st, res,
                                None) == B.MP_ERR_UNSUPPORTED
