"""The allocation-free entry point (mp_recover_noalloc), for callers that
cannot allocate GPU memory: code inside a memory budget fixed by its host
application, a plugin that only receives buffers, or a loop that may not
call the allocator.  It must decode like mp_recover, the plan-based entry
point, on two calls in a row (the second call reuses the library's static
scratch and must not see the first call's state): bit for bit when the
dictionary is stored at the plan's stride, and within the comparison rule
of the other parity tests (its own atoms and residual against the FP64
oracle) at another stride.

Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from gpu_helpers import GpuPlan, compare_to_oracle, cur_stream
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(B, psi_d, N, M, ld, y_np, eps, T, cap):
    import torch
    y = torch.from_numpy(np.ascontiguousarray(y_np, dtype=np.float32)).cuda()
    x = torch.full((M,), float("nan"), dtype=torch.float32, device="cuda")
    atoms = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    coefs = torch.zeros(cap, dtype=torch.float32, device="cuda")
    en = torch.zeros(cap, dtype=torch.float64, device="cuda")
    r = torch.full((N,), float("nan"), dtype=torch.float32, device="cuda")
    tr = B.make_trace(atoms.data_ptr(), coefs.data_ptr(), en.data_ptr(), cap, r.data_ptr())
    res = B.mp_result()
    s = B.mp_recover_noalloc(psi_d.data_ptr(), N, M, ld, y.data_ptr(), x.data_ptr(), B.mp_stop(eps, T, 0), res,
                             cur_stream(), trace=tr)
    torch.cuda.synchronize()
    n = min(res.iters, cap)
    return s, dict(result=res, x=x.cpu().numpy(), atoms=atoms.cpu().numpy()[:n], coefs=coefs.cpu().numpy()[:n],
                   energies=en.cpu().numpy()[:n], r=r.cpu().numpy())


def _padded(psi, ld):
    import torch
    M, N = psi.shape
    a = np.zeros((M, ld), dtype=np.float32)
    a[:, :N] = psi
    return torch.from_numpy(a).cuda()


@pytest.mark.parametrize("shape", [(256, 1024, 16, 1e-6), (100, 3001, 6, 1e-5), (4096, 16384, 64, 1e-5)],
                         ids=lambda s: f"N{s[0]}_M{s[1]}")
def test_noalloc_matches_plan_entry_point(shape):
    from paper_0809_1833_gb300 import binding as B
    N, M, K, eps = shape
    T = 10000
    psi = W.gaussian_dictionary(N, M, seed=4)
    signals = [W.make_plain(N, M, K, seed=s, eps=eps, T=T, psi=psi) for s in (11, 12)]
    with GpuPlan(psi) as pl:
        ld_plan = pl.query(B.MP_Q_LD_FP32)
        psi_plan_ld = _padded(psi, ld_plan)
        for prob in signals:            # two calls in a row
            ref = pl.decode(prob.y[0], eps, T)
            s, got = _noalloc(B, psi_plan_ld, N, M, ld_plan, prob.y[0], eps, T, T)
            assert s == 0, B.last_error()
            # the plan's stride: the same kernel on the same bytes, bit for bit
            assert got["result"].iters == ref["result"].iters
            assert got["result"].stop_reason == ref["result"].stop_reason
            assert got["result"].rel_residual == ref["result"].rel_residual
            for k in ("x", "atoms", "coefs", "energies", "r"):
                assert np.array_equal(got[k], ref[k]), k
    # another stride (N rounded up to 4 only): other FP32 summation order;
    # its own atoms and residual against the FP64 oracle, two calls in a row
    ld4 = (N + 3) // 4 * 4
    if ld4 != ld_plan:
        psi_ld4 = _padded(psi, ld4)
        for prob in signals:
            s, got = _noalloc(B, psi_ld4, N, M, ld4, prob.y[0], eps, T, T)
            assert s == 0, B.last_error()
            compare_to_oracle(psi, prob.y[0], eps, T, got)


def test_noalloc_rejects_bad_arguments():
    import torch
    from paper_0809_1833_gb300 import binding as B
    psi = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    y = torch.zeros(6, dtype=torch.float32, device="cuda")
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    res = B.mp_result()
    st = B.mp_stop(1e-5, 10, 0)
    # ld not a multiple of 4
    assert B.mp_recover_noalloc(psi.data_ptr(), 6, 8, 6, y.data_ptr(), x.data_ptr(), st, res, None) == B.MP_ERR_INVALID
    assert "ld" in B.last_error()
    # a non-finite or negative eps, a negative T
    for bad in (B.mp_stop(float("nan"), 10, 0), B.mp_stop(float("inf"), 10, 0), B.mp_stop(-1.0, 10, 0),
                B.mp_stop(1e-5, -1, 0)):
        assert B.mp_recover_noalloc(psi.data_ptr(), 6, 8, 8, y.data_ptr(), x.data_ptr(), bad, res,
                                    None) == B.MP_ERR_INVALID
        assert "stop" in B.last_error()
    # N beyond what the on-chip residual can hold
    big = 1 << 20
    assert B.mp_recover_noalloc(psi.data_ptr(), big, 1, big, y.data_ptr(), x.data_ptr(), st, res,
                                None) == B.MP_ERR_UNSUPPORTED
