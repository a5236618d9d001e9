"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare it with the FP64 oracle by the comparison rule for MP results.

Comparison rule (several MP paths are correct at a near tie, so only what is
unique is compared exactly).  With tol_k the FP32 error bound of step k,

    tol_k = max(1e-5, (2 Delta + 2 gamma_d ||r_k||) / max_m |c_m,k|),

where Delta = ||r_gpu - r_replay|| is the drift between the GPU's final FP32
residual and an FP64 replay of the GPU's own atom sequence, and
gamma_d ||r_k|| (gamma_d = d 2^-24, d the depth of the kernel's summation
tree) bounds one FP32 dot product's rounding for a unit atom:
  (i)   the selected-atom sequence equals the oracle's on the prefix up to
        the first step whose oracle top-two gap is <= tol_k (the whole
        sequence when there is no such step).  The floor 1e-5 is the
        literal near-tie threshold; above it the FP32 rounding itself can
        decide the order of two correlations, and either atom is an MP step;
  (ii)  x~ is within ``x_tol`` relative L2 of the oracle's x~;
  (iii) replaying the GPU's sequence in FP64, every selected atom is an MP
        choice up to the FP32 error: ratio_k >= 1 - tol_k.
"""
import numpy as np

GAP_TIE = 1e-5
U32 = 2.0 ** -24
U64 = 2.0 ** -53
# FP64 near-tie floor: far below any FP32 effect, above FP64 rounding of a
# correlation of the sizes tested
GAP_TIE64 = 1e-13


def summation_depth(N):
    """Depth of the FP32 summation tree of one correlation: one FMA chain
    per lane over the 128-float segments, two combining adds, and a 5-level
    warp butterfly."""
    ld = (N + 31) // 32 * 32
    return (ld + 127) // 128 + 7


def summation_depth64(N):
    """Depth of the FP64 summation tree of one correlation (two FMA chains
    per lane over 64-double segments, one combining add, the butterfly),
    plus N for the oracle's own FP64 sum, whose order is not specified."""
    ld = (N + 31) // 32 * 32
    return (ld + 63) // 64 + 6 + N


def torch_mod():
    import torch
    return torch


def cur_stream():
    torch = torch_mod()
    return torch.cuda.current_stream().cuda_stream


class GpuPlan:
    """A plan over a numpy atom-major dictionary, created through the C ABI."""

    def __init__(self, psi, prec_mask=0, mode=0, layout_row_major=False, normalize=False, master64=False):
        from paper_0809_1833_gb300 import binding as B
        torch = torch_mod()
        self.B = B
        M, N = psi.shape
        self.N, self.M = N, M
        lay = B.MP_LAYOUT_ROW_MAJOR if layout_row_major else B.MP_LAYOUT_ATOM_MAJOR
        src = np.ascontiguousarray(psi.T if layout_row_major else psi,
                                   dtype=np.float64 if master64 else np.float32)
        d = torch.from_numpy(src).cuda()
        if master64:
            self.plan = B.mp_plan_create_f64(N, M, d.data_ptr(), lay, prec_mask | (1 << B.MP_PREC_FP64),
                                             normalize, cur_stream())
        else:
            self.plan = B.mp_plan_create(N, M, d.data_ptr(), lay, prec_mask, normalize, cur_stream())
        del d
        if mode:
            B.mp_plan_set_option(self.plan, B.MP_OPT_PLAIN_MODE, mode)

    def set(self, opt, val):
        self.B.mp_plan_set_option(self.plan, opt, val)

    def query(self, what):
        return self.B.mp_plan_query(self.plan, what)

    def decode(self, y, eps, T, trace_cap=None, raise_on_error=True):
        """Decode one signal; returns dict(status, result, x, atoms, coefs, energies, r)."""
        torch = torch_mod()
        B = self.B
        yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).cuda()
        x = torch.full((self.M,), float("nan"), dtype=torch.float32, device="cuda")
        cap = min(int(T), 200000) if trace_cap is None else int(trace_cap)
        cap = max(cap, 1)
        atoms = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        coefs = torch.zeros(cap, dtype=torch.float32, device="cuda")
        en = torch.zeros(cap, dtype=torch.float64, device="cuda")
        r = torch.full((self.N,), float("nan"), dtype=torch.float32, device="cuda")
        tr = B.make_trace(atoms.data_ptr(), coefs.data_ptr(), en.data_ptr(), cap, r.data_ptr())
        s, res = B.mp_recover(self.plan, yd.data_ptr(), x.data_ptr(), eps, T, tr, True, cur_stream(),
                              raise_on_error=raise_on_error)
        torch.cuda.synchronize()
        n = min(res.iters, cap)
        return dict(status=s, result=res, x=x.cpu().numpy(), atoms=atoms.cpu().numpy()[:n],
                    coefs=coefs.cpu().numpy()[:n], energies=en.cpu().numpy()[:n], r=r.cpu().numpy())

    def decode64(self, y, eps, T, trace_cap=None, raise_on_error=True):
        """FP64 decode (mp_recover_f64) of y given in FP64; same dict as decode."""
        torch = torch_mod()
        B = self.B
        yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).cuda()
        x = torch.full((self.M,), float("nan"), dtype=torch.float64, device="cuda")
        cap = min(int(T), 200000) if trace_cap is None else int(trace_cap)
        cap = max(cap, 1)
        atoms = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        coefs = torch.zeros(cap, dtype=torch.float64, device="cuda")
        en = torch.zeros(cap, dtype=torch.float64, device="cuda")
        r = torch.full((self.N,), float("nan"), dtype=torch.float64, device="cuda")
        tr = B.make_trace_f64(atoms.data_ptr(), coefs.data_ptr(), en.data_ptr(), cap, r.data_ptr())
        s, res = B.mp_recover_f64(self.plan, yd.data_ptr(), x.data_ptr(), eps, T, tr, True, cur_stream(),
                                  raise_on_error=raise_on_error)
        torch.cuda.synchronize()
        n = min(res.iters, cap)
        return dict(status=s, result=res, x=x.cpu().numpy(), atoms=atoms.cpu().numpy()[:n],
                    coefs=coefs.cpu().numpy()[:n], energies=en.cpu().numpy()[:n], r=r.cpu().numpy())

    def close(self):
        if self.plan:
            self.B.mp_plan_destroy(self.plan)
            self.plan = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def first_near_tie(gaps):
    idx = np.nonzero(np.asarray(gaps) <= GAP_TIE)[0]
    return int(idx[0]) if idx.size else None


def compare_to_oracle(psi, y, eps, T, gpu, ora=None, x_tol=1e-4, check_follow=True, fp64=False, gram_period=0):
    """Apply rules (i)-(iii); returns a dict of diagnostics, asserts on failure.
    ``check_follow=False`` skips the FP64 replay when the whole sequence and
    the iteration count already match the oracle literally.  ``fp64``: the
    GPU path computed in FP64, so gamma_d = d 2^-53 (d from
    summation_depth64) and the near-tie floor is GAP_TIE64.  ``gram_period``
    R > 0: the correlations were updated through the Gram matrix for up to
    R - 1 steps after each direct computation; each update adds at most
    |c_prev| |G - Psi^T Psi| + 2^-24 |c_m| <= (N + 2) 2^-24 ||r|| of error
    (G entries are N-term FP32 FMA chains of unit atoms), so gamma_d grows
    by 2 R (N + 2) 2^-24 (a factor 2 for ||r|| at the refresh vs now)."""
    from oracle import mp_oracle as orc
    if ora is None:
        ora = orc.mp(psi, y, eps, T)
    res = gpu["result"]
    ga = np.asarray(gpu["atoms"], dtype=np.int64)
    oa = ora["atoms"]
    N = np.asarray(psi).shape[1]
    div = next((k for k in range(min(len(ga), len(oa))) if ga[k] != oa[k]), None)
    literal = div is None and len(ga) == len(oa)
    out = dict(first_divergence=div, iters=res.iters, oracle_iters=ora["iters"])
    Delta = 0.0
    f = None
    if (check_follow or not literal) and len(ga):
        f = orc.follow(psi, y, ga)
        Delta = float(np.linalg.norm(gpu["r"].astype(np.float64) - f["r"]))
        out["drift"] = Delta
    gamma = summation_depth64(N) * U64 if fp64 else summation_depth(N) * U32
    if gram_period > 0:
        gamma += 2 * gram_period * (N + 2) * U32
    floor = GAP_TIE64 if fp64 else GAP_TIE
    if len(oa):
        rk = np.sqrt(np.concatenate([[ora["e0"]], ora["energies"][:-1]]))
        tol = np.maximum(floor, (2 * Delta + 2 * gamma * rk) / np.maximum(np.abs(ora["coefs"]), 1e-300))
        ties = np.nonzero(ora["gaps"] <= tol)[0]
        tie = int(ties[0]) if ties.size else None
    else:
        tie = None
    out["first_near_tie"] = tie
    lim = len(oa) if tie is None else tie
    n = min(lim, len(ga))
    assert np.array_equal(ga[:n], oa[:n]), f"atom sequence diverges at {div} before first near-tie {tie}"
    if div is None and tie is None and res.iters != ora["iters"]:
        # only legitimate when the stop test sits at the rounding level:
        # the GPU's FP32 energy differs from the FP64 one by ~2 ||r|| Delta
        k = min(res.iters, ora["iters"])
        e_k = ora["energies"][k - 1] if k else ora["e0"]
        thr2 = eps * eps * ora["e0"]
        slack = 4 * np.sqrt(e_k) * Delta + 4 * gamma * e_k + 1e-9 * thr2
        assert abs(e_k - thr2) <= slack, (res.iters, ora["iters"], e_k, thr2, slack)
    nx = np.linalg.norm(ora["x"])
    xerr = np.linalg.norm(gpu["x"].astype(np.float64) - ora["x"]) / (nx if nx > 0 else 1.0)
    assert xerr <= x_tol, f"x relative L2 error {xerr:.3e} > {x_tol}"
    out["x_rel_err"] = xerr
    if f is not None:
        tolf = np.maximum(floor, (2 * Delta + 2 * gamma * f["rnorm"]) / np.maximum(f["cmax"], 1e-300))
        bad = np.nonzero(f["ratio"] < 1 - tolf)[0]
        assert bad.size == 0, f"follow ratio below bound at steps {bad[:5]}: {f['ratio'][bad[:5]]}"
        out["min_ratio"] = float(f["ratio"].min())
    return out
