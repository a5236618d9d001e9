"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare it with the FP64 oracle by the comparison rule for MP results.

Comparison rule (several MP paths are correct at a near tie, so only what is
unique is compared exactly):
  (i)   literal: the selected-atom sequence equals the oracle's on the
        prefix up to the first step whose oracle top-two gap is <= 1e-5
        (relative); the whole sequence when there is no such step.  This is
        asserted by default.  A test that drives a decode to the rounding
        floor of its arithmetic (eps far below what FP32 or FP64 resolves,
        more steps than the signal needs) or updates the correlations by
        the Gram recurrence passes ``strict=False`` and names why; it then
        asserts the sequence up to the first step whose gap is within the
        worst-case error bound
            tol_k = max(1e-5, (2 Delta + 2 d u ||r_k||) / |c_k|)
        (u the unit roundoff, d the summation depth of one correlation,
        |c_k| = max_m |c_m| before step k, Delta = ||r_path - r_replay|| the
        drift of the path's own final residual from an FP64 replay of its
        atom sequence).  Delta must itself stay within 16 times the
        random-walk rounding estimate u sqrt(d + 1) sqrt(sum_j ||r_j||^2),
        so a path that drifts more is caught rather than given a wider
        window.
  (ii)  x~ is within ``x_tol`` relative L2 of the oracle's x~;
  (iii) replaying the path's sequence in FP64, every selected atom is an MP
        choice up to the same bound: ratio_k >= 1 - tol_k.

Every comparison reports the first divergence, the literal cut-off (first
gap <= 1e-5) and the FP32-bound cut-off (first gap <= tol_k).  With the
environment variable MP_PARITY_LOG set to a file path, each appends them as
one JSON line.
"""
import json
import os

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


def first_near_tie(gaps, floor=None):
    idx = np.nonzero(np.asarray(gaps) <= (GAP_TIE if floor is None else floor))[0]
    return int(idx[0]) if idx.size else None


def log_parity(rec):
    """Append one comparison's diagnostics to $MP_PARITY_LOG (if set)."""
    path = os.environ.get("MP_PARITY_LOG")
    if not path:
        return
    rec = dict(rec)
    rec.setdefault("test", os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0])
    with open(path, "a") as f:
        f.write(json.dumps(rec, default=float) + "\n")


def compare_to_oracle(psi, y, eps, T, gpu, ora=None, x_tol=1e-4, check_follow=True, fp64=False, gram_period=0,
                      strict=True, label=None, gram_rescored=False):
    """Apply rules (i)-(iii); returns a dict of diagnostics, asserts on failure.
    ``gpu`` holds the path's own result, atoms, x~ and final residual ``r``.
    ``check_follow=False`` skips the FP64 replay when the whole sequence and
    the iteration count already match the oracle literally.  ``fp64``: the
    path computed in FP64 (u = 2^-53, d from summation_depth64).
    ``gram_period`` R > 0: the correlations were updated through the Gram
    matrix for up to R - 1 steps after each direct computation; each update
    adds at most |c_prev| |G - Psi^T Psi| + 2^-24 |c_m| <= (N + 2) 2^-24 ||r||
    of error (G entries are N-term FP32 FMA chains of unit atoms), so the
    depth of the correlations that rank the candidates grows by 2 R (N + 2)
    (a factor 2 for ||r|| at the refresh vs now).  ``gram_rescored``: the
    path rescored its candidates in FP32 and updated r with that exact
    coefficient (the batched Gram mode), so the residual's drift bound keeps
    the plain depth; otherwise (the plain Gram decode commits the
    recurrence's coefficient) the drift bound takes the widened depth too.
    ``strict=False``: rule (i) up to the FP32-bound cut-off instead of the
    literal one (see the module docstring for when a test may ask)."""
    from oracle import mp_oracle as orc
    if ora is None:
        ora = orc.mp(psi, y, eps, T)
    res = gpu["result"]
    ga = np.asarray(gpu["atoms"], dtype=np.int64)
    oa = ora["atoms"]
    N = np.asarray(psi).shape[1]
    div = next((k for k in range(min(len(ga), len(oa))) if ga[k] != oa[k]), None)
    literal_match = div is None and len(ga) == len(oa)
    out = dict(first_divergence=div, iters=res.iters, oracle_iters=ora["iters"], N=N, M=int(np.asarray(psi).shape[0]),
               strict=bool(strict))
    if label is not None:
        out["label"] = label
    u = U64 if fp64 else U32
    d_plain = summation_depth64(N) if fp64 else summation_depth(N)
    d = d_plain + (2 * gram_period * (N + 2) if gram_period > 0 else 0)  # the correlations that rank
    d_r = d_plain if gram_rescored else d                                # the residual's arithmetic
    gamma = d * u
    floor = GAP_TIE64 if fp64 else GAP_TIE
    r_all = np.sqrt(np.concatenate([[ora["e0"]], ora["energies"]]))   # oracle ||r|| before each step and at the end
    Delta = 0.0
    f = None
    if (check_follow or not literal_match or not strict) and len(ga):
        f = orc.follow(psi, y, ga)
        Delta = float(np.linalg.norm(np.asarray(gpu["r"]).astype(np.float64) - f["r"]))
        out["drift"] = Delta
    lit = first_near_tie(ora["gaps"], GAP_TIE) if len(oa) else None
    tie = None
    if len(oa):
        tol = np.maximum(floor, (2 * Delta + 2 * gamma * r_all[:-1]) / np.maximum(np.abs(ora["coefs"]), 1e-300))
        ties = np.nonzero(ora["gaps"] <= tol)[0]
        tie = int(ties[0]) if ties.size else None
    out["literal_cutoff"] = lit          # first oracle gap <= 1e-5 (None: none)
    out["fp32_bound_cutoff"] = tie       # first oracle gap <= tol_k
    out["first_near_tie"] = lit if strict else tie
    nl = min(len(oa) if lit is None else lit, len(ga))
    out["literal_rule_holds"] = bool(np.array_equal(ga[:nl], oa[:nl]))
    try:
        if strict:
            assert out["literal_rule_holds"], (
                f"atom sequence diverges at {div} before the first 1e-5 gap {lit} "
                f"(FP32-bound cut-off {tie}, gap there {ora['gaps'][div]:.3e})")
        else:
            n = min(len(oa) if tie is None else tie, len(ga))
            assert np.array_equal(ga[:n], oa[:n]), f"atom sequence diverges at {div} before the FP32-bound cut-off {tie}"
        if f is not None:
            n_t = min(len(ga), len(r_all))
            D_T = u * np.sqrt(d_r + 1) * np.sqrt(np.sum(r_all[:n_t] ** 2))
            out["drift_over_estimate"] = Delta / D_T if D_T > 0 else 0.0
            assert Delta <= 16 * D_T + 1e-300, f"drift {Delta:.3e} exceeds 16x the rounding estimate {D_T:.3e}"
        cut = lit if strict else tie
        if div is None and cut is None and res.iters != ora["iters"]:
            # only legitimate when the stop test sits at the rounding level:
            # the path's energy differs from the FP64 one by ~2 ||r|| Delta
            k = min(res.iters, ora["iters"])
            e_k = ora["energies"][k - 1] if k else ora["e0"]
            thr2 = eps * eps * ora["e0"]
            slack = 4 * np.sqrt(e_k) * Delta + 4 * gamma * e_k + 1e-9 * thr2
            assert abs(e_k - thr2) <= slack, (res.iters, ora["iters"], e_k, thr2, slack)
        nx = np.linalg.norm(ora["x"])
        xerr = np.linalg.norm(np.asarray(gpu["x"]).astype(np.float64) - ora["x"]) / (nx if nx > 0 else 1.0)
        out["x_rel_err"] = xerr
        assert xerr <= x_tol, f"x relative L2 error {xerr:.3e} > {x_tol}"
        if f is not None:
            tolf = np.maximum(floor, (2 * Delta + 2 * gamma * f["rnorm"]) / np.maximum(f["cmax"], 1e-300))
            out["min_ratio"] = float(f["ratio"].min())
            bad = np.nonzero(f["ratio"] < 1 - tolf)[0]
            assert bad.size == 0, f"follow ratio below bound at steps {bad[:5]}: {f['ratio'][bad[:5]]}"
    finally:
        log_parity(out)
    return out


def batched_decode(pl, prec, Y, stops, cap=4096):
    """mp_recover_batched over the rows of Y (host array): returns dict with
    status, results, X, atoms, coefs, energies (B rows of ``cap`` steps) and
    R, each signal's final FP32 residual from the batched path itself."""
    torch = torch_mod()
    from paper_0809_1833_gb300 import binding as B
    Bn, N = Y.shape
    Yd = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).cuda()
    X = torch.full((Bn, pl.M), float("nan"), dtype=torch.float32, device="cuda")
    atoms = torch.full((Bn, cap), -1, dtype=torch.int32, device="cuda")
    coefs = torch.zeros((Bn, cap), dtype=torch.float32, device="cuda")
    en = torch.zeros((Bn, cap), dtype=torch.float64, device="cuda")
    R = torch.full((Bn, N), float("nan"), dtype=torch.float32, device="cuda")
    tr = B.make_trace(atoms.data_ptr(), coefs.data_ptr(), en.data_ptr(), cap, R.data_ptr())
    s, res = B.mp_recover_batched(pl.plan, prec, Yd.data_ptr(), X.data_ptr(), Bn, stops, tr, cur_stream(),
                                  raise_on_error=False)
    torch.cuda.synchronize()
    return dict(status=s, results=res, X=X.cpu().numpy(), atoms=atoms.cpu().numpy(), coefs=coefs.cpu().numpy(),
                energies=en.cpu().numpy(), R=R.cpu().numpy())


def batched_signal(out, b):
    """Signal b of a batched_decode as the dict compare_to_oracle takes."""
    r = out["results"][b]
    n = min(r.iters, out["atoms"].shape[1])
    return dict(result=r, x=out["X"][b], atoms=out["atoms"][b, :n], r=out["R"][b])
