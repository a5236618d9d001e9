"""Batched decode (mp_recover_batched) on the tensor cores.

* The tcgen05 GEMM is checked element by element (mp_debug_correlations)
  against an FP64 product of the same quantised operands.
* The batched MP result is compared with the FP32 persistent kernel: the
  rescore uses the same FP32 correlation order, so whenever the FP32 argmax
  is among the 8 low-precision candidates the batched path reproduces the
  plain path bit for bit; and every signal meets the oracle rule.
"""
import numpy as np
import pytest

from gpu_helpers import GpuPlan, batched_decode, compare_to_oracle, cur_stream
from oracle import mp_oracle as orc
from paper_0809_1833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def B():
    from paper_0809_1833_gb300 import binding
    return binding


def torch():
    import torch as t
    return t


def bf16_round(a):
    T = torch()
    return T.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(T.bfloat16).to(T.float32).numpy()


def e4m3_rows(a):
    """Per-row E4M3 quantisation as the library defines it: scale
    s = max|row| / 448 (FP32), codes = RNE_e4m3(row * (448 / max|row|))."""
    T = torch()
    a = np.ascontiguousarray(a, dtype=np.float32)
    amax = np.max(np.abs(a), axis=1).astype(np.float32)
    inv = np.where(amax > 0, np.float32(448.0) / np.where(amax > 0, amax, 1), np.float32(1)).astype(np.float32)
    q = T.from_numpy((a * inv[:, None]).astype(np.float32)).to(T.float8_e4m3fn).to(T.float32).numpy()
    s = np.where(amax > 0, amax / np.float32(448.0), np.float32(1)).astype(np.float32)
    return q.astype(np.float64), s.astype(np.float64)


# (signals per tile, atoms per tile)
TILES = [(128, 256), (128, 128), (256, 256), (256, 128), (256, 224), (128, 160)]


@pytest.mark.parametrize("tile", TILES, ids=lambda t: f"TM{t[0]}_TN{t[1]}")
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("shape", [(256, 1000, 200), (100, 300, 5), (2048, 1024, 130), (192, 777, 600)],
                         ids=lambda s: f"N{s[0]}_M{s[1]}_B{s[2]}")
def test_tensor_core_correlations(prec, shape, tile):
    """Every tile shape gives the exact quantised product: 128- and
    256-signal tiles (two MMAs per staged atom slice, one TMEM buffer at 256
    atoms) whose second row block is full, partial or absent, row tiles
    beyond the batch and a ragged last atom tile."""
    T = torch()
    N, M, Bn = shape
    psi = W.gaussian_dictionary(N, M, seed=3)
    rng = np.random.default_rng([N, M, Bn])
    R = rng.standard_normal((Bn, N)).astype(np.float32)
    p = B().MP_PREC_BF16 if prec == "bf16" else B().MP_PREC_FP8E4M3
    with GpuPlan(psi, prec_mask=1 << p) as pl:
        pl.set(B().MP_OPT_BATCH_TILE_M, tile[0])
        pl.set(B().MP_OPT_BATCH_TILE_N, tile[1])
        Rd = T.from_numpy(R).cuda()
        C = T.full((Bn, M), float("nan"), dtype=T.float32, device="cuda")
        B().mp_debug_correlations(pl.plan, p, Rd.data_ptr(), Bn, C.data_ptr(), cur_stream())
        assert (pl.query(B().MP_Q_BATCH_TILE_M), pl.query(B().MP_Q_BATCH_TILE_N)) == tile
        C = C.cpu().numpy().astype(np.float64)
    if prec == "bf16":
        A = bf16_round(R).astype(np.float64)
        P = bf16_round(psi).astype(np.float64)
        ref = A @ P.T
        mag = np.abs(A) @ np.abs(P).T
    else:
        qa, sa = e4m3_rows(R)
        qp, sp = e4m3_rows(psi)
        ref = (qa @ qp.T) * sa[:, None] * sp[None, :]
        mag = (np.abs(qa) @ np.abs(qp).T) * sa[:, None] * sp[None, :]
    # FP32 accumulation of exact products: |err| <= K 2^-24 sum|products| (+ scaling)
    tol = (N + 8) * 2.0 ** -24 * mag + 1e-30
    err = np.abs(C - ref)
    assert np.all(np.isfinite(C))
    assert np.all(err <= tol), f"max err/tol {np.max(err / tol):.3g}"


def n_sms():
    return torch().cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("tn", [256, 128])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_tensor_core_correlations_two_block_tiles(prec, tn):
    """256-signal tiles are taken while the batch has more 128-row tiles
    than the GPU has SMs: 600 rows x 8192 atoms is past that point, with a
    last row tile of one block (and, at 128 atoms per tile, CTAs that run
    two tiles through both accumulator buffers).  Exact quantised product."""
    T = torch()
    N, M, Bn = 256, 8192, 600
    assert -(-Bn // 128) * (M // tn) > n_sms()
    psi = W.gaussian_dictionary(N, M, seed=4)
    R = np.random.default_rng(11).standard_normal((Bn, N)).astype(np.float32)
    p = B().MP_PREC_BF16 if prec == "bf16" else B().MP_PREC_FP8E4M3
    with GpuPlan(psi, prec_mask=1 << p) as pl:
        pl.set(B().MP_OPT_BATCH_TILE_M, 256)
        pl.set(B().MP_OPT_BATCH_TILE_N, tn)
        Rd = T.from_numpy(R).cuda()
        C = T.full((Bn, M), float("nan"), dtype=T.float32, device="cuda")
        B().mp_debug_correlations(pl.plan, p, Rd.data_ptr(), Bn, C.data_ptr(), cur_stream())
        C = C.cpu().numpy().astype(np.float64)
    if prec == "bf16":
        A = bf16_round(R).astype(np.float64)
        P = bf16_round(psi).astype(np.float64)
        ref, mag = A @ P.T, np.abs(A) @ np.abs(P).T
    else:
        qa, sa = e4m3_rows(R)
        qp, sp = e4m3_rows(psi)
        ref = (qa @ qp.T) * sa[:, None] * sp[None, :]
        mag = (np.abs(qa) @ np.abs(qp).T) * sa[:, None] * sp[None, :]
    tol = (N + 8) * 2.0 ** -24 * mag + 1e-30
    assert np.all(np.isfinite(C))
    assert np.all(np.abs(C - ref) <= tol), f"max err/tol {np.max(np.abs(C - ref) / tol):.3g}"


def test_batched_decode_switching_tile_rows_equals_128_row_tiles():
    """A 700-signal decode over 8192 atoms starts on 256-signal tiles and
    moves to 128-signal tiles as signals finish; the GEMM's products do not
    depend on the tile, so every signal's atoms, x~ and iteration count
    equal those of the decode on 128-signal tiles bit for bit."""
    prob = W.make_batched(256, 8192, 700, 2, 16, seed=8, eps=1e-5, T=3000)
    assert -(-prob.B // 128) * (8192 // 256) > n_sms()
    p = B().MP_PREC_BF16
    out = {}
    for tm in (256, 128):
        with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
            pl.set(B().MP_OPT_BATCH_TILE_M, tm)
            pl.set(B().MP_OPT_BATCH_TILE_N, 256)
            s, res, X, atoms, _ = run_batched(pl, p, prob.y, (prob.eps, prob.T))
            assert s == 0
            out[tm] = (res, X, atoms)
            Rb = run_batched.R
            if tm == 256:
                for b in (0, 350, 699):
                    r = res[b]
                    assert r.status == 0 and r.stop_reason == B().MP_STOP_CONVERGED
                    o = dict(result=r, x=X[b], atoms=atoms[b, :r.iters], r=Rb[b])
                    compare_to_oracle(prob.psi, prob.y[b], prob.eps, prob.T, o, check_follow=False)
    (r2, X2, a2), (r1, X1, a1) = out[256], out[128]
    assert [r.iters for r in r2] == [r.iters for r in r1]
    assert np.array_equal(X2, X1) and np.array_equal(a2, a1)


# two-SM tiles (MP_OPT_BATCH_PAIR): 256 signals x TN atoms per cluster of two CTAs
PAIR_TN = [256, 224, 160, 128]


def correlations(psi, R, prec, opts):
    """mp_debug_correlations under the given plan options; returns
    (C float64, (tile_m, tile_n, pair) the engine used)."""
    T = torch()
    with GpuPlan(psi, prec_mask=1 << prec) as pl:
        for k, v in opts:
            pl.set(k, v)
        Rd = T.from_numpy(R).cuda()
        C = T.full((R.shape[0], psi.shape[0]), float("nan"), dtype=T.float32, device="cuda")
        B().mp_debug_correlations(pl.plan, prec, Rd.data_ptr(), R.shape[0], C.data_ptr(), cur_stream())
        used = (pl.query(B().MP_Q_BATCH_TILE_M), pl.query(B().MP_Q_BATCH_TILE_N), pl.query(B().MP_Q_BATCH_PAIR))
        return C.cpu().numpy().astype(np.float64), used


@pytest.mark.parametrize("tn", PAIR_TN)
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("shape", [(256, 8192, 600), (100, 300, 5), (192, 777, 200), (2048, 1024, 130)],
                         ids=lambda s: f"N{s[0]}_M{s[1]}_B{s[2]}")
def test_pair_tile_correlations(prec, shape, tn):
    """Two-SM tiles give the exact quantised product and the same FP32 bits
    as single-CTA 128-row tiles: 600 rows x 8192 atoms (more tiles than
    clusters, so clusters run several tiles through both accumulator
    buffers), a batch of 5 (the odd CTA of the pair has no active rows), a
    second row block of 72 rows (loaded as a whole block) and ragged last atom tiles."""
    N, M, Bn = shape
    psi = W.gaussian_dictionary(N, M, seed=5)
    R = np.random.default_rng([N, M, Bn, 1]).standard_normal((Bn, N)).astype(np.float32)
    p = B().MP_PREC_BF16 if prec == "bf16" else B().MP_PREC_FP8E4M3
    C, used = correlations(psi, R, p, [(B().MP_OPT_BATCH_PAIR, 2), (B().MP_OPT_BATCH_TILE_N, tn)])
    assert used == (256, tn, 1)
    C1, used1 = correlations(psi, R, p, [(B().MP_OPT_BATCH_PAIR, 1), (B().MP_OPT_BATCH_TILE_M, 128),
                                          (B().MP_OPT_BATCH_TILE_N, 128)])
    assert used1 == (128, 128, 0)
    if prec == "bf16":
        A = bf16_round(R).astype(np.float64)
        P = bf16_round(psi).astype(np.float64)
        ref, mag = A @ P.T, np.abs(A) @ np.abs(P).T
    else:
        qa, sa = e4m3_rows(R)
        qp, sp = e4m3_rows(psi)
        ref = (qa @ qp.T) * sa[:, None] * sp[None, :]
        mag = (np.abs(qa) @ np.abs(qp).T) * sa[:, None] * sp[None, :]
    tol = (N + 8) * 2.0 ** -24 * mag + 1e-30
    assert np.all(np.isfinite(C))
    assert np.all(np.abs(C - ref) <= tol), f"max err/tol {np.max(np.abs(C - ref) / tol):.3g}"
    assert np.array_equal(C, C1)


@pytest.mark.parametrize("tn", [256, 224])
def test_pair_tile_decode_equals_128_row_tiles(tn):
    """The 700-signal decode over 8192 atoms on two-SM tiles (more tiles than
    clusters while the batch is full, one row pair at the end): every
    signal's atoms, x~, residual and iteration count equal the decode on
    single-CTA 128-signal tiles bit for bit; three signals meet the oracle
    rule."""
    prob = W.make_batched(256, 8192, 700, 2, 16, seed=8, eps=1e-5, T=3000)
    p = B().MP_PREC_BF16
    out = {}
    for key, opts in (("pair", [(B().MP_OPT_BATCH_PAIR, 2), (B().MP_OPT_BATCH_TILE_N, tn)]),
                      ("single", [(B().MP_OPT_BATCH_PAIR, 1), (B().MP_OPT_BATCH_TILE_M, 128),
                                  (B().MP_OPT_BATCH_TILE_N, 256)])):
        with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
            for k, v in opts:
                pl.set(k, v)
            s, res, X, atoms, _ = run_batched(pl, p, prob.y, (prob.eps, prob.T))
            assert s == 0
            assert pl.query(B().MP_Q_BATCH_PAIR) == (1 if key == "pair" else 0)
            out[key] = (res, X, atoms, run_batched.R.copy())
    (r2, X2, a2, R2), (r1, X1, a1, R1) = out["pair"], out["single"]
    assert [r.iters for r in r2] == [r.iters for r in r1]
    assert np.array_equal(X2, X1) and np.array_equal(a2, a1) and np.array_equal(R2, R1)
    for b in (0, 350, 699):
        r = r2[b]
        assert r.status == 0 and r.stop_reason == B().MP_STOP_CONVERGED
        o = dict(result=r, x=X2[b], atoms=a2[b, :r.iters], r=R2[b])
        compare_to_oracle(prob.psi, prob.y[b], prob.eps, prob.T, o, check_follow=False)


def test_pair_option_checks():
    psi = W.gaussian_dictionary(64, 300, seed=3)
    prob = W.make_batched(64, 300, 4, 1, 3, seed=2, psi=psi, eps=1e-5, T=500)
    p = B().MP_PREC_BF16
    with GpuPlan(psi, prec_mask=1 << p) as pl:
        for bad in (-1, 3):
            with pytest.raises(B().MpError) as ei:
                pl.set(B().MP_OPT_BATCH_PAIR, bad)
            assert ei.value.status == B().MP_ERR_INVALID
        for bad in (96, 100, 288):
            with pytest.raises(B().MpError) as ei:
                pl.set(B().MP_OPT_BATCH_TILE_N, bad)
            assert ei.value.status == B().MP_ERR_INVALID
        # 224 atoms per tile on single-CTA tiles, then on two-SM tiles
        pl.set(B().MP_OPT_BATCH_PAIR, 1)
        pl.set(B().MP_OPT_BATCH_TILE_N, 224)
        s, res1, X1, _, _ = run_batched(pl, p, prob.y, (prob.eps, prob.T))
        assert s == 0 and pl.query(B().MP_Q_BATCH_PAIR) == 0 and pl.query(B().MP_Q_BATCH_TILE_N) == 224
        pl.set(B().MP_OPT_BATCH_PAIR, 2)
        s, res, X, atoms, _ = run_batched(pl, p, prob.y, (prob.eps, prob.T))
        assert s == 0 and pl.query(B().MP_Q_BATCH_PAIR) == 1 and pl.query(B().MP_Q_BATCH_TILE_N) == 224
        assert np.array_equal(X, X1)
        for b in range(prob.B):
            ora = orc.mp(psi, prob.y[b], prob.eps, prob.T)
            assert list(atoms[b, :res[b].iters]) == list(ora["atoms"])


def run_batched(pl, prec, Y, stops, cap=4096):
    out = batched_decode(pl, prec, Y, stops, cap)
    run_batched.energies = out["energies"]
    run_batched.R = out["R"]          # each signal's final residual from the batched path
    return out["status"], out["results"], out["X"], out["atoms"], out["coefs"]


@pytest.mark.parametrize("tile", [128, 256], ids=lambda t: f"TM{t}")
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_batched_matches_plain_and_oracle(prec, tile):
    prob = W.make_batched(256, 1024, 300, 2, 16, seed=5, eps=1e-5, T=3000)
    p = B().MP_PREC_BF16 if prec == "bf16" else B().MP_PREC_FP8E4M3
    with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
        pl.set(B().MP_OPT_BATCH_TILE_M, tile)
        s, res, X, atoms, _ = run_batched(pl, p, prob.y, (prob.eps, prob.T))
        assert s == 0
        n_same = 0
        for b in range(prob.B):
            r = res[b]
            assert r.status == 0 and r.stop_reason == B().MP_STOP_CONVERGED
            plain = pl.decode(prob.y[b], prob.eps, prob.T)
            if (r.iters == plain["result"].iters and np.array_equal(atoms[b, :r.iters], plain["atoms"])):
                # same atoms: the same FP32 update and the same FP64 energy order
                assert np.array_equal(X[b], plain["x"]), b
                assert np.array_equal(run_batched.R[b], plain["r"]), b
                assert np.array_equal(run_batched.energies[b, :r.iters], plain["energies"]), b
                n_same += 1
            out = dict(result=r, x=X[b], atoms=atoms[b, :r.iters], r=run_batched.R[b])
            if b % 10 == 0:   # full oracle rule on a sample of the signals
                ora = orc.mp(prob.psi, prob.y[b], prob.eps, prob.T)
                compare_to_oracle(prob.psi, prob.y[b], prob.eps, prob.T, out, ora=ora, check_follow=False)
                assert orc.support_score(X[b], prob.supports[b]) == 1.0
        # the 8-candidate rescore recovers the FP32 choice at (nearly) every step
        assert n_same >= prob.B - 3, n_same


def test_autotuner_picks_a_valid_shape_and_results_do_not_depend_on_it():
    prob = W.make_batched(256, 2048, 260, 2, 12, seed=6, eps=1e-5, T=2000)
    p = B().MP_PREC_BF16
    with GpuPlan(prob.psi, prec_mask=1 << p) as pl:
        tn, tm, pair = B().mp_plan_autotune_shape(pl.plan, p, prob.B)
        if pair:
            assert tm == 256 and tn in (192, 224, 256)
        else:
            assert tn in (128, 224, 256) and tm in (128, 256)
        assert B().mp_plan_autotune_shape(pl.plan, p, prob.B) == (tn, tm, pair)   # cached per size bucket
        assert B().mp_plan_autotune(pl.plan, p, prob.B) == (tn, tm)
        s, res, X, _, _ = run_batched(pl, p, prob.y, (prob.eps, prob.T))
        assert s == 0
        q = (B().MP_Q_BATCH_TILE_N, B().MP_Q_BATCH_TILE_M, B().MP_Q_BATCH_PAIR)
        assert tuple(pl.query(k) for k in q) == (tn, tm, pair)
        # another shape: single-CTA if the tuner took a pair, else a pair
        other = (256, 128, 0) if pair else (224, 256, 1)
        pl.set(B().MP_OPT_BATCH_PAIR, 2 if other[2] else 1)
        pl.set(B().MP_OPT_BATCH_TILE_N, other[0])
        if not other[2]:
            pl.set(B().MP_OPT_BATCH_TILE_M, other[1])
        s2, res2, X2, _, _ = run_batched(pl, p, prob.y, (prob.eps, prob.T))
        assert tuple(pl.query(k) for k in q) == other
    assert s2 == 0 and np.array_equal(X, X2)
    assert [r.iters for r in res] == [r.iters for r in res2]


def test_batched_edge_cases():
    psi = W.gaussian_dictionary(64, 300, seed=2)
    prob = W.make_batched(64, 300, 6, 1, 3, seed=2, psi=psi, eps=1e-5, T=500)
    Y = prob.y.copy()
    Y[1] = 0.0                  # y = 0
    Y[3, 7] = np.nan            # non-finite signal
    stops = [(1e-5, 500), (1e-5, 500), (1e-5, 0), (1e-5, 500), (2.0, 500), (0.0, 9)]
    p = B().MP_PREC_BF16
    with GpuPlan(psi, prec_mask=1 << p) as pl:
        s, res, X, atoms, _ = run_batched(pl, p, Y, stops)
        assert s == B().MP_ERR_NONFINITE
        assert res[1].iters == 0 and res[1].stop_reason == B().MP_STOP_ZERO_Y and not np.any(X[1])
        assert res[2].iters == 0 and res[2].stop_reason == B().MP_STOP_MAX_ITERS and not np.any(X[2])
        assert res[3].status == B().MP_ERR_NONFINITE and res[3].iters == 0
        assert res[4].iters == 0 and res[4].stop_reason == B().MP_STOP_CONVERGED
        assert res[5].iters == 9 and res[5].stop_reason == B().MP_STOP_MAX_ITERS
        for b in (0, 5):
            ora = orc.mp(psi, Y[b], stops[b][0], stops[b][1])
            assert list(atoms[b, :res[b].iters]) == list(ora["atoms"])
        # a second call on the same plan (state reuse), B = 1
        s, res1, X1, _, _ = run_batched(pl, p, prob.y[:1], (1e-5, 500))
        assert s == 0 and res1[0].iters == res[0].iters and np.array_equal(X1[0], X[0])
        # precision that the plan does not hold
        s, _, _, _, _ = run_batched(pl, B().MP_PREC_FP8E4M3, prob.y[:1], (1e-5, 500))
        assert s == B().MP_ERR_UNSUPPORTED


def test_gemm_timing_diagnostic():
    """mp_debug_time_gemm times every valid tile shape (and the shape a batch
    would use) and rejects bad shapes, arguments and precisions the plan does
    not hold with the documented status codes."""
    psi = W.gaussian_dictionary(256, 2048, seed=9)
    p = B().MP_PREC_BF16
    with GpuPlan(psi, prec_mask=1 << p) as pl:
        for shape in [(0, 0)] + [t for t in TILES] + [(256, tn, 1) for tn in PAIR_TN]:
            us = B().mp_debug_time_gemm(pl.plan, p, 300, shape, reps=3)
            assert 0.0 < us < 1e6, (shape, us)
        for bad in [(192, 256), (128, 64), (256, 100), (64, 128), (256, 0), (256, 200), (128, 256, 1),
                    (256, 96, 1), (256, 200, 1), (256, 288, 1), (256, 256, 2)]:
            with pytest.raises(B().MpError) as ei:
                B().mp_debug_time_gemm(pl.plan, p, 300, bad, reps=3)
            assert ei.value.status == B().MP_ERR_INVALID, bad
        with pytest.raises(B().MpError) as ei:
            B().mp_debug_time_gemm(pl.plan, p, 0, (0, 0), reps=3)
        assert ei.value.status == B().MP_ERR_INVALID
        with pytest.raises(B().MpError) as ei:
            B().mp_debug_time_gemm(pl.plan, B().MP_PREC_FP8E4M3, 300, (0, 0), reps=3)
        assert ei.value.status == B().MP_ERR_UNSUPPORTED
