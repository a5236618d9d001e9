"""Benchmark of the Matching Pursuit decoder on GB300.

One step = one complete decode (every MP iteration until ||r|| <= eps ||y||
or T) of one signal of the plain FP32 workload N=4096, M=16384, K=256
(256 MiB dictionary, larger than L2, so every iteration streams it from HBM).
Inputs are resident in HBM before the timed region.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank decodes its own signals with its own copy
of the dictionary (independent problems, no collective on the data path);
the time is the max over ranks and ``value`` counts the recoveries of all
ranks (weak scaling).

``--impl reference`` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MP recoveries/s & HBM GB/s vs peak, batched low-prec vs plain FP32; p99 latency"
WORKLOAD = "plain_fp32_N4096_M16384_K256"
KERNEL_SOURCES = ["paper_0809_1833_gb300/csrc/mp_plain.cu", "paper_0809_1833_gb300/csrc/mp_device.cuh",
                  "paper_0809_1833_gb300/csrc/mp_dot.cuh"]


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def tensor_peak():
    """Dense BF16 tensor throughput, TFLOP/s: the measured burst figure,
    else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if d.get("bf16_tflops"):
            return float(d["bf16_tflops"])
    return 1900.0


def traffic_record():
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken
    on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "plain_stream_N4096_M16384_K256.traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_hash") != kernel_hash():
        return None
    return d


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------- problem

def make_problem(n_signals, seed=0):
    from paper_0809_1833_gb300 import workloads as W
    w = W.WORKLOADS[WORKLOAD]
    psi = W.gaussian_dictionary(w["N"], w["M"], seed)
    sigs = [W.make_plain(w["N"], w["M"], w["K"], seed=seed + 1000 * i + 1, eps=w["eps"], T=w["T"], psi=psi)
            for i in range(n_signals)]
    Y = np.stack([s.y[0] for s in sigs])
    return w, psi, Y, sigs


def workload_config(w, world):
    """The ``config`` object of both arms' JSON lines (identical keys)."""
    return {"workload": WORKLOAD, "N": w["N"], "M": w["M"], "K": w["K"], "eps": w["eps"], "T": w["T"],
            "l2": "inputs exceed L2: the 256 MiB dictionary is streamed from HBM every iteration",
            "parallelism": f"dp{world} (independent signals)"}


def oracle_per_iteration(psi, y, eps, n):
    """Seconds per FP64 oracle iteration over the first ``n`` iterations of
    one decode.  Each oracle call widens the dictionary to a fresh FP64 copy
    before its loop; a call with T = 0 (the copy and nothing else) is timed
    right before and subtracted.  Returns (s per iteration, iterations,
    seconds of the timed call)."""
    from oracle import mp_oracle as orc
    t0 = time.perf_counter()
    orc.mp(psi, y, eps, 0, record=False)
    t1 = time.perf_counter()
    out = orc.mp(psi, y, eps, n, record=False)
    t2 = time.perf_counter()
    return max((t2 - t1) - (t1 - t0), 1e-9) / max(out["iters"], 1), out["iters"], t2 - t1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_sample(psi, y, eps, full_iters, budget_s):
    est, _, _ = oracle_per_iteration(psi, y, eps, 8)
    n = int(max(4, min(full_iters, budget_s / est)))
    per_iter, done, dt = oracle_per_iteration(psi, y, eps, n)
    return per_iter, done, dt


def cpu_baseline(psi, y, eps, T, full_iters, budget_s=15.0, single_budget_s=10.0):
    """The FP64 oracle on the host cores over the first iterations of one
    decode, extrapolated to recoveries/s with the full decode's iteration
    count: on all cores (this process) and single-threaded (a child process
    with the BLAS thread count set to 1 before numpy loads)."""
    per_iter, done, dt = _oracle_sample(psi, y, eps, full_iters, budget_s)
    cores = os.cpu_count()
    out = {"value": 1.0 / (per_iter * full_iters), "unit": "recoveries/s", "cores": cores, "kind": "oracle",
           "sample": f"first {done} of {full_iters} iterations of one decode of {WORKLOAD} "
                     f"(FP64 numpy, {dt:.1f} s, the FP64 copy of the dictionary timed apart and subtracted); "
                     f"recoveries/s = 1/(s per iteration x {full_iters})",
           "s_per_iteration": per_iter, "cpu_model": cpu_model()}
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        p = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", str(single_budget_s),
                            "--cpu-worker-iters", str(full_iters)], env=env, capture_output=True, text=True,
                           timeout=600)
        one = json.loads(p.stdout.strip().splitlines()[-1])
        out["single_thread"] = {"value": 1.0 / (one["s_per_iteration"] * full_iters), "unit": "recoveries/s",
                                "cores": 1, "s_per_iteration": one["s_per_iteration"],
                                "sample": f"first {one['iterations']} iterations, {one['seconds']:.1f} s, "
                                          f"BLAS threads 1"}
    except Exception as ex:
        out["single_thread"] = {"value": None, "why": f"{type(ex).__name__}: {ex}"[:200]}
    return out


def cpu_worker(budget_s, full_iters):
    """Child process of cpu_baseline: the same oracle sample with the thread
    count the environment sets; prints one JSON line."""
    w, psi, Y, _ = make_problem(1)
    per_iter, done, dt = _oracle_sample(psi, Y[0], w["eps"], full_iters, budget_s)
    print(json.dumps({"s_per_iteration": per_iter, "iterations": done, "seconds": dt}), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, psi, Y, sigs = make_problem(1)
    from oracle import mp_oracle as orc
    # iteration count of the full decode of this signal, from one untimed
    # full oracle run; each timed step is a bounded prefix of it, with the
    # oracle's one-off FP64 copy of the dictionary timed apart and subtracted
    full_iters = orc.mp(psi, Y[0], w["eps"], w["T"], record=False)["iters"]
    sample_iters = 100
    per_iters, step_s = [], []
    for i in range(args.warmup + args.steps):
        pi, done, dt = oracle_per_iteration(psi, Y[0], w["eps"], sample_iters)
        if i >= args.warmup:
            per_iters.append(pi)
            step_s.append(dt)
    per_iter = sum(per_iters) / len(per_iters)
    v = 1.0 / (per_iter * full_iters)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "recoveries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(step_s) / len(step_s),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, args.gpus),
            "cpu_baseline": {"value": v, "unit": "recoveries/s", "cores": os.cpu_count(), "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"each step = {sample_iters} FP64 oracle iterations of one decode, minus "
                                       f"the oracle's one-off FP64 copy of the dictionary (timed apart); "
                                       f"recoveries/s = 1/(s per iteration x {full_iters})"},
            "e2e": {"value": v, "unit": "recoveries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_0809_1833_gb300 import binding as B

    from paper_0809_1833_gb300 import dp
    n_sig = 4
    w, psi_np, Y_np, sigs = make_problem(n_sig, seed=dp.rank_seed(0, rank))
    N, M = w["N"], w["M"]
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    psi = torch.from_numpy(psi_np).to(dev)
    plan = B.mp_plan_create(N, M, psi.data_ptr(), prec_mask=0, stream=sptr)
    del psi
    Y = torch.from_numpy(Y_np).to(dev)
    X = torch.empty((n_sig, M), dtype=torch.float32, device=dev)
    mode = B.mp_plan_query(plan, B.MP_Q_PLAIN_MODE)

    def step(i):
        b = i % n_sig
        B.mp_recover(plan, Y[b].data_ptr(), X[b].data_ptr(), w["eps"], w["T"], None, False, sptr)

    # iterations per signal (device-side counts) for the algorithmic bytes
    iters = []
    for b in range(n_sig):
        _, r = B.mp_recover(plan, Y[b].data_ptr(), X[b].data_ptr(), w["eps"], w["T"], None, True, sptr)
        iters.append(r.iters)
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = B.mp_plan_query(plan, B.MP_Q_KERNEL_LAUNCHES)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        step(i)
        ev[i][1].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = B.mp_plan_query(plan, B.MP_Q_KERNEL_LAUNCHES) - l0
    clk = clocks.stop()
    per_launch_ms = [a.elapsed_time(b) for a, b in ev]
    # max time over ranks, recoveries summed over ranks (no data-path collective)
    elapsed_s, total_recoveries = dp.aggregate(start.elapsed_time(end) / 1e3, args.steps, dev)
    elapsed_ms = 1e3 * elapsed_s
    value = total_recoveries / elapsed_s

    # roofline of the persistent kernel: algorithmic bytes = 4 N M per iteration
    step_iters = [iters[i % n_sig] for i in range(args.steps)]
    alg_bytes = [4.0 * N * M * it for it in step_iters]
    achieved = sum(alg_bytes) / (sum(per_launch_ms) / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    tr = traffic_record()
    traffic = None
    if tr is not None:
        traffic = tr["dram_bytes_per_iteration"] * (sum(step_iters) / len(step_iters))

    # end to end through the host-buffer entry point
    y_host = [np.ascontiguousarray(Y_np[b]) for b in range(n_sig)]
    x_host = np.empty(M, dtype=np.float32)
    for i in range(2):
        B.mp_recover_host(plan, y_host[i % n_sig], x_host, w["eps"], w["T"])
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        B.mp_recover_host(plan, y_host[i % n_sig], x_host, w["eps"], w["T"])
    e2e_s, e2e_total = dp.aggregate(time.perf_counter() - t0, args.steps, dev)
    e2e = {"value": e2e_total / e2e_s, "unit": "recoveries/s", "h2d_bytes_per_step": 4 * N,
           "d2h_bytes_per_step": 4 * M + 56}

    line = {
        "metric": METRIC, "value": value, "unit": "recoveries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, world),
        "run": {"signals": n_sig, "iterations_per_decode": iters, "plain_mode": int(mode)},
        "hbm_gbs": achieved,
        "us_per_iteration": 1e3 * sum(per_launch_ms) / sum(step_iters),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "mp_plain_kernel<3> (grid streaming)",
                     "algorithmic_bytes_per_launch": sum(alg_bytes) / len(alg_bytes)},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        "paper_context": {"speedup": "GPU vs CPU up to 31x in single and 21x in double precision at M=15000",
                          "hardware": "GeForce GTX 280 (GT200, 240 stream processors, 1 GB) with CUBLAS "
                                      "(CUDA 2.0) vs AMD Phenom 9950 (2.6 GHz) with CBLAS (GSL 1.11)",
                          "workload": "Sec. 4: Bernoulli Psi, N = M/2, K = 0.07M, eps = 1e-7, T = N",
                          "use": "context only (other workload and hardware); see bench.py --paper-timing"},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(psi_np, Y_np[0], w["eps"], w["T"], iters[0], args.cpu_budget)
    B.mp_plan_destroy(plan)
    if rank == 0 and not args.no_batched:
        line["plain_small"] = plain_small_measure()
        line["variants"] = variants_measure()
        # batched low-precision form vs the plain FP32 kernel on the same signals
        line["batched"] = [batched_measure("bf16", n_oracle=4, variants=((256, 0), (512, 896))),
                           batched_measure("fp8", n_plain=4, n_oracle=1, variants=((512, 0),))]
        line["fp8_gemm_peak"] = fp8_gemm_peak()
        # tensor-core fraction of the GEMM: BF16 against the measured burst
        # peak, FP8 against the vendor library's E4M3 rate measured above
        bf16_peak = tensor_peak()
        for bm in line["batched"]:
            g = bm["gemm_full_batch"]
            pk = bf16_peak if bm["precision"] == "bf16" else line["fp8_gemm_peak"]["tflops"]
            g["peak_tflops"] = pk
            g["frac"] = g["tflops"] / pk if pk else None
    if rank == 0 and args.served_duration > 0:
        line["served"] = served_measure(args.served_rate, args.served_duration, gram=args.served_gram)
        if args.served_gram == 0 and args.served_gram_duration > 0:
            # the same workload served with Gram-updated correlations (R = 64)
            line["served_gram"] = served_measure(args.served_rate, args.served_gram_duration, gram=64)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


BATCHED = {"bf16": "batched_bf16_N2048_M8192_B1024", "fp8": "batched_fp8_N8192_M32768_B256"}


def plain_small_measure(reps=20):
    """The 1 MiB plain workload (N=256, M=1024, K=16): the dictionary sits in
    shared memory, so an iteration costs the exchange, not the stream.
    Times every launch shape that can hold it."""
    import torch
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import workloads as W
    name = "plain_fp32_N256_M1024_K16"
    w = W.WORKLOADS[name]
    prob = W.make_workload(name, seed=0)
    s = torch.cuda.current_stream().cuda_stream
    d = torch.from_numpy(prob.psi).cuda()
    plan = B.mp_plan_create(prob.N, prob.M, d.data_ptr(), stream=s)
    y = torch.from_numpy(prob.y[0]).cuda()
    x = torch.empty(prob.M, device="cuda")
    out = {"workload": name, "auto_mode": B.mp_plan_query(plan, B.MP_Q_PLAIN_MODE), "shapes": {}}
    for mode, label in ((1, "cluster_resident"), (2, "grid_resident"), (3, "grid_stream")):
        B.mp_plan_set_option(plan, B.MP_OPT_PLAIN_MODE, mode)
        if B.mp_plan_query(plan, B.MP_Q_PLAIN_MODE) != mode:
            continue
        _, r = B.mp_recover(plan, y.data_ptr(), x.data_ptr(), w["eps"], w["T"], None, True, s)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            B.mp_recover(plan, y.data_ptr(), x.data_ptr(), w["eps"], w["T"], None, False, s)
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3 / reps
        out["shapes"][label] = {"ctas": B.mp_plan_query(plan, B.MP_Q_PLAIN_CTAS), "iterations": r.iters,
                                "us_per_iteration": 1e6 * t / r.iters, "recoveries_per_s": 1.0 / t,
                                "dictionary_GBps_from_smem": 4.0 * prob.N * prob.M * r.iters / t / 1e9}
    B.mp_plan_destroy(plan)
    # the per-iteration floor: the same launch shape on 16 atoms, so an
    # iteration is the cluster exchange and the residual update alone
    tiny = W.gaussian_dictionary(prob.N, 16, seed=1)
    d = torch.from_numpy(tiny).cuda()
    plan = B.mp_plan_create(prob.N, 16, d.data_ptr(), stream=s)
    B.mp_recover(plan, y.data_ptr(), x.data_ptr(), 0.0, 2000, None, True, s)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        B.mp_recover(plan, y.data_ptr(), x.data_ptr(), 0.0, 2000, None, False, s)
    b.record()
    torch.cuda.synchronize()
    out["iteration_floor_us"] = 1e3 * a.elapsed_time(b) / (5 * 2000)
    out["iteration_floor_shape"] = f"mode {B.mp_plan_query(plan, B.MP_Q_PLAIN_MODE)}, 16 atoms, 2000 iterations"
    B.mp_plan_destroy(plan)
    return out


def fp8_gemm_peak(n=8192, reps=20):
    """Dense E4M3 GEMM throughput of this GPU through the vendor library
    (torch._scaled_mm, 8192^3, burst): the denominator for the FP8
    correlations, which the measured peaks do not include."""
    import torch
    try:
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.tensor(1.0, device="cuda")
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        e1.record()
        torch.cuda.synchronize()
        return {"tflops": 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12,
                "how": f"torch._scaled_mm E4M3 x E4M3 -> BF16, {n}^3, {reps} launches after 3 warm-up"}
    except Exception as ex:   # the installed torch may not offer FP8 GEMMs
        return {"tflops": None, "how": f"unavailable: {type(ex).__name__}: {ex}"[:200]}


def variants_measure(n_sig=4, gram_period=32):
    """The benchmark's workload (N=4096, M=16384, K=256) through the two
    decodes beside direct MP: MP with Gram-updated correlations (period R;
    not in the paper, same MP iteration with c_m -= c G[m*][m] between direct
    recomputations) and OMP (the method Sec. 5 names next).  CUDA events per
    decode; the Gram matrix build is timed once, apart."""
    import torch
    from paper_0809_1833_gb300 import binding as B
    w, psi_np, Y_np, sigs = make_problem(n_sig)
    st = torch.cuda.current_stream()
    s = st.cuda_stream
    d = torch.from_numpy(psi_np).cuda()
    plan = B.mp_plan_create(w["N"], w["M"], d.data_ptr(), stream=s)
    del d
    Y = torch.from_numpy(Y_np).cuda()
    x = torch.empty(w["M"], dtype=torch.float32, device="cuda")
    out = {"workload": WORKLOAD, "signals": n_sig}

    def timed(fn):
        recs = []
        for i in range(n_sig):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn(plan, Y[i].data_ptr(), x.data_ptr(), w["eps"], w["T"], None, False, s)
            b.record(st)
            b.synchronize()
            _, r = B.mp_plan_last_result(plan)
            xh = x.cpu().numpy().astype(np.float64)
            xt = sigs[i].x_true[0]
            recs.append((a.elapsed_time(b), r.iters, float(np.sum((xh - xt) ** 2) / np.sum(xt ** 2)) * 100))
        ms = sum(r[0] for r in recs)
        it = sum(r[1] for r in recs)
        return {"recoveries_per_s": 1e3 * n_sig / ms, "ms_per_decode": ms / n_sig, "iterations_per_decode": it / n_sig,
                "us_per_iteration": 1e3 * ms / it, "E_pct_max": max(r[2] for r in recs)}

    B.mp_recover(plan, Y[0].data_ptr(), x.data_ptr(), w["eps"], 2, None, True, s)        # warm-up
    out["direct_mp"] = timed(B.mp_recover)
    B.mp_plan_set_option(plan, B.MP_OPT_PLAIN_GRAM, gram_period)
    t0 = time.perf_counter()
    B.mp_recover(plan, Y[0].data_ptr(), x.data_ptr(), w["eps"], 0, None, True, s)        # builds G
    g_s = time.perf_counter() - t0
    out["gram_mp"] = timed(B.mp_recover)
    out["gram_mp"].update(period=gram_period, gram_build_s=g_s,
                          gram_bytes=B.mp_plan_query(plan, B.MP_Q_GRAM_BYTES),
                          gram_build_tflops=2.0 * w["M"] * w["M"] * w["N"] / g_s / 1e12)
    B.mp_plan_set_option(plan, B.MP_OPT_PLAIN_GRAM, 0)
    B.mp_recover_omp(plan, Y[0].data_ptr(), x.data_ptr(), w["eps"], 2, None, True, s)    # scratch
    out["omp"] = timed(B.mp_recover_omp)
    B.mp_plan_destroy(plan)
    # the floor under the grid shapes' iteration: the same N on one atom per
    # CTA, so an iteration is the grid barrier, the residual update and the
    # FP64 energy alone (OMP adds four such barriers per step, Gram MP runs
    # on this floor plus one row of G)
    G = torch.cuda.get_device_properties(0).multi_processor_count
    tiny = np.ascontiguousarray(psi_np[:G])
    d = torch.from_numpy(tiny).cuda()
    fp = B.mp_plan_create(w["N"], G, d.data_ptr(), stream=s)
    floors = {}
    for mode, label in ((2, "grid_resident"), (3, "grid_stream")):
        B.mp_plan_set_option(fp, B.MP_OPT_PLAIN_MODE, mode)
        B.mp_recover(fp, Y[0].data_ptr(), x.data_ptr(), 0.0, 100, None, True, s)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        B.mp_recover(fp, Y[0].data_ptr(), x.data_ptr(), 0.0, 2000, None, False, s)
        b.record(st)
        b.synchronize()
        floors[label] = 1e3 * a.elapsed_time(b) / 2000
    B.mp_plan_destroy(fp)
    out["grid_iteration_floor_us"] = floors
    out["floor_shape"] = f"N = {w['N']}, {G} atoms (one per CTA), 2000 iterations"
    return out


def batched_measure(prec_name, reps=3, n_plain=16, profile=False, profile_shape=(256, 256), n_oracle=0,
                    variants=(), profile_gram=0):
    """Batched low-precision decode of a whole batched workload vs the plain
    FP32 kernel on the same signals (the first ``n_plain`` of them); x~ of
    ``n_oracle`` signals spread over the batch against full FP64 oracle
    decodes.  ``variants``: (R, S) pairs; each also times the same batch
    with Gram-updated correlations, refresh period R (S = 0: every step;
    S > 0: direct GEMM steps while more than S signals are active, Gram
    steps after), and compares its x~ with the direct decode's bit for bit.
    ``profile_gram`` R > 0 with ``profile``: the profiling case decodes with
    Gram-updated steps of period R instead of GEMM steps."""
    import torch
    from oracle import mp_oracle as orc
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import workloads as W
    name = BATCHED[prec_name]
    w = W.WORKLOADS[name]
    prob = W.make_workload(name, seed=0)
    prec = B.MP_PREC_BF16 if prec_name == "bf16" else B.MP_PREC_FP8E4M3
    s = torch.cuda.current_stream().cuda_stream
    d = torch.from_numpy(prob.psi).cuda()
    plan = B.mp_plan_create(prob.N, prob.M, d.data_ptr(), prec_mask=1 << prec, stream=s)
    del d
    if profile:
        # under a profiler the autotuner's timings are distorted: pin the
        # shape it picks in unprofiled runs
        tn, tm, pair = shape_parts(profile_shape)
        B.mp_plan_set_option(plan, B.MP_OPT_BATCH_PAIR, 2 if pair else 1)
        B.mp_plan_set_option(plan, B.MP_OPT_BATCH_TILE_N, tn)
        if not pair:
            B.mp_plan_set_option(plan, B.MP_OPT_BATCH_TILE_M, tm)
        if profile_gram:
            B.mp_plan_set_option(plan, B.MP_OPT_BATCH_GRAM, profile_gram)
    Y = torch.from_numpy(prob.y).cuda()
    X = torch.empty((prob.B, prob.M), device="cuda")
    stop = (w["eps"], w["T"])
    B.mp_recover_batched(plan, prec, Y.data_ptr(), X.data_ptr(), prob.B, stop, None, s)   # builds the graph
    if profile:
        torch.cuda.synchronize()
        B.mp_recover_batched(plan, prec, Y.data_ptr(), X.data_ptr(), prob.B, stop, None, s)
        B.mp_plan_destroy(plan)
        return {"profile_case": name}
    times = []
    shape = {"signals_per_tile": B.mp_plan_query(plan, B.MP_Q_BATCH_TILE_M),
             "atoms_per_tile": B.mp_plan_query(plan, B.MP_Q_BATCH_TILE_N), "chosen_by": "autotuner"}
    l0 = B.mp_plan_query(plan, B.MP_Q_KERNEL_LAUNCHES)
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        _, res = B.mp_recover_batched(plan, prec, Y.data_ptr(), X.data_ptr(), prob.B, stop, None, s)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b) / 1e3)
    launches = (B.mp_plan_query(plan, B.MP_Q_KERNEL_LAUNCHES) - l0) // reps
    tb = statistics.median(times)
    iters = np.array([r.iters for r in res])
    # how many steps of the decode ran with at most k signals active
    active = np.array([(iters > t).sum() for t in range(int(iters.max()))])
    active_profile = {"steps": int(iters.max()),
                      "steps_with_at_most": {str(k): int((active <= k).sum()) for k in (128, 256, 384, 512)}}
    Xh = X.cpu().numpy()
    supp_b = [orc.support_score(Xh[i], prob.supports[i]) for i in range(prob.B)]
    # x~ against the true sparse signal x (every signal; the FP64 oracle's
    # x~ is compared on a sample by --fp8-error)
    xerr = np.linalg.norm(Xh.astype(np.float64) - prob.x_true, axis=1) / np.linalg.norm(prob.x_true, axis=1)
    xs = torch.empty(prob.M, device="cuda")
    tp, supp_p = 0.0, []
    for i in range(n_plain):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        B.mp_recover(plan, Y[i].data_ptr(), xs.data_ptr(), w["eps"], w["T"], None, False, s)
        b.record()
        torch.cuda.synchronize()
        tp += a.elapsed_time(b) / 1e3
        supp_p.append(orc.support_score(xs.cpu().numpy(), prob.supports[i]))
    # the correlation GEMM alone at the batch's shape, full batch (first step)
    g_us = B.mp_debug_time_gemm(plan, prec, prob.B, reps=20)
    var_out = []
    for R_sw, S_sw in variants:
        B.mp_plan_set_option(plan, B.MP_OPT_BATCH_GRAM, R_sw)
        B.mp_plan_set_option(plan, B.MP_OPT_BATCH_GRAM_BELOW, S_sw)
        Xs = torch.empty_like(X)
        # the first decode builds the plan's Gram matrix (timed apart: a
        # one-off per dictionary, like the BF16 copy)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.mp_recover_batched(plan, prec, Y.data_ptr(), Xs.data_ptr(), prob.B, stop, None, s)
        torch.cuda.synchronize()
        first_s = time.perf_counter() - t0
        ts, l0 = [], B.mp_plan_query(plan, B.MP_Q_KERNEL_LAUNCHES)
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            _, res_s = B.mp_recover_batched(plan, prec, Y.data_ptr(), Xs.data_ptr(), prob.B, stop, None, s)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        ls = (B.mp_plan_query(plan, B.MP_Q_KERNEL_LAUNCHES) - l0) // reps
        tsw = statistics.median(ts)
        Xsh = Xs.cpu().numpy()
        same = np.all(Xsh == Xh, axis=1) & np.array([r.iters == q.iters for r, q in zip(res_s, res)])
        mode = (f"direct BF16 GEMM steps while more than {S_sw} signals are active, then Gram-updated steps"
                if S_sw else "Gram-updated steps throughout (no GEMM)")
        var_out.append({
            "mode": mode + f"; correlations computed directly in FP32 at admission or switch and every {R_sw} "
                           "of a signal's steps",
            "gram_period": R_sw, "switch_below": S_sw, "recoveries_per_s": prob.B / tsw, "ms_per_batch": 1e3 * tsw,
            "speedup_vs_direct": tb / tsw, "signals_equal_to_direct_bitwise": int(same.sum()),
            "support_score_min": float(min(orc.support_score(Xsh[i], prob.supports[i]) for i in range(prob.B))),
            "effective_tflops": 2.0 * prob.N * prob.M * float(iters.sum()) / tsw / 1e12,
            "effective_tflops_note": "direct-step-equivalent correlation work (2 N M per signal-step) per second",
            "gpu_launches_per_batch": int(ls), "gram_bytes": B.mp_plan_query(plan, B.MP_Q_GRAM_BYTES),
            "first_call_s_with_gram_build": first_s})
    gemm = {"rows": prob.B, "us_per_launch": g_us, "tflops": 2.0 * prob.N * prob.M * prob.B / g_us / 1e6,
            "how": "mp_debug_time_gemm: GEMM + top-8 epilogue on the full batch of synthetic rows, CUDA events, "
                   "mean of 20 launches after 2 warm-up"}
    B.mp_plan_destroy(plan)
    oracle_sample = []
    for i in (np.linspace(0, prob.B - 1, n_oracle).astype(int) if n_oracle else []):
        t0 = time.perf_counter()
        o = orc.mp(prob.psi, prob.y[i], w["eps"], w["T"], record=False)
        nx = np.linalg.norm(o["x"])
        oracle_sample.append({"signal": int(i), "x_rel_err_vs_oracle":
                              float(np.linalg.norm(Xh[i].astype(np.float64) - o["x"]) / (nx if nx > 0 else 1.0)),
                              "iters": int(res[i].iters), "oracle_iters": int(o["iters"]),
                              "oracle_s": time.perf_counter() - t0})
    flops = 2.0 * prob.N * prob.M * float(iters.sum())
    rec_b, rec_p = prob.B / tb, n_plain / tp
    return {"workload": name, "precision": prec_name, "signals": prob.B, "recoveries_per_s": rec_b,
            "ms_per_batch": 1e3 * tb, "plain_fp32_recoveries_per_s": rec_p, "speedup_vs_plain": rec_b / rec_p,
            "plain_sample": f"first {n_plain} signals through mp_recover",
            "support_score_mean": float(np.mean(supp_b)), "support_score_min": float(np.min(supp_b)),
            "plain_support_score_mean": float(np.mean(supp_p)),
            "x_rel_err_vs_truth_mean": float(np.mean(xerr)), "x_rel_err_vs_truth_max": float(np.max(xerr)),
            "x_rel_err_vs_oracle_max": max((e["x_rel_err_vs_oracle"] for e in oracle_sample), default=None),
            "oracle_sample": oracle_sample,
            "iterations_total": int(iters.sum()), "iterations_max": int(iters.max()),
            "effective_tflops": flops / tb / 1e12, "gpu_launches_per_batch": int(launches), "gemm_shape": shape,
            "active_rows_profile": active_profile,
            "gemm_full_batch": gemm, "gram_variants": var_out}


def shape_parts(shape):
    """--profile-shape "atoms,signals[,pair]" -> (atoms per tile, signals
    per tile, 1 for a two-SM tile)."""
    tn = int(shape[0])
    tm = int(shape[1]) if len(shape) > 1 else 128
    pair = int(shape[2]) if len(shape) > 2 else 0
    return tn, tm, pair


def gemm_profile_case(prec_name, shape, rows=None):
    """Three launches of the batched workload's correlation GEMM (``rows``
    active synthetic rows, default the full batch) at shape = (atoms per
    tile, signals per tile): the case an ncu capture of the GEMM takes
    (-s 2 -c 1)."""
    import torch
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import workloads as W
    import __graft_entry__
    __graft_entry__.build()
    w = W.WORKLOADS[BATCHED[prec_name]]
    prec = B.MP_PREC_BF16 if prec_name == "bf16" else B.MP_PREC_FP8E4M3
    psi = W.gaussian_dictionary(w["N"], w["M"], seed=0)
    d = torch.from_numpy(psi).cuda()
    plan = B.mp_plan_create(w["N"], w["M"], d.data_ptr(), prec_mask=1 << prec)
    del d
    tn, tm, pair = shape_parts(shape)
    rows = rows or w["B"]
    us = B.mp_debug_time_gemm(plan, prec, rows, (tm, tn, pair), reps=1)
    B.mp_plan_destroy(plan)
    return {"profile_case": BATCHED[prec_name], "rows": rows, "gemm_shape": [tm, tn, pair], "us": us,
            "tflops": 2.0 * w["N"] * w["M"] * rows / us / 1e6}


def gemm_sweep(prec_name, shape, rows=(64, 128, 256, 384, 512, 768, 1024)):
    """The batched workload's correlation GEMM alone (GEMM + top-8 epilogue,
    synthetic rows) at several active-row counts, mean of 50 launches each
    with CUDA events: how the step's GEMM time falls as a batch drains."""
    import torch
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import workloads as W
    import __graft_entry__
    __graft_entry__.build()
    w = W.WORKLOADS[BATCHED[prec_name]]
    prec = B.MP_PREC_BF16 if prec_name == "bf16" else B.MP_PREC_FP8E4M3
    psi = W.gaussian_dictionary(w["N"], w["M"], seed=0)
    d = torch.from_numpy(psi).cuda()
    plan = B.mp_plan_create(w["N"], w["M"], d.data_ptr(), prec_mask=1 << prec)
    del d
    tn, tm, pair = shape_parts(shape)
    us = {str(r): B.mp_debug_time_gemm(plan, prec, r, (tm, tn, pair), reps=50) for r in rows if r <= w["B"]}
    B.mp_plan_destroy(plan)
    return {"gemm_sweep": BATCHED[prec_name], "gemm_shape": [tm, tn, pair], "us_by_active_rows": us}


def served_measure(rate=2000.0, duration=60.0, pool_s=5.0, seed=0, max_slots=256, drain_s=120.0, n_oracle=2,
                   gram=0):
    """Poisson arrivals over the four resident dictionaries of the served
    workload; every request is submitted at its arrival time through the
    server's C ABI and polled until done.  Reports offered / completed rates,
    rejections and latency percentiles (server clock: submit -> result
    ready; client clock: submit -> successful poll), the support score of
    every completed request, and x~ against the FP64 oracle for the first
    ``n_oracle`` completed requests of each dictionary.

    Signals: per dictionary a pool of distinct seeded signals as large as
    ``pool_s`` seconds of that dictionary's arrivals (K ~ U{4..N/16}); a
    request takes the next signal of its dictionary's pool.  ``gram`` > 0
    serves every dictionary in the Gram mode with that period
    (MP_OPT_BATCH_GRAM)."""
    import torch
    from oracle import mp_oracle as orc
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import workloads as W
    wl = W.WORKLOADS["served_4dict_poisson2000"]
    dicts = wl["dicts"]
    prec = B.MP_PREC_BF16
    s = torch.cuda.current_stream().cuda_stream
    pool = max(16, int(np.ceil(rate * pool_s / len(dicts))))
    plans, pools, psis = [], [], []
    t_gen = time.perf_counter()
    for di, (N, M) in enumerate(dicts):
        psi = W.gaussian_dictionary(N, M, seed + 10 + di)
        psis.append(psi)
        d = torch.from_numpy(psi).cuda()
        plans.append(B.mp_plan_create(N, M, d.data_ptr(), prec_mask=1 << prec, stream=s))
        if gram:
            B.mp_plan_set_option(plans[-1], B.MP_OPT_BATCH_GRAM, gram)
        del d
        g = np.random.default_rng([seed, 50 + di])
        ys, sups = [], []
        for k in range(pool):
            K = int(g.integers(4, N // 16 + 1))
            x, supp = W.sparse_signal(M, K, g, wl["values"])
            ys.append(np.ascontiguousarray(W.encode(psi, x)))
            sups.append(supp)
        pools.append((ys, sups))
    t_gen = time.perf_counter() - t_gen
    srv = B.mp_server_create(96 << 30, max_slots, 1 << 20)
    ids = [B.mp_server_add_dictionary(srv, p, prec) for p in plans]
    slots = [B.mp_server_dictionary_slots(srv, i) for i in ids]
    arr, dsel, _ = W.served_requests(dicts, rate, duration, seed)
    xbuf = [np.empty(M, np.float32) for (_, M) in dicts]
    # warm-up: one request per dictionary
    for di in range(len(dicts)):
        _, t = B.mp_server_submit(srv, ids[di], pools[di][0][0], wl["eps"], wl["T"])
        while B.mp_server_poll(srv, t)[0] == B.MP_PENDING:
            time.sleep(0.001)
    B.mp_server_reset_stats(srv)
    pending, lat, rejected, n_sub = {}, [], 0, 0
    next_sig = [0] * len(dicts)
    scores, sampled = [], []
    t0 = time.perf_counter()
    i, n = 0, len(arr)
    while i < n or pending:
        now = time.perf_counter() - t0
        while i < n and arr[i] <= now:
            di = int(dsel[i])
            k = next_sig[di] % pool
            next_sig[di] += 1
            st, t = B.mp_server_submit(srv, ids[di], pools[di][0][k], wl["eps"], wl["T"])
            if st == 0:
                pending[t] = (now, di, k)
                n_sub += 1
            else:
                rejected += 1
            i += 1
        done = []
        for t, (ts, di, k) in pending.items():
            st, _ = B.mp_server_poll(srv, t, xbuf[di])
            if st == B.MP_OK:
                done.append(t)
                lat.append(time.perf_counter() - t0 - ts)
                scores.append(orc.support_score(xbuf[di], pools[di][1][k]))
                if sum(1 for q in sampled if q[0] == di) < n_oracle:
                    sampled.append((di, k, xbuf[di].copy()))
            if len(done) >= 256:
                break
        for t in done:
            del pending[t]
        if now > duration + drain_s:
            break
        if not done and (i >= n or arr[i] > now + 5e-4):
            time.sleep(2e-4)
    wall = time.perf_counter() - t0
    stt = B.mp_server_get_stats(srv)
    B.mp_server_destroy(srv)
    for p in plans:
        B.mp_plan_destroy(p)
    # x~ of sampled requests against the FP64 oracle's decode of the same y
    errs = []
    for di, k, xg in sampled:
        o = orc.mp(psis[di], pools[di][0][k], wl["eps"], wl["T"], record=False)
        nx = np.linalg.norm(o["x"])
        errs.append({"dictionary": list(dicts[di]), "x_rel_err_vs_oracle":
                     float(np.linalg.norm(xg.astype(np.float64) - o["x"]) / (nx if nx > 0 else 1.0)),
                     "oracle_iters": int(o["iters"])})
    lat = np.array(lat)
    scores = np.array(scores) if scores else np.zeros(0)
    return {"workload": "served_4dict_poisson2000", "dictionaries": [list(d) for d in dicts], "precision": "bf16",
            "correlations": f"Gram-updated, direct BF16 GEMM every {gram} steps" if gram else
                            "direct BF16 GEMM every step",
            "slots_per_dictionary": slots, "gram_period": gram, "offered_rps": rate, "duration_s": duration, "requests": int(n),
            "submitted_rps": float(n_sub + rejected) / max(min(wall, duration), 1e-9),
            "unfinished_at_stop": len(pending),
            "submitted": int(n_sub), "rejected": int(rejected), "rejected_pct": 100.0 * rejected / max(n, 1),
            "completed": int(stt.completed), "completed_rps": float(stt.completed) / wall, "wall_s": wall,
            "server_p50_ms": 1e3 * stt.latency_p50_s, "server_p99_ms": 1e3 * stt.latency_p99_s,
            "client_p50_ms": 1e3 * float(np.percentile(lat, 50)) if lat.size else None,
            "client_p99_ms": 1e3 * float(np.percentile(lat, 99)) if lat.size else None,
            "support_score_mean": float(scores.mean()) if scores.size else None,
            "support_score_min": float(scores.min()) if scores.size else None,
            "support_scored_requests": int(scores.size),
            "oracle_sample": errs,
            "x_rel_err_vs_oracle_max": max((e["x_rel_err_vs_oracle"] for e in errs), default=None),
            "signal_pool": f"{pool} distinct seeded signals per dictionary ({pool_s:g} s of arrivals), "
                           f"K ~ U{{4..N/16}}, taken in turn by that dictionary's requests",
            "signal_generation_s": t_gen}


def gram_steps(prec_name="bf16", rows=(1024, 768, 512, 256, 64), settings=((256, 0), (320, 0), (512, 896)),
               reps=5):
    """Direct against Gram-updated steps on a batched workload.  Per-step
    device time at several active-signal counts: the first n signals decoded
    with the iteration cap at 16 and at 48 (nearly all of them still active
    at 48), (t48 - t16) / 32 steps, direct and with Gram steps from
    admission (R = 1024: no refresh inside the window).  Then the whole
    batch in each (R, S) setting (S = 0: Gram steps from admission; S > 0:
    direct steps while more than S signals are active), with the count of
    signals whose x~ equals the direct decode's bit for bit.  One JSON line
    per measurement."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import workloads as W
    name = BATCHED[prec_name]
    w = W.WORKLOADS[name]
    prob = W.make_workload(name, seed=0)
    prec = B.MP_PREC_BF16 if prec_name == "bf16" else B.MP_PREC_FP8E4M3
    d = torch.from_numpy(prob.psi).cuda()
    plan = B.mp_plan_create(prob.N, prob.M, d.data_ptr(), prec_mask=1 << prec)
    del d
    Yall = torch.from_numpy(prob.y).cuda()
    X = torch.empty((prob.B, prob.M), device="cuda")

    def t_ms(n, T):
        Y = Yall[:n]
        B.mp_recover_batched(plan, prec, Y.data_ptr(), X.data_ptr(), n, (w["eps"], T))
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            _, res = B.mp_recover_batched(plan, prec, Y.data_ptr(), X.data_ptr(), n, (w["eps"], T))
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts), res

    for gram in (0, 1024):
        B.mp_plan_set_option(plan, B.MP_OPT_BATCH_GRAM, gram)
        B.mp_plan_set_option(plan, B.MP_OPT_BATCH_GRAM_BELOW, 0)
        for n in rows:
            n = min(n, prob.B)
            t1, _ = t_ms(n, 16)
            t2, res = t_ms(n, 48)
            print(json.dumps({"gram_steps": name, "step": "gram" if gram else "direct", "signals": n,
                              "active_at_step_48": int(sum(r.iters >= 48 for r in res)),
                              "us_per_step": (t2 - t1) * 1e3 / 32}), flush=True)
    B.mp_plan_set_option(plan, B.MP_OPT_BATCH_GRAM, 0)
    t0, _ = t_ms(prob.B, w["T"])
    x0 = X.cpu().numpy()
    print(json.dumps({"gram_steps": name, "decode": "direct", "ms": t0, "recoveries_per_s": prob.B / t0 * 1e3}),
          flush=True)
    for R, S in settings:
        B.mp_plan_set_option(plan, B.MP_OPT_BATCH_GRAM, R)
        B.mp_plan_set_option(plan, B.MP_OPT_BATCH_GRAM_BELOW, S)
        t, _ = t_ms(prob.B, w["T"])
        x = X.cpu().numpy()
        print(json.dumps({"gram_steps": name, "decode": "gram", "gram_period": R, "switch_below": S, "ms": t,
                          "recoveries_per_s": prob.B / t * 1e3,
                          "signals_equal_to_direct_bitwise": int(np.all(x == x0, axis=1).sum())}), flush=True)
    B.mp_plan_destroy(plan)


def step_breakdown(rows=(1, 2, 4, 8, 16), dict_index=3, reps=3, gram=0, T=None):
    """Per-step device time of the batched BF16 decode on one served
    dictionary at a few active-row counts: the whole step (mp_recover_batched
    on that many signals, divided by the steps the longest one needed), the
    correlation GEMM alone (mp_debug_time_gemm at the same rows, synthetic
    residuals) and their difference (select / rescore / update and the
    graph's step hand-off), next to the floor of reading the BF16 dictionary
    once from HBM.  One JSON line per row count.  ``gram`` > 0: the Gram
    mode with that period (no GEMM runs in that mode; the GEMM column is
    the direct step's, for comparison).  ``T`` caps the iterations (a small
    case for a profiler)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import workloads as W
    wl = W.WORKLOADS["served_4dict_poisson2000"]
    N, M = wl["dicts"][dict_index]
    prec = B.MP_PREC_BF16
    psi = W.gaussian_dictionary(N, M, 10 + dict_index)
    d = torch.from_numpy(psi).cuda()
    plan = B.mp_plan_create(N, M, d.data_ptr(), prec_mask=1 << prec)
    if gram:
        B.mp_plan_set_option(plan, B.MP_OPT_BATCH_GRAM, gram)
    del d
    hbm, _ = measured_peaks()
    g = np.random.default_rng([0, 77])
    for nrow in rows:
        ys = []
        for _ in range(nrow):
            K = int(g.integers(4, N // 16 + 1))
            x, _ = W.sparse_signal(M, K, g, wl["values"])
            ys.append(W.encode(psi, x))
        Y = torch.from_numpy(np.stack(ys)).cuda()
        X = torch.empty((nrow, M), device="cuda")
        Tcap = T or wl["T"]
        B.mp_recover_batched(plan, prec, Y.data_ptr(), X.data_ptr(), nrow, (wl["eps"], Tcap))
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            _, res = B.mp_recover_batched(plan, prec, Y.data_ptr(), X.data_ptr(), nrow, (wl["eps"], Tcap))
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b) * 1e3)
        steps = max(r.iters for r in res)
        step_us = statistics.median(times) / steps
        gemm_us = B.mp_debug_time_gemm(plan, prec, nrow, reps=50)
        print(json.dumps({"step_breakdown": {
            "dictionary": [N, M], "active_rows": nrow, "steps": steps, "us_per_step": step_us, "gram_period": gram,
            "gemm_us": gemm_us, "rest_us": step_us - gemm_us,
            "gemm_shape": [B.mp_plan_query(plan, B.MP_Q_BATCH_TILE_M), B.mp_plan_query(plan, B.MP_Q_BATCH_TILE_N)],
            "hbm_floor_us": 2.0 * N * M / (hbm * 1e3)}}), flush=True)
    B.mp_plan_destroy(plan)


def shard_overhead(iters=300):
    """Per-iteration cost of the atom-sharded decode's host loop
    (paper_0809_1833_gb300/sharded.py) on one GPU, on the benchmark's
    dictionary as a single shard: the persistent kernel (mp_recover) capped
    at ``iters`` iterations; the sharded loop with no exchange (two kernel
    launches and a Python step per iteration); and the same with the record
    all-gathered every iteration through a one-rank NCCL group (the
    collective's launch and synchronisation, no link transfer).  Prints one
    JSON line."""
    import torch
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import sharded as S
    w, psi_np, Y_np, _ = make_problem(1)
    N, M = w["N"], w["M"]
    st = torch.cuda.current_stream()
    d = torch.from_numpy(psi_np).cuda()
    plan = B.mp_plan_create(N, M, d.data_ptr(), stream=st.cuda_stream)
    del d
    y = torch.from_numpy(Y_np[0]).cuda()
    x = torch.empty(M, device="cuda")

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    t_dir, _ = timed(lambda: B.mp_recover(plan, y.data_ptr(), x.data_ptr(), 0.0, iters, None, True, st.cuda_stream))
    ops = S.ShardOps(plan, 0, y, stream=st.cuda_stream)
    t_loc, r_loc = timed(lambda: S.sharded_recover(ops, 0.0, iters, check_every=iters + 1))
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ.setdefault("MASTER_PORT", "29533")
    out = {"workload": WORKLOAD, "iterations": iters,
           "direct_us_per_iteration": 1e6 * t_dir / iters,
           "sharded_no_exchange_us_per_iteration": 1e6 * t_loc / iters,
           "record_bytes": B.mp_shard_record_bytes(plan)}
    try:
        dist.init_process_group("nccl", rank=0, world_size=1)
        g = dist.new_group([0])
        recs = torch.empty(B.mp_shard_record_bytes(plan), dtype=torch.uint8, device="cuda")

        def with_gather():
            ops.init(0.0, iters)
            for _ in range(iters):
                rec = ops.local()
                dist.all_gather_into_tensor(recs, rec, group=g)
                ops.apply(recs, 1)
            return ops.result()
        t_g, _ = timed(with_gather)
        out["sharded_nccl_1rank_us_per_iteration"] = 1e6 * t_g / iters
        dist.destroy_process_group()
    except Exception as ex:   # no NCCL here
        out["sharded_nccl_1rank_us_per_iteration"] = None
        out["nccl"] = f"{type(ex).__name__}: {ex}"[:200]
    out["host_loop_overhead_us"] = out["sharded_no_exchange_us_per_iteration"] - out["direct_us_per_iteration"]
    B.mp_plan_destroy(plan)
    print(json.dumps({"shard_overhead": out}), flush=True)


def fp8_error(n_sample=2):
    """The FP8 batched workload (N=8192, M=32768, 256 signals) decoded in one
    batch; for the first n_sample signals the FP64 oracle's decode of the same
    y (FP64 throughout) is the reference: relative L2 difference of x~, both
    iteration counts, and both errors against the true signal.  The oracle
    takes about half a minute per signal on 16 host cores."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from oracle import mp_oracle as orc
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import workloads as W
    name = BATCHED["fp8"]
    w = W.WORKLOADS[name]
    prob = W.make_workload(name, seed=0)
    prec = B.MP_PREC_FP8E4M3
    s = torch.cuda.current_stream().cuda_stream
    d = torch.from_numpy(prob.psi).cuda()
    plan = B.mp_plan_create(prob.N, prob.M, d.data_ptr(), prec_mask=1 << prec, stream=s)
    del d
    Y = torch.from_numpy(prob.y).cuda()
    X = torch.empty((prob.B, prob.M), device="cuda")
    _, res = B.mp_recover_batched(plan, prec, Y.data_ptr(), X.data_ptr(), prob.B, (w["eps"], w["T"]), None, s)
    torch.cuda.synchronize()
    Xh = X.cpu().numpy().astype(np.float64)
    B.mp_plan_destroy(plan)
    for i in range(n_sample):
        t0 = time.perf_counter()
        o = orc.mp(prob.psi, prob.y[i], w["eps"], w["T"])
        dt = time.perf_counter() - t0
        xo = np.asarray(o["x"], dtype=np.float64)
        nx = np.linalg.norm(prob.x_true[i])
        print(json.dumps({"fp8_vs_fp64": {
            "workload": name, "signal": i, "eps": w["eps"],
            "fp8_iters": int(res[i].iters), "fp64_iters": int(o["iters"]),
            "x_rel_diff_fp8_vs_fp64": float(np.linalg.norm(Xh[i] - xo) / np.linalg.norm(xo)),
            "fp8_x_rel_err_vs_truth": float(np.linalg.norm(Xh[i] - prob.x_true[i]) / nx),
            "fp64_x_rel_err_vs_truth": float(np.linalg.norm(xo - prob.x_true[i]) / nx),
            "fp8_rel_residual": float(res[i].rel_residual),
            "fp8_support_score": float(orc.support_score(Xh[i].astype(np.float32), prob.supports[i])),
            "oracle_s": dt}}), flush=True)


def served_sweep(rates, duration=5.0):
    """The served workload at increasing Poisson rates (C5's lambda sweep):
    one JSON line per rate with offered / submitted / completed rates,
    rejections and latency percentiles; arrivals last `duration` seconds and
    the backlog then gets at most 10 s to drain."""
    import __graft_entry__
    __graft_entry__.build()
    for r in rates:
        print(json.dumps({"served_sweep": served_measure(r, duration, drain_s=10.0)}), flush=True)


def run_profile_case(iters):
    """Small case for ncu: the full-size dictionary, one decode capped at
    ``iters`` iterations (one launch of the streaming kernel)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_0809_1833_gb300 import binding as B
    w, psi_np, Y_np, _ = make_problem(1)
    s = torch.cuda.current_stream().cuda_stream
    psi = torch.from_numpy(psi_np).cuda()
    plan = B.mp_plan_create(w["N"], w["M"], psi.data_ptr(), stream=s)
    del psi
    y = torch.from_numpy(Y_np[0]).cuda()
    x = torch.empty(w["M"], dtype=torch.float32, device="cuda")
    _, r = B.mp_recover(plan, y.data_ptr(), x.data_ptr(), w["eps"], iters, None, True, s)
    print(json.dumps({"profile_case": WORKLOAD, "iterations": r.iters,
                      "dram_bytes_algorithmic_per_iteration": 4 * w["N"] * w["M"]}))
    B.mp_plan_destroy(plan)


def run_profile64_case(M, iters):
    """Small case for ncu: Sec. 4's FP64 timing problem at M (N = M/2), one
    FP64 decode capped at ``iters`` iterations (one kernel launch)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import workloads as W
    prob = W.paper_timing_problem(M, seed=0, fp64=True)
    N = prob.psi.shape[1]
    sh = torch.cuda.current_stream().cuda_stream
    psi = torch.from_numpy(prob.psi).cuda()
    plan = B.mp_plan_create_f64(N, M, psi.data_ptr(), stream=sh)
    del psi
    y = torch.from_numpy(prob.y[0]).cuda()
    x = torch.empty(M, dtype=torch.float64, device="cuda")
    _, r = B.mp_recover_f64(plan, y.data_ptr(), x.data_ptr(), prob.eps, iters, None, True, sh)
    print(json.dumps({"profile_case": f"paper_timing_fp64_M{M}", "iterations": r.iters,
                      "mode": B.mp_plan_query(plan, B.MP_Q_PLAIN64_MODE),
                      "fp64_flops_algorithmic_per_iteration": 2 * N * M}))
    B.mp_plan_destroy(plan)


PAPER_TIMING_SIZES = [1000, 3000, 5000, 7000, 9000, 11000, 13000, 15000]


def paper_timing_sweep(sizes, reps=3, cpu_budget_s=4.0):
    """Sec. 4's CPU-vs-GPU sweep: M = 1000..15000, N = M/2, K = 0.07M,
    Bernoulli Psi, eps = 1e-7, T = N; one decode per size and precision
    (the FP32 decode on the FP32 dictionary, the FP64 decode on the same
    dictionary drawn in FP64), timed with CUDA events after a warm-up decode.
    The CPU column is the FP64 oracle on the host cores, timed over a bounded
    prefix of the decode and scaled by the GPU FP64 run's iteration count.
    One JSON line per size."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import workloads as W
    from oracle import mp_oracle as orc
    st = torch.cuda.current_stream()
    sh = st.cuda_stream
    for M in sizes:
        row = {"M": M}
        for prec in ("fp32", "fp64"):
            prob = W.paper_timing_problem(M, seed=0, fp64=prec == "fp64")
            N, T, eps = prob.N, prob.T, prob.eps
            row.update(N=N, K=len(prob.supports[0]), T=T, eps=eps)
            dt = torch.float64 if prec == "fp64" else torch.float32
            psi = torch.from_numpy(prob.psi).cuda()
            if prec == "fp64":
                plan = B.mp_plan_create_f64(N, M, psi.data_ptr(), stream=sh)
                rec, mode_q = B.mp_recover_f64, B.MP_Q_PLAIN64_MODE
            else:
                plan = B.mp_plan_create(N, M, psi.data_ptr(), stream=sh)
                rec, mode_q = B.mp_recover, B.MP_Q_PLAIN_MODE
            del psi
            y = torch.from_numpy(prob.y[0]).cuda()
            x = torch.empty(M, dtype=dt, device="cuda")
            rec(plan, y.data_ptr(), x.data_ptr(), eps, T, None, True, sh)
            times = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                rec(plan, y.data_ptr(), x.data_ptr(), eps, T, None, False, sh)
                e1.record(st)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            _, r = B.mp_plan_last_result(plan)
            xh = x.cpu().numpy().astype(np.float64)
            xt = prob.x_true[0]
            ms = statistics.median(times)
            row[prec] = {"ms_per_decode": ms, "iterations": r.iters, "stop_reason": r.stop_reason,
                         "rel_residual": r.rel_residual, "mode": B.mp_plan_query(plan, mode_q),
                         "us_per_iteration": 1e3 * ms / max(r.iters, 1),
                         "dictionary_gbs": (prob.psi.itemsize * N * M * r.iters) / (ms * 1e6),
                         "E_pct": 100.0 * float(np.sum((xh - xt) ** 2) / np.sum(xt ** 2))}
            B.mp_plan_destroy(plan)
            if prec == "fp64":
                # CPU leg: the FP64 oracle over a bounded prefix of the same decode
                t0 = time.perf_counter()
                orc.mp(prob.psi, prob.y[0], eps, 1, record=False)
                t1 = time.perf_counter()
                n = 2
                while True:
                    t2 = time.perf_counter()
                    o = orc.mp(prob.psi, prob.y[0], eps, n, record=False)
                    t3 = time.perf_counter()
                    if (t3 - t2) > cpu_budget_s / 4 or n >= r.iters:
                        break
                    n *= 4
                per_iter = max((t3 - t2) - (t1 - t0), 1e-9) / max(o["iters"] - 1, 1)
                row["cpu_fp64_oracle"] = {"ms_per_decode_est": 1e3 * per_iter * r.iters,
                                          "ms_per_iteration": 1e3 * per_iter, "iterations_timed": o["iters"],
                                          "cores": os.cpu_count()}
        c = row["cpu_fp64_oracle"]["ms_per_decode_est"]
        row["speedup_vs_cpu_oracle"] = {"fp32": c / row["fp32"]["ms_per_decode"],
                                        "fp64": c / row["fp64"]["ms_per_decode"]}
        print(json.dumps({"paper_timing": row}), flush=True)


def phase_diagram(trials=100, prec_name="bf16"):
    """Sec. 3's reconstruction-error diagram E(sigma, rho) (Eq. 14): M = 1000,
    sigma = K/M and rho = N/M on a 0.05 grid, ``trials`` signals per cell,
    eps = 1e-7, T = N.  One batched decode per rho (its 20 x trials signals
    share that rho's Bernoulli dictionary).  Prints one JSON line: the mean
    E per cell (rows rho, columns sigma), the fraction of signals with
    E < 1 %, and the decode time per rho."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_0809_1833_gb300 import binding as B
    from paper_0809_1833_gb300 import workloads as W
    P = {"bf16": B.MP_PREC_BF16, "fp8": B.MP_PREC_FP8E4M3}[prec_name]
    st = torch.cuda.current_stream()
    grid = list(W.PHASE_GRID)
    E_rows, ok_rows, secs, iters = [], [], [], []
    for rho in grid:
        prob = W.phase_diagram_batch(rho, grid, trials)
        psi = torch.from_numpy(prob.psi).cuda()
        plan = B.mp_plan_create(prob.N, prob.M, psi.data_ptr(), prec_mask=1 << P, stream=st.cuda_stream)
        del psi
        Y = torch.from_numpy(prob.y).cuda()
        X = torch.empty((prob.B, prob.M), dtype=torch.float32, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s, res = B.mp_recover_batched(plan, P, Y.data_ptr(), X.data_ptr(), prob.B, (prob.eps, prob.T), None,
                                      st.cuda_stream)
        e1.record(st)
        e1.synchronize()
        B.check(s, "mp_recover_batched")
        secs.append(e0.elapsed_time(e1) / 1e3)
        iters.append(int(sum(r.iters for r in res)))
        xt = prob.x_true
        E = 100.0 * np.sum((X.cpu().numpy().astype(np.float64) - xt) ** 2, axis=1) / np.sum(xt ** 2, axis=1)
        E = E.reshape(len(grid), trials)
        E_rows.append([float(v) for v in E.mean(axis=1)])
        ok_rows.append([float(v) for v in (E < 1.0).mean(axis=1)])
        B.mp_plan_destroy(plan)
    print(json.dumps({"phase_diagram": {"M": W.PHASE_M, "trials": trials, "precision": prec_name,
                                        "eps": 1e-7, "T": "N", "sigma": grid, "rho": grid,
                                        "E_pct_mean": E_rows, "frac_E_below_1pct": ok_rows,
                                        "decode_s_per_rho": secs, "signal_iterations_per_rho": iters,
                                        "total_decode_s": sum(secs)}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--profile", type=int, default=0,
                    help="profiling case: one decode capped at this many iterations, then exit")
    ap.add_argument("--profile-batched", choices=["bf16", "fp8"], default=None,
                    help="profiling case: one batched decode of that workload, then exit")
    ap.add_argument("--profile-shape", default="256,256",
                    help="GEMM atoms per tile, signals per tile and (optional third value 1) a two-SM "
                         "tile for --profile-batched / --profile-gemm / --gemm-sweep")
    ap.add_argument("--profile-rows", type=int, default=None, help="active rows of the --profile-gemm case")
    ap.add_argument("--gemm-sweep", choices=["bf16", "fp8"], default=None,
                    help="time the batched workload's GEMM alone at several active-row counts (--profile-shape)")
    ap.add_argument("--profile-gemm", choices=["bf16", "fp8"], default=None,
                    help="profiling case: the batched workload's correlation GEMM on its full batch of "
                         "synthetic rows, 3 launches (2 warm-up), at --profile-shape, then exit")
    ap.add_argument("--profile64", type=int, nargs=2, metavar=("M", "ITERS"), default=None,
                    help="profiling case: Sec. 4's FP64 problem at M, one decode capped at ITERS, then exit")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-only", type=int, default=0, metavar="REPEATS",
                    help="print only the batched BF16 and FP8 lines, REPEATS times")
    ap.add_argument("--served-duration", type=float, default=60.0,
                    help="seconds of Poisson arrivals for the served measurement (0 = skip)")
    ap.add_argument("--served-rate", type=float, default=2000.0)
    ap.add_argument("--served-only", action="store_true", help="run only the served measurement")
    ap.add_argument("--fp8-error", type=int, default=None, metavar="S",
                    help="run only the FP8 workload's decode against the FP64 oracle on S sampled signals")
    ap.add_argument("--served-sweep", nargs="*", type=float, default=None,
                    help="run only the served workload at these Poisson rates, req/s "
                         "(default 1000 2000 3000 4000 6000 8000 12000)")
    ap.add_argument("--paper-timing", nargs="*", type=int, default=None,
                    help="run only Sec. 4's CPU-vs-GPU size sweep (FP32 and FP64) at these M "
                         f"(default {PAPER_TIMING_SIZES})")
    ap.add_argument("--phase-diagram", choices=["bf16", "fp8"], default=None,
                    help="run only Sec. 3's E(sigma, rho) diagram with the batched decode in this precision")
    ap.add_argument("--trials", type=int, default=100, help="signals per phase-diagram cell")
    ap.add_argument("--step-breakdown", action="store_true",
                    help="run only the per-step time breakdown of the batched BF16 decode on the largest served "
                         "dictionary at 1-16 active rows")
    ap.add_argument("--served-gram-duration", type=float, default=30.0,
                    help="seconds of the extra served record with Gram-updated correlations (R = 64) in the "
                         "default line (0 = skip)")
    ap.add_argument("--served-gram", type=int, default=0,
                    help="serve in the Gram mode with this refresh period (a multiple of 16; 0 = direct steps)")
    ap.add_argument("--breakdown-rows", type=int, nargs="*", default=None,
                    help="active-row counts of --step-breakdown (default 1 2 4 8 16)")
    ap.add_argument("--breakdown-T", type=int, default=None, help="iteration cap of --step-breakdown")
    ap.add_argument("--profile-gram", type=int, default=0, metavar="R",
                    help="with --profile-batched: the decode takes Gram-updated steps of period R")
    ap.add_argument("--gram-steps", choices=["bf16", "fp8"], default=None,
                    help="per-step time of direct and Gram-updated steps, and whole decodes in the Gram settings")
    ap.add_argument("--shard-overhead", action="store_true",
                    help="run only the per-iteration cost of the atom-sharded host loop on one GPU")
    ap.add_argument("--cpu-worker", type=float, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-worker-iters", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_worker is not None:
        cpu_worker(args.cpu_worker, args.cpu_worker_iters)
        return
    if args.shard_overhead:
        shard_overhead()
        return
    if args.gram_steps:
        if args.gram_steps == "fp8":
            gram_steps("fp8", rows=(256, 128, 64), settings=((512, 0), (1024, 0)), reps=2)
        else:
            gram_steps("bf16")
        return
    if args.step_breakdown:
        step_breakdown(rows=tuple(args.breakdown_rows or (1, 2, 4, 8, 16)), gram=args.served_gram,
                       T=args.breakdown_T)
        return
    if args.phase_diagram:
        phase_diagram(args.trials, args.phase_diagram)
        return
    if args.paper_timing is not None:
        paper_timing_sweep(args.paper_timing or PAPER_TIMING_SIZES)
        return
    if args.fp8_error is not None:
        fp8_error(args.fp8_error)
        return
    if args.served_sweep is not None:
        served_sweep(args.served_sweep or [1000, 2000, 3000, 4000, 6000, 8000, 12000])
        return
    if args.served_only:
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps(served_measure(args.served_rate, args.served_duration, gram=args.served_gram)))
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.profile64:
        run_profile64_case(*args.profile64)
        return
    if args.gemm_sweep:
        shape = tuple(int(v) for v in args.profile_shape.split(","))
        print(json.dumps(gemm_sweep(args.gemm_sweep, shape)))
        return
    if args.profile_gemm:
        shape = tuple(int(v) for v in args.profile_shape.split(","))
        print(json.dumps(gemm_profile_case(args.profile_gemm, shape, args.profile_rows)))
        return
    if args.batched_only:
        import __graft_entry__
        __graft_entry__.build()
        for _ in range(args.batched_only):
            for prec in ("bf16", "fp8"):
                print(json.dumps(batched_measure(prec, n_plain=2)))
        return
    if args.profile_batched:
        import __graft_entry__
        __graft_entry__.build()
        shape = tuple(int(v) for v in args.profile_shape.split(","))
        print(json.dumps(batched_measure(args.profile_batched, profile=True, profile_shape=shape,
                                         profile_gram=args.profile_gram)))
    elif args.profile:
        run_profile_case(args.profile)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
