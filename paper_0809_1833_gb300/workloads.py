"""Seeded synthetic workloads for the Matching Pursuit decoder.

This module only *draws* problem instances (a dictionary Psi with unit
columns, K-sparse signals x and their encodings y = Psi x, Sec. 2 Eqs. 2-4).
It holds none of the decoder's arithmetic, so both the FP64 oracle tests and
the CUDA-path tests take their inputs from here without sharing any of the
method's code.

Storage convention (used by every consumer): the dictionary is returned
**atom-major**, an ``(M, N)`` float32 C-contiguous array whose row ``m`` is
the column psi_m of the paper's N x M matrix (Eq. 3).

Recipes (numpy PCG64 via ``default_rng([seed, stream])``):

* Gaussian dictionary: i.i.d. N(0,1) entries drawn directly in atom-major
  order, each atom normalised to unit L2 norm in FP64 (Eq. 4), then rounded
  to FP32.
* Bernoulli dictionary (Eq. 13): entries +-1/sqrt(N) with probability 1/2,
  sign(0) taken as +1.  For N a power of 4 the stored FP32 atoms have unit
  norm exactly.
* Signals: K distinct support indices drawn uniformly without replacement;
  values either sign*U[1,2] ("pm12") or N(0,1) with |x| < 0.5 clamped up to
  sign*0.5 ("normal_clamped"), or U[-1,1] ("uniform11", the paper's Sec. 3
  experiment).
* Encoding: y = Psi x computed in FP64 from the FP32-stored atoms, then
  rounded to FP32, so (Psi_fp32, y_fp32) is the instance both sides solve.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Named workloads (sizes of the paper-derived configurations)
# --------------------------------------------------------------------------

WORKLOADS = {
    # single-signal FP32 decode, dictionary fits in on-chip memory
    "plain_fp32_N256_M1024_K16": dict(
        kind="plain", N=256, M=1024, K=16, eps=1e-6, T=20000, values="pm12"),
    # single-signal FP32 decode, 256 MiB dictionary streamed from HBM
    "plain_fp32_N4096_M16384_K256": dict(
        kind="plain", N=4096, M=16384, K=256, eps=1e-5, T=10000, values="pm12"),
    # 1024 signals sharing one dictionary, BF16 correlations
    "batched_bf16_N2048_M8192_B1024": dict(
        kind="batched", N=2048, M=8192, B=1024, Kmin=8, Kmax=128, eps=1e-5,
        T=10000, values="pm12", prec="bf16"),
    # 256 signals, FP8-E4M3 per-column-scaled correlations
    "batched_fp8_N8192_M32768_B256": dict(
        kind="batched", N=8192, M=32768, B=256, Kmin=64, Kmax=512, eps=1e-4,
        T=10000, values="normal_clamped", prec="fp8"),
    # served mix over four resident dictionaries
    "served_4dict_poisson2000": dict(
        kind="served", dicts=[(512, 2048), (1024, 4096), (2048, 8192), (4096, 16384)],
        rate=2000.0, duration=60.0, eps=1e-5, T=10000, values="pm12"),
}


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


# --------------------------------------------------------------------------
# Dictionaries
# --------------------------------------------------------------------------

def gaussian_dictionary(N: int, M: int, seed: int = 0) -> np.ndarray:
    """Atom-major (M, N) float32 dictionary with unit-norm atoms (Eq. 4)."""
    g = _rng(seed, 0)
    P = g.standard_normal((M, N))
    P /= np.sqrt(np.einsum("mn,mn->m", P, P))[:, None]
    return np.ascontiguousarray(P, dtype=np.float32)


def bernoulli_dictionary(N: int, M: int, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """Atom-major (M, N) dictionary, entries +-1/sqrt(N) (Eq. 13), stored in
    ``dtype`` (float32, or float64 for the double-precision runs; the signs
    do not depend on it)."""
    g = _rng(seed, 0)
    s = np.where(g.random((M, N)) < 0.5, -1.0, 1.0)
    return np.ascontiguousarray(s / math.sqrt(N), dtype=dtype)


def orthonormal_dictionary(N: int, seed: int = 0) -> np.ndarray:
    """Atom-major (N, N) float64 orthonormal dictionary (QR of a Gaussian)."""
    g = _rng(seed, 0)
    Q, R = np.linalg.qr(g.standard_normal((N, N)))
    Q = Q * np.sign(np.diag(R))[None, :]
    return np.ascontiguousarray(Q.T)          # rows = columns of Q


# --------------------------------------------------------------------------
# Signals
# --------------------------------------------------------------------------

def sparse_signal(M: int, K: int, g: np.random.Generator, values: str = "pm12"):
    """Return (x float64 dense (M,), support int64 sorted)."""
    K = int(min(K, M))
    supp = np.sort(g.choice(M, size=K, replace=False)).astype(np.int64)
    x = np.zeros(M, dtype=np.float64)
    if values == "pm12":
        x[supp] = g.choice([-1.0, 1.0], size=K) * g.uniform(1.0, 2.0, size=K)
    elif values == "normal_clamped":
        v = g.standard_normal(K)
        small = np.abs(v) < 0.5
        v[small] = np.where(v[small] >= 0, 0.5, -0.5)
        x[supp] = v
    elif values == "uniform11":
        x[supp] = g.uniform(-1.0, 1.0, size=K)
    else:
        raise ValueError(f"unknown value distribution {values!r}")
    return x, supp


def encode(psi_atoms: np.ndarray, x: np.ndarray, dtype=np.float32) -> np.ndarray:
    """y = Psi x (Eq. 2) in FP64 from the stored atoms, rounded to ``dtype``."""
    nz = np.nonzero(x)[0]
    P = psi_atoms[nz].astype(np.float64)
    y = x[nz] @ P if nz.size else np.zeros(psi_atoms.shape[1])
    return y.astype(dtype)


@dataclass
class Problem:
    psi: np.ndarray                  # (M, N) float32 atom-major
    y: np.ndarray                    # (B, N) float32 (B=1 for a single signal)
    x_true: np.ndarray               # (B, M) float64
    supports: list = field(default_factory=list)
    eps: float = 1e-5
    T: int = 10000

    @property
    def N(self):
        return self.psi.shape[1]

    @property
    def M(self):
        return self.psi.shape[0]

    @property
    def B(self):
        return self.y.shape[0]


def make_plain(N: int, M: int, K: int, seed: int = 0, eps: float = 1e-5,
               T: int = 10000, values: str = "pm12", dictionary: str = "gaussian",
               psi: np.ndarray | None = None) -> Problem:
    """One K-sparse signal encoded with a fresh (or given) dictionary."""
    if psi is None:
        psi = (gaussian_dictionary if dictionary == "gaussian" else bernoulli_dictionary)(N, M, seed)
    x, supp = sparse_signal(M, K, _rng(seed, 1), values)
    y = encode(psi, x)
    return Problem(psi, y[None, :], x[None, :], [supp], eps, T)


def make_batched(N: int, M: int, B: int, Kmin: int, Kmax: int, seed: int = 0,
                 eps: float = 1e-5, T: int = 10000, values: str = "pm12",
                 psi: np.ndarray | None = None) -> Problem:
    """B signals sharing one dictionary, K_b ~ U{Kmin..Kmax} per signal."""
    if psi is None:
        psi = gaussian_dictionary(N, M, seed)
    g = _rng(seed, 2)
    Ks = g.integers(Kmin, Kmax + 1, size=B)
    Y = np.empty((B, N), dtype=np.float32)
    X = np.zeros((B, M), dtype=np.float64)
    supps = []
    for b in range(B):
        x, s = sparse_signal(M, int(Ks[b]), g, values)
        X[b] = x
        Y[b] = encode(psi, x)
        supps.append(s)
    return Problem(psi, Y, X, supps, eps, T)


def make_workload(name: str, seed: int = 0, B: int | None = None) -> Problem:
    """Instance of a named workload (``B`` may shrink a batched one)."""
    w = WORKLOADS[name]
    if w["kind"] == "plain":
        return make_plain(w["N"], w["M"], w["K"], seed, w["eps"], w["T"], w["values"])
    if w["kind"] == "batched":
        return make_batched(w["N"], w["M"], B or w["B"], w["Kmin"], w["Kmax"], seed,
                            w["eps"], w["T"], w["values"])
    raise ValueError(f"{name} is not a single-dictionary workload")


def paper_timing_problem(M: int, seed: int = 0, fp64: bool = False) -> Problem:
    """Sec. 4 timing sweep instance: N=floor(M/2), K=floor(0.07M), Bernoulli
    dictionary, U[-1,1] values, T=N, eps=1e-7.  ``fp64``: dictionary and y
    kept in FP64 (the double-precision run; same signs and signal)."""
    N, K = M // 2, int(0.07 * M)
    if not fp64:
        return make_plain(N, M, K, seed, 1e-7, N, "uniform11", "bernoulli")
    psi = bernoulli_dictionary(N, M, seed, np.float64)
    x, supp = sparse_signal(M, K, _rng(seed, 1), "uniform11")
    return Problem(psi, encode(psi, x, np.float64)[None, :], x[None, :], [supp], 1e-7, N)


PHASE_M = 1000
PHASE_GRID = tuple(round(0.05 * i, 2) for i in range(1, 21))     # sigma and rho: 0.05 .. 1.00


def phase_diagram_batch(rho: float, sigmas, trials: int, M: int = PHASE_M, seed: int = 0) -> Problem:
    """Sec. 3's phase-diagram experiment at one rho = N/M: a Bernoulli
    dictionary (Eq. 13) with N = round(rho M) rows, and ``trials`` signals
    for each sigma = K/M (K = max(1, round(sigma M)) nonzeros with U[-1,1]
    values), sigma-major; eps = 1e-7 and T = N as in the paper's run.  The
    batch shares the dictionary, so one batched decode covers a column of
    the diagram."""
    N = max(1, int(round(rho * M)))
    psi = bernoulli_dictionary(N, M, seed=1000 * seed + N)
    g = _rng(seed, 10000 + N)
    Y, X, supps = [], [], []
    for sg in sigmas:
        K = max(1, int(round(sg * M)))
        for _ in range(trials):
            x, supp = sparse_signal(M, K, g, "uniform11")
            X.append(x)
            Y.append(encode(psi, x))
            supps.append(supp)
    return Problem(psi, np.stack(Y), np.stack(X), supps, 1e-7, N)


def poisson_arrivals(rate: float, duration: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    g = _rng(seed, 3)
    n = int(rate * duration * 1.2 + 100)
    t = np.cumsum(g.exponential(1.0 / rate, size=n))
    return t[t < duration]


def served_requests(dicts, rate: float, duration: float, seed: int = 0):
    """(arrival_s, dict_index, K) per request: dictionary uniform over
    ``dicts`` and K ~ U{4..N/16}."""
    arr = poisson_arrivals(rate, duration, seed)
    g = _rng(seed, 4)
    d = g.integers(0, len(dicts), size=arr.size)
    K = np.array([g.integers(4, dicts[i][0] // 16 + 1) for i in d], dtype=np.int64)
    return arr, d, K
