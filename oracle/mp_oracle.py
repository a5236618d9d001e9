"""FP64 CPU oracle for Matching Pursuit — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this module.  The product path (the CUDA library and
its Python binding) never calls it and shares no code with it.

What it computes (Andrecut, "Fast GPU Implementation of Sparse Signal
Recovery from Random Projections", Sec. 3, Eqs. 8-12):

    t <- 0, x~ <- 0, r <- y                                   (Eq. 8)
    while ||r||_2 > eps ||y||_2 and t < T:
        i  <- argmax_i |<r, psi_i>|                           (Eq. 9)
        x~_i <- x~_i + <r, psi_i>                             (Eq. 10)
        r  <- r - <r, psi_i> psi_i                            (Eq. 11)
        t  <- t + 1                                           (Eq. 12)
    return x~

Readings of the paper taken here (each is listed with its reason in the
design notes of the repository):

* Indices are 0-based (Sec. 2 numbers atoms 0..M-1); Eq. 9's {1..M} is the
  same set shifted.
* Ties in |<r, psi_i>| go to the smallest index, the i?amax rule the paper
  states for its argmax kernel (Sec. 4).
* ||r|| is recomputed from r every iteration (the paper calls nrm2 each
  pass, Sec. 4); the loop test is evaluated before every iteration, in the
  squared form ``e > eps^2 * e0`` with e = <r, r> and e0 = <y, y> in FP64.
  In exact arithmetic it is the same test as Eq. 8's loop condition.
* The threshold is eps*||y|| as the pseudocode of Sec. 3 states (the
  printed listings take sqrt(eps*||y||); the pseudocode is followed).
* An atom may be selected again; x~ accumulates.

Precision: the dictionary and y are widened to FP64 on entry (exact for the
FP32 values the GPU path stores), and every step runs in FP64.
"""
from __future__ import annotations

import numpy as np

STOP_CONVERGED = 0      # ||r|| <= eps ||y||
STOP_MAX_ITERS = 1      # t reached T
STOP_ZERO_Y = 2         # y == 0: nothing to decode


def mp(psi_atoms, y, eps, T, record=True):
    """Run Matching Pursuit in FP64.

    psi_atoms : (M, N) array, row m is the atom psi_m (unit L2 norm, Eq. 4).
    y         : (N,) measurement vector (Eq. 2).
    eps, T    : stopping parameters of Eq. 8's loop.

    Returns a dict with the solution ``x`` (M,), the final residual ``r``,
    the iteration count ``iters``, ``stop_reason``, and, if ``record``, the
    per-step ``atoms``, ``coefs`` (the <r, psi_i> added in Eq. 10),
    ``energies`` (<r, r> after each step) and ``gaps`` (relative gap between
    the largest and second-largest |<r, psi_m>| at each step).
    """
    P = np.array(psi_atoms, dtype=np.float64, copy=True)
    r = np.array(y, dtype=np.float64, copy=True).reshape(-1)
    M, N = P.shape
    assert r.shape == (N,), "y must have one entry per dictionary row"
    x = np.zeros(M, dtype=np.float64)

    e0 = float(np.dot(r, r))                       # ||y||^2
    thr2 = float(eps) * float(eps) * e0            # (eps ||y||)^2
    e = e0
    t = 0
    atoms, coefs, energies, gaps = [], [], [], []
    while e > thr2 and t < T:                      # loop test of Eq. 8
        c = P @ r                                  # <r, psi_m> for every m (Eq. 9)
        a = np.abs(c)
        i = int(np.argmax(a))                      # first maximiser = smallest index
        ci = float(c[i])
        x[i] += ci                                 # Eq. 10
        r -= ci * P[i]                             # Eq. 11
        e = float(np.dot(r, r))                    # ||r||^2 recomputed from r
        t += 1                                     # Eq. 12
        if record:
            atoms.append(i)
            coefs.append(ci)
            energies.append(e)
            if M > 1:
                second = float(np.partition(a, M - 2)[M - 2])
                gaps.append((float(a[i]) - second) / float(a[i]) if a[i] > 0 else 0.0)
            else:
                gaps.append(1.0)

    if e0 == 0.0:
        reason = STOP_ZERO_Y
    elif e <= thr2:
        reason = STOP_CONVERGED
    else:
        reason = STOP_MAX_ITERS
    out = dict(x=x, r=r, iters=t, stop_reason=reason, e0=e0, e=e,
               rel_residual=(np.sqrt(e / e0) if e0 > 0 else 0.0))
    if record:
        out.update(atoms=np.array(atoms, dtype=np.int64),
                   coefs=np.array(coefs, dtype=np.float64),
                   energies=np.array(energies, dtype=np.float64),
                   gaps=np.array(gaps, dtype=np.float64))
    return out


def follow(psi_atoms, y, atoms):
    """Replay a given atom sequence in FP64 (Eqs. 9-11 with i imposed).

    At each step the coefficient is the FP64 <r, psi_i> of the imposed atom,
    and the returned ``ratio[k]`` is |<r, psi_{atoms[k]}>| / max_m |<r, psi_m>|
    before step k: 1.0 where the imposed atom is an MP choice.  ``cmax[k]``
    and ``rnorm[k]`` are max_m |<r, psi_m>| and ||r|| before step k.
    Returns dict(ratio, cmax, rnorm, x, r).
    """
    P = np.array(psi_atoms, dtype=np.float64, copy=True)
    r = np.array(y, dtype=np.float64, copy=True).reshape(-1)
    x = np.zeros(P.shape[0], dtype=np.float64)
    ratio = np.empty(len(atoms), dtype=np.float64)
    cmaxs = np.empty(len(atoms), dtype=np.float64)
    rnorm = np.empty(len(atoms), dtype=np.float64)
    for k, i in enumerate(np.asarray(atoms, dtype=np.int64)):
        c = P @ r
        cmax = float(np.max(np.abs(c)))
        ratio[k] = abs(float(c[i])) / cmax if cmax > 0 else 1.0
        cmaxs[k] = cmax
        rnorm[k] = float(np.sqrt(np.dot(r, r)))
        x[i] += float(c[i])
        r -= float(c[i]) * P[i]
    return dict(ratio=ratio, cmax=cmaxs, rnorm=rnorm, x=x, r=r)


def reconstruction_error(x_rec, x_true):
    """E(sigma, rho) of Eq. 14, in percent."""
    x_rec = np.asarray(x_rec, dtype=np.float64)
    x_true = np.asarray(x_true, dtype=np.float64)
    return float(np.sum((x_rec - x_true) ** 2) / np.sum(x_true ** 2) * 100.0)


def support_score(x_rec, support):
    """|top-K(|x_rec|) intersect supp(x)| / K with K = |supp(x)|."""
    support = np.asarray(support, dtype=np.int64)
    K = support.size
    if K == 0:
        return 1.0
    top = np.argsort(-np.abs(np.asarray(x_rec)), kind="stable")[:K]
    return len(set(top.tolist()) & set(support.tolist())) / K
