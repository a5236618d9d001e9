"""Brute-force checks for tiny Matching Pursuit instances — TEST
INFRASTRUCTURE ONLY (imported by ``tests/`` alone).

Everything here is written with explicit Python loops and no BLAS call, so
it is independent of how ``mp_oracle`` lays out its matrix products:

* ``mp_loops``  — the iteration of Sec. 3 (Eqs. 8-12) with every inner
  product an explicit sum and the argmax a left-to-right scan that keeps
  the first maximiser (the smallest-index rule of Sec. 4).
* ``l0_supports`` — the l0 problem of Eq. 6 by enumeration: every support
  of size 1, 2, ... is tried with a least-squares fit, and the smallest
  size that reproduces y is returned with all supports of that size.
"""
from __future__ import annotations

import itertools

import numpy as np


def _dot(u, v):
    s = 0.0
    for a, b in zip(u, v):
        s += a * b
    return s


def mp_loops(psi_atoms, y, eps, T):
    """Eqs. 8-12 with explicit loops; psi_atoms[m] is the atom psi_m."""
    P = [[float(v) for v in row] for row in psi_atoms]
    r = [float(v) for v in y]
    M = len(P)
    x = [0.0] * M
    e0 = _dot(r, r)
    thr2 = float(eps) * float(eps) * e0
    e = e0
    t = 0
    atoms, coefs, energies = [], [], []
    while e > thr2 and t < T:
        best_i, best_a, best_c = 0, -1.0, 0.0
        for m in range(M):
            c = _dot(P[m], r)
            if abs(c) > best_a:           # strict: keeps the first maximiser
                best_i, best_a, best_c = m, abs(c), c
        x[best_i] += best_c
        r = [rn - best_c * pn for rn, pn in zip(r, P[best_i])]
        e = _dot(r, r)
        t += 1
        atoms.append(best_i)
        coefs.append(best_c)
        energies.append(e)
    return dict(x=np.array(x), r=np.array(r), iters=t, atoms=atoms,
                coefs=coefs, energies=energies, e0=e0)


def l0_supports(psi_atoms, y, kmax, tol=1e-9):
    """Smallest k <= kmax with some size-k support S such that y lies in
    span{psi_m : m in S} (Eq. 6); returns (k, [supports])."""
    P = np.asarray(psi_atoms, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ny = float(np.sqrt(_dot(y, y)))
    if ny == 0.0:
        return 0, [()]
    M = P.shape[0]
    for k in range(1, kmax + 1):
        hits = []
        for S in itertools.combinations(range(M), k):
            A = P[list(S)].T                        # N x k
            coef, *_ = np.linalg.lstsq(A, y, rcond=None)
            res = y - A @ coef
            if np.sqrt(_dot(res, res)) <= tol * ny:
                hits.append(S)
        if hits:
            return k, hits
    return None, []
