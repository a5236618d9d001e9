"""Orthogonal Matching Pursuit in FP64 -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs
import this module; the product path never does.

The paper closes (Sec. 5) by naming Orthogonal Matching Pursuit as the next
method to implement on the GPU.  Its definition (Pati, Rezaiifar and
Krishnaprasad, 1993) keeps MP's selection and replaces MP's one-coefficient
update by a least-squares fit on every atom selected so far:

  1. c = Psi^T r; i = the smallest index maximising |c_i|   (Eq. 9, Sec. 4 ties)
  2. S <- S + {i}
  3. x_S = argmin_z ||y - Psi_S z||_2                     (replaces Eq. 10)
  4. r = y - Psi_S x_S                                     (replaces Eq. 11)
  5. stop when ||r|| <= eps ||y|| (squared, before each step) or t = T.

r is then orthogonal to every selected atom, so no atom is selected twice
while the selected atoms are independent.  One more stop applies: when the
selected atom lies in the span of S (its component orthogonal to span(S)
has norm <= ``rank_tol``, e.g. after N independent atoms in R^N), the fit
cannot grow and the run stops with ``STOP_RANK``.

Written from the definition above with numpy's least squares as the only
library step; no blocking or incremental factorisation.
"""
import numpy as np

STOP_CONVERGED = 0
STOP_MAX_ITERS = 1
STOP_ZERO_Y = 2
STOP_RANK = 3


def omp(psi_atoms, y, eps, T, rank_tol=1e-9, record=True):
    """Run OMP in FP64.  Same arguments and result keys as ``mp_oracle.mp``
    (``coefs`` holds <r, psi_i> at selection); ``x`` is the least-squares
    solution on the selected atoms."""
    P = np.array(psi_atoms, dtype=np.float64, copy=True)
    y = np.array(y, dtype=np.float64, copy=True).reshape(-1)
    M, N = P.shape
    assert y.shape == (N,)
    r = y.copy()
    x = np.zeros(M, dtype=np.float64)
    S = []
    xs = np.zeros(0)
    e0 = float(np.dot(y, y))
    thr2 = float(eps) * float(eps) * e0
    e = e0
    t = 0
    reason = None
    atoms, coefs, energies, gaps = [], [], [], []
    while e > thr2 and t < T:
        c = P @ r                                   # step 1
        a = np.abs(c)
        i = int(np.argmax(a))
        if S:
            A = P[S].T
            z = np.linalg.lstsq(A, P[i], rcond=None)[0]
            if np.linalg.norm(P[i] - A @ z) <= rank_tol:
                reason = STOP_RANK
                break
        S.append(i)                                 # step 2
        A = P[S].T
        xs = np.linalg.lstsq(A, y, rcond=None)[0]   # step 3
        r = y - A @ xs                              # step 4
        e = float(np.dot(r, r))
        t += 1
        if record:
            atoms.append(i)
            coefs.append(float(c[i]))
            energies.append(e)
            if M > 1:
                second = float(np.partition(a, M - 2)[M - 2])
                gaps.append((float(a[i]) - second) / float(a[i]) if a[i] > 0 else 0.0)
            else:
                gaps.append(1.0)
    if S:
        x[S] = xs
    if reason is None:
        if e0 == 0.0:
            reason = STOP_ZERO_Y
        elif e <= thr2:
            reason = STOP_CONVERGED
        else:
            reason = STOP_MAX_ITERS
    out = dict(x=x, r=r, iters=t, stop_reason=reason, e0=e0, e=e,
               rel_residual=(np.sqrt(e / e0) if e0 > 0 else 0.0), support=np.array(S, dtype=np.int64))
    if record:
        out.update(atoms=np.array(atoms, dtype=np.int64), coefs=np.array(coefs, dtype=np.float64),
                   energies=np.array(energies, dtype=np.float64), gaps=np.array(gaps, dtype=np.float64))
    return out


def follow(psi_atoms, y, atoms):
    """Replay a given selection sequence with OMP's fit (steps 2-4 with i
    imposed).  ``ratio[k]`` = |<r, psi_{atoms[k]}>| / max_m |<r, psi_m>|
    before step k (1.0 where the imposed atom is an OMP choice); ``cmax``
    and ``rnorm`` as in ``mp_oracle.follow``; ``x``, ``r`` after the last step."""
    P = np.array(psi_atoms, dtype=np.float64, copy=True)
    y = np.array(y, dtype=np.float64, copy=True).reshape(-1)
    r = y.copy()
    S = []
    xs = np.zeros(0)
    n = len(atoms)
    ratio, cmaxs, rnorm = np.empty(n), np.empty(n), np.empty(n)
    for k, i in enumerate(np.asarray(atoms, dtype=np.int64)):
        c = P @ r
        cmax = float(np.max(np.abs(c)))
        ratio[k] = abs(float(c[i])) / cmax if cmax > 0 else 1.0
        cmaxs[k] = cmax
        rnorm[k] = float(np.sqrt(np.dot(r, r)))
        S.append(int(i))
        A = P[S].T
        xs = np.linalg.lstsq(A, y, rcond=None)[0]
        r = y - A @ xs
    x = np.zeros(P.shape[0])
    if S:
        np.add.at(x, S, xs)
    return dict(ratio=ratio, cmax=cmaxs, rnorm=rnorm, x=x, r=r)
