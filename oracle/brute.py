"""Oracle: the full QUAPI path sum enumerated path by path (tiny N only).

TEST INFRASTRUCTURE (see oracle/__init__.py): never imported by the product.

Eq. quapi_red_rho written out: every forward/backward sequence of points
q_0 .. q_N contributes

  rho0[s+_0, s-_0] * prod_{j=1..N} U[s+_j, s+_{j-1}] conj(U[s-_j, s-_{j-1}])
                    * exp(-sum_{k=1..N} sum_{k'=1..k} (q+_k - q-_k)
                                   (eta_{k-k'} q+_{k'} - conj(eta_{k-k'}) q-_{k'}))

to <s+_N| rho(N dt) |s-_N>, with eta_d = 0 for d >= Delta k_max and point 0
carrying no box (reading R1 of oracle/iquapi.py).  No iteration, no window,
no merging: an independent formulation used to pin oracle/iquapi.py in the
unmasked, unfiltered case, where the pre-merge is exact.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg


def rho_by_enumeration(M: int, q, hs, dt: float, eta, dkmax: int, rho0, N: int) -> np.ndarray:
    q = np.asarray(q, dtype=np.float64)
    eta = np.asarray(eta, dtype=np.complex128)
    rho0 = np.asarray(rho0, dtype=np.complex128)
    U = scipy.linalg.expm(-1j * np.asarray(hs, dtype=np.complex128) * dt)
    # eta_{k,k'} for k, k' in 1..N (lower triangle incl. diagonal), truncated
    E = np.zeros((N + 1, N + 1), dtype=np.complex128)
    for k in range(1, N + 1):
        for kp in range(1, k + 1):
            d = k - kp
            if d < dkmax:
                E[k, kp] = eta[d]
    rho = np.zeros((M, M), dtype=np.complex128)
    if N == 0:
        return rho0.copy()
    # all sequences (s_0 .. s_N) for one branch
    seqs = np.array(list(itertools.product(range(M), repeat=N + 1)), dtype=np.int64)
    # amplitude factors of one branch: forward prod U[s_j, s_{j-1}], backward conj
    fwd = np.ones(len(seqs), dtype=np.complex128)
    for j in range(1, N + 1):
        fwd *= U[seqs[:, j], seqs[:, j - 1]]
    bwd = np.conj(fwd)
    qs = q[seqs]                                   # (n, N+1)
    for i in range(len(seqs)):                     # forward branch
        a0 = seqs[i, 0]
        qp = qs[i]
        for jb in range(len(seqs)):                # backward branch
            b0 = seqs[jb, 0]
            if rho0[a0, b0] == 0:
                continue
            qm = qs[jb]
            phi = 0.0 + 0.0j
            for k in range(1, N + 1):
                dq = qp[k] - qm[k]
                if dq == 0.0:
                    continue
                acc = 0.0 + 0.0j
                for kp in range(1, k + 1):
                    acc += E[k, kp] * qp[kp] - np.conj(E[k, kp]) * qm[kp]
                phi += dq * acc
            rho[seqs[i, N], seqs[jb, N]] += rho0[a0, b0] * fwd[i] * bwd[jb] * np.exp(-phi)
    return rho


def rho_by_enumeration_symmetric(M: int, q, hs, dt: float, Qh, dkmax: int, rho0, N: int) -> np.ndarray:
    """The same path sum with the symmetric Trotter splitting (Sec. 2, Eq.
    quapi_red_rho and Eq. inf_fun from point 0 to point N): point k holds the
    bath over an interval centred on k dt, point 0 over [0, dt/2] and point N
    over [N dt - dt/2, N dt].  The coefficient of two points is the double
    integral of the bath correlation over their intervals, written with
    Q(t) (the double integral from 0) at the intervals' ends:
        later interval [a1, a2], earlier [b1, b2]:  Q(a2-b1) - Q(a2-b2) - Q(a1-b1) + Q(a1-b2),
        one interval of length L with itself:       Q(L),
    given here as Qh[j] = Q(j dt / 2); zero for points dkmax or more steps
    apart.  Intervals are handled in units of dt/2."""
    q = np.asarray(q, dtype=np.float64)
    Qh = np.asarray(Qh, dtype=np.complex128)
    rho0 = np.asarray(rho0, dtype=np.complex128)
    if N == 0:
        return rho0.copy()
    U = scipy.linalg.expm(-1j * np.asarray(hs, dtype=np.complex128) * dt)

    def interval(k):
        if k == 0:
            return (0, 1)
        if k == N:
            return (2 * N - 1, 2 * N)
        return (2 * k - 1, 2 * k + 1)

    E = np.zeros((N + 1, N + 1), dtype=np.complex128)
    for k in range(N + 1):
        a1, a2 = interval(k)
        for kp in range(k + 1):
            if k - kp >= dkmax:
                continue
            if kp == k:
                E[k, k] = Qh[a2 - a1]
            else:
                b1, b2 = interval(kp)
                E[k, kp] = Qh[a2 - b1] - Qh[a2 - b2] - Qh[a1 - b1] + Qh[a1 - b2]
    seqs = np.array(list(itertools.product(range(M), repeat=N + 1)), dtype=np.int64)
    fwd = np.ones(len(seqs), dtype=np.complex128)
    for j in range(1, N + 1):
        fwd *= U[seqs[:, j], seqs[:, j - 1]]
    qs = q[seqs]
    rho = np.zeros((M, M), dtype=np.complex128)
    for i in range(len(seqs)):
        qp = qs[i]
        for jb in range(len(seqs)):
            if rho0[seqs[i, 0], seqs[jb, 0]] == 0:
                continue
            qm = qs[jb]
            phi = 0.0 + 0.0j
            for k in range(N + 1):
                dq = qp[k] - qm[k]
                if dq == 0.0:
                    continue
                acc = 0.0 + 0.0j
                for kp in range(k + 1):
                    acc += E[k, kp] * qp[kp] - np.conj(E[k, kp]) * qm[kp]
                phi += dq * acc
            rho[seqs[i, N], seqs[jb, N]] += rho0[seqs[i, 0], seqs[jb, 0]] * fwd[i] * np.conj(fwd[jb]) * np.exp(-phi)
    return rho
