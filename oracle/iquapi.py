"""Oracle: plain FP64 iterative QUAPI with MACGIC pre-merging, mask and filter.

TEST INFRASTRUCTURE (see oracle/__init__.py): never imported by the product.

Definitions followed (paper sections and equations):
  * reduced density matrix as a path sum over forward/backward system
    points, Eq. quapi_red_rho, with the bare propagator of Eqs. SysP0/SysP,
    S(q_j, q_{j-1}) = U[s+_j, s+_{j-1}] * conj(U[s-_j, s-_{j-1}]),
    U = exp(-i H_S dt), and the influence functional of Eq. inf_fun with
    Toeplitz coefficients eta_{k,k'} = eta_{k-k'} cut at the memory length
    Delta k_max (Sec. 2, finite memory);
  * MACGIC coarse graining: paths identical on the mask are merged, keeping
    the path of largest weight and the summed weight (Sec. 2.1);
  * the pre-merging order of Sec. 3.1: at step t the stored set Omega(t-1)
    is merged on the mask shifted by one step (mask[i] -> mask[i] + 1 in the
    paper's footnote, i.e. window positions P' = {p - 1 : p in P, p >= 1}
    of the older set), then every merged entry is extended by the M^2 new
    (s+, s-) pairs (routine propagation(), Sec. 3.2), children below the
    filter threshold are dropped, and rho(t) is the sum of the surviving
    children by end point.

Readings where the paper is silent:
  R1 box convention: point k >= 1 carries the box ((k-1) dt, k dt]; point 0
     (the initial state) carries none, so it enters S but not the influence
     functional.  The newest point's influence is applied when it is created.
  R2 window: a stored path holds the newest min(t+1, Delta k_max) points;
     lags 0 .. Delta k_max - 1 enter the influence functional.
  R3 the pre-merge runs only once the stored window is full
     (t >= Delta k_max); before that nothing merges.  P' always holds
     position 0, whose point is needed by the bare propagator.
  R4 group sum = sum over all members; representative = the member of
     largest |amplitude|; weights equal to a relative 1e-12 count as equal
     and among equal weights the smaller packed key wins (the paper's
     concurrent insert leaves the choice among equal weights open).
  R5 filter: a child is kept when |amp|^2 >= theta^2, applied before rho.

The original post-merging order (Sec. 2.1, Scheme macgic; step_post) is the
comparison the paper makes: every stored path is extended with its own
history and the children are merged on the mask P itself after the step;
the peak intermediate set is M^2 times the merged one.

Packed key used for the tie-break order and for exporting paths: with
bs = max(1, ceil(log2 M)) bits per state and b = 2 bs bits per point, window
position p (0 = newest) occupies bits [b p, b p + b): s+ in the low bs bits,
s- in the high bs bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.linalg

TIE_REL = 1e-12


def short_time_propagator(hs: np.ndarray, dt: float) -> np.ndarray:
    """U = exp(-i H_S dt) (hbar = 1)."""
    return scipy.linalg.expm(-1j * np.asarray(hs, dtype=np.complex128) * dt)


def state_bits(M: int):
    bs = max(1, math.ceil(math.log2(M)))
    return bs, 2 * bs


def packed_keys(sp: np.ndarray, sm: np.ndarray, M: int) -> np.ndarray:
    """Packed uint64 key of each path (rows of sp/sm, column p = window position p)."""
    bs, b = state_bits(M)
    n, L = sp.shape
    key = np.zeros(n, dtype=np.uint64)
    for p in range(L):
        code = sp[:, p].astype(np.uint64) | (sm[:, p].astype(np.uint64) << np.uint64(bs))
        key |= code << np.uint64(b * p)
    return key


def premerge_positions(mask, dkmax: int):
    """P' = {p - 1 : p in P, p >= 1} together with position 0 (reading R3)."""
    P = sorted(set(int(p) for p in mask))
    return sorted(set([p - 1 for p in P if p >= 1] + [0]))


def check_mask(mask, dkmax: int):
    P = sorted(set(int(p) for p in mask))
    if not P or P[0] < 0 or P[-1] >= dkmax:
        raise ValueError("mask positions must lie in [0, dkmax)")
    if 0 not in P or (dkmax >= 2 and 1 not in P):
        raise ValueError("mask must contain positions 0 and 1")
    return P


@dataclass
class Paths:
    """Stored set Omega_vec(t): forward points sp, backward points sm (column 0 =
    newest), complex amplitudes amp."""
    sp: np.ndarray
    sm: np.ndarray
    amp: np.ndarray


@dataclass
class StepStats:
    t: int
    groups: int          # entries after the pre-merge (= parents of this step)
    extended: int        # children generated, groups * M^2
    kept: int            # children surviving the filter
    near_tie: int        # group decisions within 1e-13 of the tie window edge
    near_theta: int      # children within 2e-12 (relative, on |amp|^2) of theta^2


@dataclass
class Result:
    rho: np.ndarray                      # (steps + 1, M, M)
    paths: Paths
    stats: List[StepStats] = field(default_factory=list)


def initial_paths(rho0: np.ndarray, q=None, ep: Optional[EndPoints] = None) -> Paths:
    """One path per nonzero element of rho(0); with the symmetric splitting
    each carries point 0's half-interval self factor."""
    a, b = np.nonzero(rho0)
    amp = rho0[a, b].astype(np.complex128)
    if ep is not None:
        q = np.asarray(q, dtype=np.float64)
        amp = amp * np.exp(-(q[a] - q[b]) * (ep.eta00 * q[a] - np.conj(ep.eta00) * q[b]))
    return Paths(sp=a.reshape(-1, 1).astype(np.int64),
                 sm=b.reshape(-1, 1).astype(np.int64),
                 amp=amp)


def premerge(paths: Paths, Pp, M: int):
    """Merge paths identical on the window positions Pp.

    Returns (rep_sp, rep_sm, S, near_tie): the representative path of each
    group (largest |amp|, reading R4) and the summed amplitude S.  Keys
    wider than 64 bits (b * window > 64, e.g. M = 8 with 12 points) go
    through premerge_rows, which does not pack them."""
    if state_bits(M)[1] * paths.sp.shape[1] > 64:
        return premerge_rows(paths, Pp, M)
    cols = list(Pp)
    gkey = packed_keys(paths.sp[:, cols], paths.sm[:, cols], M)
    _, inv = np.unique(gkey, return_inverse=True)
    G = int(inv.max()) + 1 if inv.size else 0
    S = np.zeros(G, dtype=np.complex128)
    np.add.at(S, inv, paths.amp)
    w2 = paths.amp.real ** 2 + paths.amp.imag ** 2
    wmax = np.zeros(G)
    np.maximum.at(wmax, inv, w2)
    edge = (1.0 - TIE_REL) * wmax[inv]
    eligible = w2 >= edge
    near_tie = int(np.count_nonzero((np.abs(w2 - edge) <= 1e-13 * np.maximum(edge, 1e-300))
                                    & (w2 != wmax[inv])))
    key = packed_keys(paths.sp, paths.sm, M)
    best = np.full(G, np.iinfo(np.uint64).max, dtype=np.uint64)
    np.minimum.at(best, inv[eligible], key[eligible])
    is_rep = eligible & (key == best[inv])
    idx = np.nonzero(is_rep)[0]
    rep_of = np.empty(G, dtype=np.int64)
    rep_of[inv[idx]] = idx
    return paths.sp[rep_of], paths.sm[rep_of], S, near_tie


def premerge_rows(paths: Paths, Pp, M: int):
    """premerge without packed keys (any key width): groups are the distinct
    rows of the P' columns; the representative is the member of largest
    weight, ties (R4) to the member whose packed key would be smallest,
    i.e. the smallest in the order that compares the oldest position first
    and, within a position, the backward point before the forward one (the
    order of the packed key for any number of bits per point)."""
    cols = list(Pp)
    gk = np.concatenate([paths.sp[:, cols], paths.sm[:, cols]], axis=1)
    if gk.shape[0] == 0:
        return paths.sp[:0], paths.sm[:0], np.zeros(0, dtype=np.complex128), 0
    _, inv = np.unique(gk, axis=0, return_inverse=True)
    inv = np.asarray(inv).reshape(-1)
    G = int(inv.max()) + 1
    S = np.zeros(G, dtype=np.complex128)
    np.add.at(S, inv, paths.amp)
    w2 = paths.amp.real ** 2 + paths.amp.imag ** 2
    wmax = np.zeros(G)
    np.maximum.at(wmax, inv, w2)
    edge = (1.0 - TIE_REL) * wmax[inv]
    eligible = w2 >= edge
    near_tie = int(np.count_nonzero((np.abs(w2 - edge) <= 1e-13 * np.maximum(edge, 1e-300))
                                    & (w2 != wmax[inv])))
    idx = np.nonzero(eligible)[0]
    L = paths.sp.shape[1]
    keys = []   # least significant first (np.lexsort takes the last key as primary)
    for p in range(L):
        keys += [paths.sp[idx, p], paths.sm[idx, p]]
    order = idx[np.lexsort(tuple(keys) + (inv[idx],))]
    first = np.r_[True, inv[order][1:] != inv[order][:-1]]
    rep_of = np.empty(G, dtype=np.int64)
    rep_of[inv[order[first]]] = order[first]
    return paths.sp[rep_of], paths.sm[rep_of], S, near_tie


@dataclass
class EndPoints:
    """Coefficients of the symmetric Trotter splitting (Sec. 2, Eq.
    quapi_red_rho: "applying a symmetric Trotter splitting"; Eq. inf_fun
    sums from point 0 to point N).  Point k holds the bath over the interval
    centred on k dt: interior points a full interval, point 0 the half
    [0, dt/2] and the newest point N the half [N dt - dt/2, N dt].  With
    Qh[j] = Q(j dt / 2) (Q the double integral of the bath correlation,
    oracle/bath.py) and the memory cut at lags >= dkmax:
      eta00 = Q(dt/2)                     self term of a half interval
      eta0[k]  (k >= 1)                   interior point k with point 0
      etaE[d]  (d >= 1)                   the newest point with an interior point d back
      etaE0[N] (N >= 1)                   the newest point N with point 0
    Interior pairs keep the full-interval coefficients eta_d of the
    right-box reading (the same double integrals, shifted by dt/2)."""
    eta00: complex
    eta0: np.ndarray      # [dkmax], index k; eta0[0] unused
    etaE: np.ndarray      # [dkmax], index d; etaE[0] unused
    etaE0: np.ndarray     # [dkmax], index N; etaE0[0] unused


def end_points_from_Q(Qh, dkmax: int) -> EndPoints:
    """The symmetric splitting's end-point coefficients from Qh[j] = Q(j dt/2),
    j = 0 .. 2 dkmax (and more; Qh[0] = 0)."""
    Qh = np.asarray(Qh, dtype=np.complex128)
    eta0 = np.zeros(dkmax, dtype=np.complex128)
    etaE = np.zeros(dkmax, dtype=np.complex128)
    etaE0 = np.zeros(dkmax, dtype=np.complex128)
    for k in range(1, dkmax):
        eta0[k] = Qh[2 * k + 1] - Qh[2 * k] - Qh[2 * k - 1] + Qh[2 * k - 2]
        etaE[k] = Qh[2 * k + 1] - Qh[2 * k - 1] - Qh[2 * k] + Qh[2 * k - 2]
        etaE0[k] = Qh[2 * k] - 2.0 * Qh[2 * k - 1] + Qh[2 * k - 2]
    return EndPoints(eta00=complex(Qh[1]), eta0=eta0, etaE=etaE, etaE0=etaE0)


def step(paths: Paths, t: int, U, q, eta, dkmax: int, Pp, theta: float, M: int, ep: Optional[EndPoints] = None):
    """One propagation step t-1 -> t.  Returns (new paths, rho(t), stats).

    ep: the symmetric splitting's end points (None: the right-box reading
    R1).  The stored amplitudes then carry every factor with the newest
    point treated as interior (as it will be once later points exist) and
    point 0 with its half interval; rho(t) multiplies each surviving child
    by the difference between the newest point's end-point and interior
    factors."""
    if t >= dkmax:                                  # window full: pre-merge on P'
        rsp, rsm, S, near_tie = premerge(paths, Pp, M)
    else:                                           # nothing merges yet (R3)
        rsp, rsm, S, near_tie = paths.sp, paths.sm, paths.amp, 0
    G = S.size
    n_act = min(t, dkmax)
    # influence of the stored history on the new point: lags d = 1 .. n_act-1,
    # the point d steps back sits at window position d-1 of the parent
    H = np.zeros(G, dtype=np.complex128)
    for d in range(1, n_act):
        H += eta[d] * q[rsp[:, d - 1]] - np.conj(eta[d]) * q[rsm[:, d - 1]]
    if ep is not None:
        # symmetric splitting: point 0 (t steps back, position t-1 while the
        # window holds it) within memory; and the newest point's end-point
        # correction for rho(t)
        HE = np.zeros(G, dtype=np.complex128)
        for d in range(1, n_act):
            dE = ep.etaE[d] - eta[d]
            HE += dE * q[rsp[:, d - 1]] - np.conj(dE) * q[rsm[:, d - 1]]
        if t < dkmax:
            H += ep.eta0[t] * q[rsp[:, t - 1]] - np.conj(ep.eta0[t]) * q[rsm[:, t - 1]]
            dE0 = ep.etaE0[t] - ep.eta0[t]
            HE += dE0 * q[rsp[:, t - 1]] - np.conj(dE0) * q[rsm[:, t - 1]]
        dS = ep.eta00 - eta[0]           # the newest point's half interval against a full one
    L_child = min(t + 1, dkmax)
    rho = np.zeros((M, M), dtype=np.complex128)
    new_sp, new_sm, new_amp = [], [], []
    near_theta = 0
    th2 = theta * theta
    for a in range(M):
        for b in range(M):
            prop = U[a, rsp[:, 0]] * np.conj(U[b, rsm[:, 0]])
            phase = -(q[a] - q[b]) * (H + eta[0] * q[a] - np.conj(eta[0]) * q[b])
            child = S * prop * np.exp(phase)
            w2 = child.real ** 2 + child.imag ** 2
            keep = w2 >= th2
            if th2 > 0:
                near_theta += int(np.count_nonzero(np.abs(w2 - th2) <= 2e-12 * th2))
            if ep is None:
                rho[a, b] = child[keep].sum()
            else:
                corr = np.exp(-(q[a] - q[b]) * (HE + dS * q[a] - np.conj(dS) * q[b]))
                rho[a, b] = (child * corr)[keep].sum()
            k = int(np.count_nonzero(keep))
            col_a = np.full((k, 1), a, dtype=np.int64)
            col_b = np.full((k, 1), b, dtype=np.int64)
            new_sp.append(np.hstack([col_a, rsp[keep, :L_child - 1]]))
            new_sm.append(np.hstack([col_b, rsm[keep, :L_child - 1]]))
            new_amp.append(child[keep])
    out = Paths(sp=np.vstack(new_sp), sm=np.vstack(new_sm), amp=np.concatenate(new_amp))
    st = StepStats(t=t, groups=G, extended=G * M * M, kept=out.amp.size,
                   near_tie=near_tie, near_theta=near_theta)
    return out, rho, st


def merge_on(paths: Paths, positions, M: int):
    """Merge the paths identical on the given window positions: one entry per
    group, the member of largest |amp| (reading R4) with the summed
    amplitude.  Returns (merged Paths, near-tie count)."""
    rsp, rsm, S, near_tie = premerge(paths, positions, M)
    return Paths(sp=rsp, sm=rsm, amp=S), near_tie


def step_post(paths: Paths, t: int, U, q, eta, dkmax: int, P, theta: float, M: int):
    """One step t-1 -> t of the original post-merging order (Sec. 2.1, Scheme
    macgic): every stored path is extended by the M^2 new points with its
    own history (routine propagation()), children below the filter are
    dropped, rho(t) sums the survivors by end point, and the unmerged set
    Omega(t, unmerged) is then merged on the mask P itself (sorting() and
    merging()) once its window is full (t >= dkmax - 1; reading R3: no
    merging while the window fills).  Returns (merged paths, rho(t),
    stats): groups = paths extended, kept = children surviving the filter
    (the unmerged intermediate set), merged = stored paths after merging."""
    n_act = min(t, dkmax)
    # the own history of every stored path: lags d = 1 .. n_act-1
    H = np.zeros(paths.amp.size, dtype=np.complex128)
    for d in range(1, n_act):
        H += eta[d] * q[paths.sp[:, d - 1]] - np.conj(eta[d]) * q[paths.sm[:, d - 1]]
    L_child = min(t + 1, dkmax)
    rho = np.zeros((M, M), dtype=np.complex128)
    new_sp, new_sm, new_amp = [], [], []
    near_theta = 0
    th2 = theta * theta
    for a in range(M):
        for b in range(M):
            prop = U[a, paths.sp[:, 0]] * np.conj(U[b, paths.sm[:, 0]])
            phase = -(q[a] - q[b]) * (H + eta[0] * q[a] - np.conj(eta[0]) * q[b])
            child = paths.amp * prop * np.exp(phase)
            w2 = child.real ** 2 + child.imag ** 2
            keep = w2 >= th2
            if th2 > 0:
                near_theta += int(np.count_nonzero(np.abs(w2 - th2) <= 2e-12 * th2))
            rho[a, b] = child[keep].sum()
            k = int(np.count_nonzero(keep))
            new_sp.append(np.hstack([np.full((k, 1), a, dtype=np.int64), paths.sp[keep, :L_child - 1]]))
            new_sm.append(np.hstack([np.full((k, 1), b, dtype=np.int64), paths.sm[keep, :L_child - 1]]))
            new_amp.append(child[keep])
    unmerged = Paths(sp=np.vstack(new_sp), sm=np.vstack(new_sm), amp=np.concatenate(new_amp))
    near_tie = 0
    if L_child == dkmax and unmerged.amp.size:
        out, near_tie = merge_on(unmerged, sorted(P), M)
    else:
        out = unmerged
    st = StepStats(t=t, groups=paths.amp.size, extended=paths.amp.size * M * M, kept=unmerged.amp.size,
                   near_tie=near_tie, near_theta=near_theta)
    st.merged = out.amp.size
    return out, rho, st


def propagate(M: int, q, hs, dt: float, eta, dkmax: int, mask, theta: float,
              rho0, steps: int, keep_stats: bool = True, scheme: str = "pre", Qh=None) -> Result:
    """Run `steps` propagation steps from rho0; rho[t] for t = 0 .. steps.
    scheme "pre": the pre-merging order of Sec. 3.1 (step); "post": the
    original post-merging order of Sec. 2.1 (step_post).  Qh (Q at
    multiples of dt/2): the symmetric splitting's end points (pre-merging
    order only); None: the right-box reading R1."""
    q = np.asarray(q, dtype=np.float64)
    eta = np.asarray(eta, dtype=np.complex128)
    if eta.size < dkmax:
        raise ValueError("need dkmax influence coefficients")
    rho0 = np.asarray(rho0, dtype=np.complex128)
    P = check_mask(range(dkmax) if mask is None else mask, dkmax)
    Pp = premerge_positions(P, dkmax)
    U = short_time_propagator(hs, dt)
    ep = None if Qh is None else end_points_from_Q(Qh, dkmax)
    if ep is not None and scheme != "pre":
        raise ValueError("the symmetric splitting is given for the pre-merging order")
    paths = initial_paths(rho0, q, ep)
    rhos = [rho0.copy()]
    stats = []
    if scheme not in ("pre", "post"):
        raise ValueError("scheme must be 'pre' or 'post'")
    for t in range(1, steps + 1):
        if scheme == "pre":
            paths, rho, st = step(paths, t, U, q, eta, dkmax, Pp, theta, M, ep)
        else:
            paths, rho, st = step_post(paths, t, U, q, eta, dkmax, P, theta, M)
        rhos.append(rho)
        if keep_stats:
            stats.append(st)
    return Result(rho=np.array(rhos), paths=paths, stats=stats)


def propagate_workload(w, eta=None, steps: Optional[int] = None) -> Result:
    """Convenience: run a workloads.Workload (eta from oracle.bath unless given)."""
    if eta is None:
        from .bath import eta_coefficients
        eta = eta_coefficients(w.bath, w.dt, w.dkmax)
    return propagate(w.M, w.q, w.hs_array(), w.dt, eta, w.dkmax, w.mask, w.theta,
                     w.rho0_array(), w.steps if steps is None else steps)
