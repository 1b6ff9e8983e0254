"""Pins of the CPU oracle against results fixed by the mathematics.

Every check here compares the oracle with something other than itself:
closed forms of Q(t), closed forms of U, brute-force enumeration of the path
sum, Rabi oscillation at zero coupling, exact pure dephasing at zero
tunnelling, the Markov map at memory length 1 (with and without the filter,
whose rule and order the filtered map pins), a hand-made filter case, and
invariants (trace, Hermiticity).  The mutation tests at the end plant typical mistakes in a
copy of the oracle and check that at least one pin catches each.
"""
import math
import types

import numpy as np
import pytest
from scipy import special

import workloads as W
from oracle import bath as B
from oracle import brute, iquapi


# ---------------------------------------------------------------- closed forms

def ohmic_Q_closed(alpha, wc, beta, t):
    """Q(t) for J = (pi/2) alpha w e^{-w/wc}: Im part elementary, Re part from
    coth(x/2) = 1 + 2 sum e^{-n x}, the product summed through log-Gamma."""
    t = np.asarray(t, dtype=float)
    c = 1.0 / (beta * wc)
    x = t / beta
    series = 2.0 * special.loggamma(1.0 + c).real - 2.0 * special.loggamma(1.0 + c + 1j * x).real
    re = 0.5 * alpha * (0.5 * np.log1p((wc * t) ** 2) + series)
    im = -0.5 * alpha * (wc * t - np.arctan(wc * t))
    return re + 1j * im


def resonance_Q_closed(w0, gamma, lam, beta, t, nmat=400000):
    """Q(t) for the resonance of Eq. sharpSD (a damped-oscillator density),
    by residues: the two upper poles w = +-w~ + i gamma/2 and the Matsubara
    poles i nu_n of coth, then the double time integral term by term."""
    A = 2.0 * lam * gamma * w0 ** 2 / np.pi
    wt = np.sqrt(w0 ** 2 - gamma ** 2 / 4)
    wp = wt + 0.5j * gamma
    z = 1j * wp
    C = 1.0 / np.tanh(beta * wp / 2)
    n = np.arange(1, nmat + 1)
    nu = 2 * np.pi * n / beta
    D = (nu ** 2 + w0 ** 2) ** 2 - gamma ** 2 * nu ** 2
    out = []
    for tt in np.atleast_1d(t):
        I = (np.exp(z * tt) - 1 - z * tt) / z ** 2
        mats = np.sum((nu / D) * (np.expm1(-nu * tt) + nu * tt) / nu ** 2)
        out.append(A / (2 * gamma * wt) * ((C * I).real - 1j * I.imag) - (2 * A / beta) * mats)
    return np.array(out)


@pytest.mark.parametrize("alpha,wc,beta", [(0.1, 5.0, 5.0), (0.05, 5.0, 10.0),
                                           (2 / 16 / math.pi ** 2, 10.0, 5.0), (0.3, 2.0, 0.7),
                                           (0.1, 5.0, 100.0), (0.1, 5.0, 0.05), (0.1, 50.0, 5.0), (0.1, 0.5, 5.0)])
def test_ohmic_Q_matches_closed_form(alpha, wc, beta):
    ts = np.array([0.05, 0.25, 0.5, 1.3, 2.25, 4.2])
    bath = W.Bath(beta=beta, ohmic_alpha=alpha, ohmic_wc=wc)
    np.testing.assert_allclose(B.Q_of_t(bath, ts), ohmic_Q_closed(alpha, wc, beta, ts), rtol=0, atol=2e-14)


@pytest.mark.parametrize("w0,gamma,lam,beta", [(1.0, 0.05, 0.1, 10.0), (1.7, 0.3, 0.2, 2.0)])
def test_resonance_Q_matches_closed_form(w0, gamma, lam, beta):
    ts = np.array([0.1, 0.5, 1.0, 1.7])
    bath = W.Bath(beta=beta, res_w0=w0, res_gamma=gamma, res_lambda=lam)
    np.testing.assert_allclose(B.Q_of_t(bath, ts), resonance_Q_closed(w0, gamma, lam, beta, ts),
                               rtol=0, atol=1e-14)


def test_resonance_reorganisation_energy():
    from scipy import integrate
    bath = W.Bath(beta=1.0, res_w0=1.3, res_gamma=0.2, res_lambda=0.17)
    lam = integrate.quad(lambda w: B.spectral_density(bath, w) / w, 0, np.inf, points=None, limit=500)[0]
    assert abs(lam - 0.17) < 1e-9


def test_eta_is_box_integral_of_Q():
    """eta_0 = Q(dt) and sum over the triangle of box integrals equals Q(n dt):
    n eta_0 + sum_d (n-d) eta_d = Q(n dt) with Q from the closed form."""
    alpha, wc, beta, dt = 0.1, 5.0, 5.0, 0.25
    bath = W.Bath(beta=beta, ohmic_alpha=alpha, ohmic_wc=wc)
    eta = B.eta_coefficients(bath, dt, 10)
    for n in range(1, 11):
        tri = n * eta[0] + sum((n - d) * eta[d] for d in range(1, n))
        assert abs(tri - ohmic_Q_closed(alpha, wc, beta, n * dt)) < 1e-13


# ---------------------------------------------------------------- propagator

def test_propagator_two_level_closed_form():
    dt, delta = 0.37, 1.3
    hs = np.array([[0, delta / 2], [delta / 2, 0]], dtype=complex)
    U = iquapi.short_time_propagator(hs, dt)
    c, s = math.cos(delta * dt / 2), math.sin(delta * dt / 2)
    np.testing.assert_allclose(U, np.array([[c, -1j * s], [-1j * s, c]]), atol=1e-15)


def test_propagator_three_level_chain_closed_form():
    dt = 0.1
    hs = np.array(W.CHAIN3_STRUCTURED_DK12.hs, dtype=complex)
    r2 = math.sqrt(2.0)
    V = np.array([[0.5, 1 / r2, 0.5], [r2 / 2, 0.0, -r2 / 2], [0.5, -1 / r2, 0.5]])
    lam = np.array([r2, 0.0, -r2])
    Uc = V @ np.diag(np.exp(-1j * lam * dt)) @ V.T
    U = iquapi.short_time_propagator(hs, dt)
    np.testing.assert_allclose(U, Uc, atol=1e-15)
    np.testing.assert_allclose(U @ U.conj().T, np.eye(3), atol=1e-15)


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("M,dkmax,N,seed", [(2, 1, 5, 1), (2, 2, 5, 2), (2, 3, 6, 3), (2, 4, 5, 4),
                                            (2, 7, 5, 5), (3, 1, 3, 6), (3, 2, 4, 7), (3, 3, 4, 8)])
def test_iterative_equals_brute_force(M, dkmax, N, seed):
    c = W.random_case(seed, M, dkmax)
    rb = brute.rho_by_enumeration(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, c["rho0"], N)
    r = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, None, 0.0, c["rho0"], N)
    np.testing.assert_allclose(r.rho[N], rb, rtol=0, atol=2e-14)


# ---------------------------------------------------------------- special cases

@pytest.mark.parametrize("mask,dkmax", [(None, 6), ((0, 1, 2, 4), 6), ((0, 1), 5), ((0, 1, 2, 3, 4, 5, 7), 9)])
def test_rabi_at_zero_coupling(mask, dkmax):
    """eta = 0: <sigma_z>(t) = cos(Delta t), rho_updown = (i/2) sin(Delta t); the
    merge is exact here for any mask."""
    delta, dt, steps = 1.0, 0.25, 24
    hs = np.array([[0, delta / 2], [delta / 2, 0]], dtype=complex)
    r = iquapi.propagate(2, [1.0, -1.0], hs, dt, np.zeros(dkmax), dkmax, mask, 0.0,
                         np.array([[1, 0], [0, 0]], dtype=complex), steps)
    t = dt * np.arange(steps + 1)
    np.testing.assert_allclose((r.rho[:, 0, 0] - r.rho[:, 1, 1]).real, np.cos(delta * t), atol=1e-13)
    np.testing.assert_allclose(r.rho[:, 0, 1], 0.5j * np.sin(delta * t), atol=1e-13)


@pytest.mark.parametrize("dkmax,mask", [(6, None), (6, (0, 1, 3))])
def test_pure_dephasing_exact(dkmax, mask):
    """H_S = 0: rho_ab(t) = rho_ab(0) exp(-(q_a-q_b)(q_a Q - q_b Q*)) with Q the
    closed-form Q(t) up to t = dkmax dt, and the truncated triangle sum after."""
    alpha, wc, beta, dt, steps = 0.1, 5.0, 5.0, 0.25, 14
    bath = W.Bath(beta=beta, ohmic_alpha=alpha, ohmic_wc=wc)
    eta = B.eta_coefficients(bath, dt, dkmax)
    for M, q in [(2, np.array([1.0, -1.0])), (3, np.array([-1.0, 0.0, 1.0]))]:
        rho0 = np.full((M, M), 1.0 / M, dtype=complex)
        r = iquapi.propagate(M, q, np.zeros((M, M)), dt, eta, dkmax, mask, 0.0, rho0, steps)
        for n in range(steps + 1):
            if n <= dkmax:
                Q = ohmic_Q_closed(alpha, wc, beta, n * dt) if n else 0.0
            else:  # truncated memory: triangle of box integrals with lags < dkmax
                Q = n * eta[0] + sum((n - d) * eta[d] for d in range(1, dkmax))
            expect = rho0 * np.exp(-(q[:, None] - q[None, :]) * (q[:, None] * Q - q[None, :] * np.conj(Q)))
            np.testing.assert_allclose(r.rho[n], expect, atol=1e-13)


def test_markov_map_at_memory_one():
    """dkmax = 1: rho(t) = Phi^t rho0 with Phi the one-step map on coherences."""
    M = 3
    c = W.random_case(11, M, 1)
    U = iquapi.short_time_propagator(c["hs"], c["dt"])
    q, e0 = c["q"], c["eta"][0]
    Phi = np.zeros((M * M, M * M), dtype=complex)
    for a in range(M):
        for b in range(M):
            f = np.exp(-(q[a] - q[b]) * (e0 * q[a] - np.conj(e0) * q[b]))
            for ap in range(M):
                for bp in range(M):
                    Phi[a * M + b, ap * M + bp] = U[a, ap] * np.conj(U[b, bp]) * f
    r = iquapi.propagate(M, q, c["hs"], c["dt"], c["eta"], 1, None, 0.0, c["rho0"], 9)
    for n in range(10):
        np.testing.assert_allclose(r.rho[n].reshape(-1), np.linalg.matrix_power(Phi, n) @ c["rho0"].reshape(-1),
                                   atol=1e-14)


# ---------------------------------------------------------------- invariants

def _structured_case(M=2, dkmax=8):
    rng = np.random.default_rng(5)
    q = np.array([1.0, -1.0]) if M == 2 else np.array([-1.0, 0.0, 1.0])
    hs = W.random_hermitian(rng, M, 0.7)
    eta = W.random_eta(rng, dkmax, 0.08)
    rho0 = W.random_density_matrix(rng, M)
    return q, hs, eta, rho0


PREFIX_CASES = [   # (M, dkmax, k, extra mask positions): mask = {0 .. k-1} + extras, eta_d = 0 for d >= k
    (2, 8, 3, (5,)), (2, 8, 4, (6, 7)), (2, 7, 2, (4,)), (3, 6, 3, (5,)), (3, 5, 2, (3,)), (5, 4, 2, (3,)),
]


def prefix_case(M, dkmax, k, extras, cut, seed=None):
    """A random problem whose influence coefficients vanish from lag `cut`
    on, with the mask {0 .. k-1} plus the given older positions."""
    c = W.random_case(30 + dkmax + k if seed is None else seed, M, dkmax)
    eta = np.array(c["eta"], dtype=complex)
    eta[cut:] = 0.0
    return dict(c, eta=eta, mask=tuple(range(k)) + tuple(extras))


def prefix_cut(scheme, k):
    """Largest memory at which merging on the prefix mask {0 .. k-1} is exact.
    The pre-merge groups the parents on P' (Sec. 3.1), which drops parent
    position k - 1 before the children are formed, and that position meets
    the new point at lag k; the merge after extension (Sec. 2.1) groups the
    children on P, which drops child position k, first met at lag k + 1."""
    return k if scheme == "pre" else k + 1


@pytest.mark.parametrize("scheme", ["pre", "post"])
@pytest.mark.parametrize("M,dkmax,k,extras", PREFIX_CASES)
def test_masked_merge_exact_when_eta_ends_within_the_prefix(M, dkmax, k, extras, scheme):
    """Masked propagation with a nonzero bath, where the merge is exact: the
    positions a merge drops enter later influence factors (Eq. inf_fun)
    only through lags at or beyond the cut (prefix_cut), where eta vanishes,
    so summing a group's members loses nothing and the masked run on a
    window of dkmax points equals QUAPI with memory `cut` (Eq.
    quapi_red_rho), given by brute-force enumeration.  Groups have many
    members here (M^2 per dropped position), unlike the zero-coupling and
    pure-dephasing pins."""
    cut = prefix_cut(scheme, k)
    c = prefix_case(M, dkmax, k, extras, cut)
    n_brute = {2: 6, 3: 4, 5: 3}[M]
    steps = {2: 14, 3: 10, 5: 6}[M]
    r = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, c["mask"], 0.0, c["rho0"], steps,
                         scheme=scheme)
    rb = brute.rho_by_enumeration(M, c["q"], c["hs"], c["dt"], c["eta"][:cut], cut, c["rho0"], n_brute)
    np.testing.assert_allclose(r.rho[n_brute], rb, rtol=0, atol=2e-14)
    short = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"][:cut], cut, None, 0.0, c["rho0"], steps)
    np.testing.assert_allclose(r.rho, short.rho, rtol=0, atol=1e-14)
    # groups really merged members: fewer than the stored paths they came from
    if scheme == "pre":
        assert r.stats[-1].groups * M <= r.stats[-2].kept
    else:
        assert r.stats[-1].merged * M <= r.stats[-1].kept


@pytest.mark.parametrize("M,dkmax,k,extras", PREFIX_CASES)
def test_premerge_is_not_exact_one_lag_further(M, dkmax, k, extras):
    """The pre-merge on P' (the shifted mask) drops parent position k - 1,
    which meets the new point at lag k: with eta_k nonzero the masked run
    is an approximation of QUAPI with memory k + 1, while the merge after
    extension on P is still exact there.  A pre-merge on P itself (no
    shift) would be exact here as well."""
    c = prefix_case(M, dkmax, k, extras, k + 1)
    steps = {2: 14, 3: 10, 5: 6}[M]
    short = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"][:k + 1], k + 1, None, 0.0, c["rho0"], steps)
    pre = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, c["mask"], 0.0, c["rho0"], steps)
    post = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, c["mask"], 0.0, c["rho0"], steps,
                            scheme="post")
    assert np.abs(pre.rho - short.rho).max() > 1e-6
    assert np.abs(post.rho - short.rho).max() <= 1e-14


def _prefix_pins_pass(mod, scheme):
    """The two prefix-mask facts above on one case (mutation harnesses)."""
    M, dkmax, k, extras = 2, 7, 2, (4,)
    for cut in (k, k + 1):
        c = prefix_case(M, dkmax, k, extras, cut)
        r = mod.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, c["mask"], 0.0, c["rho0"], 10, scheme=scheme)
        short = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"][:cut], cut, None, 0.0, c["rho0"], 10)
        exact = np.abs(r.rho - short.rho).max() <= 1e-14
        if exact != (cut <= prefix_cut(scheme, k)):
            return False
    return True


@pytest.mark.parametrize("M,mask", [(2, (0, 1, 2, 5)), (2, (0, 1, 4, 6)), (3, (0, 1, 3))])
def test_trace_conserved_by_masked_merge(M, mask):
    q, hs, eta, rho0 = _structured_case(M, 8 if M == 2 else 5)
    dk = 8 if M == 2 else 5
    r = iquapi.propagate(M, q, hs, 0.2, eta, dk, mask, 0.0, rho0, 16)
    tr = np.trace(r.rho, axis1=1, axis2=2)
    np.testing.assert_allclose(tr, np.ones_like(tr), atol=1e-13)



@pytest.mark.parametrize("M,dkmax,steps", [(2, 8, 24), (3, 5, 12)])
@pytest.mark.parametrize("theta", [0.0, 1e-5])
def test_masked_result_converges_to_unmasked_as_the_mask_grows(M, dkmax, steps, theta):
    """Sec. 3.1: the mask trades accuracy for paths, and the result
    approaches the full iQUAPI one as Delta k_eff grows to Delta k_max.
    On these seeded structured cases, prefix masks {0 .. k-1}: the largest
    deviation from the unmasked run (same filter) falls with k (5 % slack
    per step), by more than fourfold from the smallest mask to the largest
    partial one (with a filter the different filter losses set a floor),
    and vanishes for the full window."""
    q, hs, eta, rho0 = _structured_case(M, dkmax)
    ref = iquapi.propagate(M, q, hs, 0.2, eta, dkmax, None, theta, rho0, steps).rho
    errs = [np.abs(iquapi.propagate(M, q, hs, 0.2, eta, dkmax, tuple(range(k)), theta, rho0, steps).rho
                   - ref).max() for k in range(2, dkmax + 1)]
    assert all(b <= 1.05 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-2] * 4 < errs[0], errs
    assert errs[-1] == 0.0

def test_hermitian_without_mask():
    q, hs, eta, rho0 = _structured_case(2, 6)
    r = iquapi.propagate(2, q, hs, 0.2, eta, 6, None, 0.0, rho0, 12)
    np.testing.assert_allclose(r.rho, np.conj(np.swapaxes(r.rho, 1, 2)), atol=1e-15)


def test_full_mask_and_zero_theta_are_defaults():
    q, hs, eta, rho0 = _structured_case(2, 5)
    a = iquapi.propagate(2, q, hs, 0.2, eta, 5, None, 0.0, rho0, 9)
    b = iquapi.propagate(2, q, hs, 0.2, eta, 5, tuple(range(5)), 0.0, rho0, 9)
    np.testing.assert_array_equal(a.rho, b.rho)


def test_filter_removes_paths_and_trace_loss_grows():
    q, hs, eta, rho0 = _structured_case(2, 8)
    losses, counts = [], []
    for th in (0.0, 1e-6, 1e-4, 1e-3):
        r = iquapi.propagate(2, q, hs, 0.2, eta, 8, (0, 1, 2, 5), th, rho0, 14)
        losses.append(abs(1 - np.trace(r.rho[-1]).real))
        counts.append(r.paths.amp.size)
    assert counts == sorted(counts, reverse=True) and counts[0] > counts[-1]
    assert losses[0] < 1e-13 and losses[-1] > losses[0]


# ---------------------------------------------------------------- filter

def _tls_propagator(delta, dt):
    """Closed form of exp(-i (delta/2) sigma_x dt)."""
    c, s = math.cos(delta * dt / 2), math.sin(delta * dt / 2)
    return np.array([[c, -1j * s], [-1j * s, c]])


def filtered_markov(U, q, e0, theta, rho0, steps):
    """Memory length 1 with the filter, written out term by term.

    A stored path then holds its newest point only, so the pre-merge groups
    the stored set by newest point and each group sum is an element of
    rho(t-1).  Child (a, b) of group (a', b') is the single term
        T = U[a, a'] rho(t-1)[a', b'] conj(U[b, b']) exp(-(q_a-q_b)(e0 q_a - e0* q_b)),
    and the filter acts on every such term separately: a term of modulus
    below theta is dropped before it enters rho(t), and is not carried to
    the next step (Sec. 2.1 filtering; Sec. 3.2: propagation, then
    filtering, then the density matrix).  Returns rho(0..steps) and the
    number of dropped terms and of kept terms with |T| >= theta > |T|^2."""
    M = len(q)
    out = [np.array(rho0, dtype=complex)]
    dropped = straddle = 0
    for _ in range(steps):
        cur, nxt = out[-1], np.zeros((M, M), dtype=complex)
        for a in range(M):
            for b in range(M):
                f = np.exp(-(q[a] - q[b]) * (e0 * q[a] - np.conj(e0) * q[b]))
                for ap in range(M):
                    for bp in range(M):
                        if cur[ap, bp] == 0:
                            continue          # no stored path ends there
                        term = U[a, ap] * cur[ap, bp] * np.conj(U[b, bp]) * f
                        if abs(term) >= theta:
                            nxt[a, b] += term
                            straddle += abs(term) ** 2 < theta
                        else:
                            dropped += 1
        out.append(nxt)
    return np.array(out), dropped, straddle


FILTER_PIN = dict(delta=1.0, dt=0.9, q=(1.0, -1.0), e0=0.04 + 0.03j, theta=0.06, steps=8,
                  rho0=((0.7, 0.2 - 0.3j), (0.2 + 0.3j, 0.3)))


def _filter_pin_error(mod):
    c = FILTER_PIN
    U = _tls_propagator(c["delta"], c["dt"])
    hs = np.array([[0, c["delta"] / 2], [c["delta"] / 2, 0]], dtype=complex)
    rho0 = np.array(c["rho0"], dtype=complex)
    want, _, _ = filtered_markov(U, np.array(c["q"]), c["e0"], c["theta"], rho0, c["steps"])
    r = mod.propagate(2, c["q"], hs, c["dt"], np.array([c["e0"]]), 1, None, c["theta"], rho0, c["steps"])
    return np.abs(r.rho - want).max()


def test_filtered_markov_map_at_memory_one():
    """The filter pinned by the term-wise Markov map (the case exercises
    dropped terms and kept terms whose squared modulus is below theta)."""
    c = FILTER_PIN
    U = _tls_propagator(c["delta"], c["dt"])
    _, dropped, straddle = filtered_markov(U, np.array(c["q"]), c["e0"], c["theta"],
                                           np.array(c["rho0"], dtype=complex), c["steps"])
    assert dropped >= 5 and straddle >= 5
    assert _filter_pin_error(iquapi) <= 1e-14


@pytest.mark.parametrize("theta,amps,kept", [
    # |amp| >= theta > |amp|^2 is kept; |amp| < theta is dropped
    (0.1, (0.2, 0.05j, -0.05j, 0.8), (0, 3)),
    # |amp| < theta <= |amp|^2 (theta > 1) is dropped
    (2.0, (1.5, 0.5j, -0.5j, 2.5), (3,)),
])
def test_filter_rule_on_a_hand_made_set(theta, amps, kept):
    """H_S = 0 and eta = 0 make every child a copy of its parent (the other
    children are exactly zero): the surviving children and rho(t) follow
    from the rule |amp| >= theta, applied before rho is summed."""
    sp = np.array([[0], [0], [1], [1]])
    sm = np.array([[0], [1], [0], [1]])
    paths = iquapi.Paths(sp, sm, np.array(amps, dtype=complex))
    U = iquapi.short_time_propagator(np.zeros((2, 2)), 0.1)
    out, rho, st = iquapi.step(paths, 1, U, np.array([1.0, -1.0]), np.zeros(1), 1, [0], theta, 2)
    want_keys = sorted(int(sp[i, 0]) | int(sm[i, 0]) << 1 for i in kept)
    assert sorted(int(k) for k in iquapi.packed_keys(out.sp, out.sm, 2)) == want_keys
    want_rho = np.zeros((2, 2), dtype=complex)
    for i in kept:
        want_rho[sp[i, 0], sm[i, 0]] = amps[i]
    np.testing.assert_array_equal(rho, want_rho)
    assert st.kept == len(kept)


def test_mask_validation():
    with pytest.raises(ValueError):
        iquapi.check_mask((0, 2), 6)
    with pytest.raises(ValueError):
        iquapi.check_mask((0, 1, 6), 6)
    assert iquapi.premerge_positions((0, 1, 2, 3, 4, 5, 6, 7, 8, 12), 16) == [0, 1, 2, 3, 4, 5, 6, 7, 11]
    assert iquapi.premerge_positions((0,), 1) == [0]


def test_packed_key_layout():
    sp = np.array([[1, 0, 1]])
    sm = np.array([[0, 1, 1]])
    # position p uses bits [2p, 2p+2): s+ low bit, s- high bit
    assert int(iquapi.packed_keys(sp, sm, 2)[0]) == (1 | 0 << 1) | ((0 | 1 << 1) << 2) | ((1 | 1 << 1) << 4)
    sp3 = np.array([[2, 1]])
    sm3 = np.array([[0, 2]])
    assert int(iquapi.packed_keys(sp3, sm3, 3)[0]) == (2 | 0 << 2) | ((1 | 2 << 2) << 4)


def test_representative_is_largest_weight_then_smallest_key():
    """A group of three members, two with equal |amp| (to 1e-14 relative):
    the representative is the smaller key of the two; the sum is over all."""
    M = 2
    sp = np.array([[0, 1, 0], [0, 1, 1], [0, 0, 1]])
    sm = np.array([[0, 0, 1], [0, 0, 0], [0, 1, 0]])
    amp = np.array([0.3 + 0.4j, 0.5 * (1 + 1e-14), 0.1j])
    rsp, rsm, S, _ = iquapi.premerge(iquapi.Paths(sp, sm, amp), [0], M)
    assert S.size == 1 and abs(S[0] - amp.sum()) < 1e-15
    keys = iquapi.packed_keys(sp, sm, M)
    want = int(min(keys[0], keys[1]))
    assert int(iquapi.packed_keys(rsp, rsm, M)[0]) == want


# ---------------------------------------------------------------- post-merging order

@pytest.mark.parametrize("M,dkmax,N,seed", [(2, 1, 5, 1), (2, 2, 5, 2), (2, 3, 6, 3), (2, 4, 5, 4),
                                            (3, 1, 3, 6), (3, 2, 4, 7), (3, 3, 4, 8)])
def test_post_merging_equals_brute_force_without_mask(M, dkmax, N, seed):
    """Without a mask the post-merge joins only children identical on the
    whole window, i.e. of parents that differ in the departing point alone,
    whose histories (lags < dkmax) are equal: the exact path sum."""
    c = W.random_case(seed, M, dkmax)
    rb = brute.rho_by_enumeration(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, c["rho0"], N)
    r = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, None, 0.0, c["rho0"], N, scheme="post")
    np.testing.assert_allclose(r.rho[N], rb, rtol=0, atol=2e-14)
    # the merged set holds at most one path per distinct window
    assert all(st.merged <= (M * M) ** min(st.t + 1, dkmax) for st in r.stats)


@pytest.mark.parametrize("mask,dkmax", [((0, 1, 2, 4), 6), ((0, 1), 5), ((0, 1, 2, 3, 4, 5, 7), 9)])
def test_post_merging_rabi_at_zero_coupling(mask, dkmax):
    delta, dt, steps = 1.0, 0.25, 24
    hs = np.array([[0, delta / 2], [delta / 2, 0]], dtype=complex)
    r = iquapi.propagate(2, [1.0, -1.0], hs, dt, np.zeros(dkmax), dkmax, mask, 0.0,
                         np.array([[1, 0], [0, 0]], dtype=complex), steps, scheme="post")
    t = dt * np.arange(steps + 1)
    np.testing.assert_allclose((r.rho[:, 0, 0] - r.rho[:, 1, 1]).real, np.cos(delta * t), atol=1e-13)
    np.testing.assert_allclose(r.rho[:, 0, 1], 0.5j * np.sin(delta * t), atol=1e-13)


@pytest.mark.parametrize("M,mask", [(2, (0, 1, 2, 5)), (3, (0, 1, 3))])
def test_post_merging_conserves_trace_and_bounds_the_merged_set(M, mask):
    q, hs, eta, rho0 = _structured_case(M, 8 if M == 2 else 5)
    dk = 8 if M == 2 else 5
    r = iquapi.propagate(M, q, hs, 0.2, eta, dk, mask, 0.0, rho0, 16, scheme="post")
    tr = np.trace(r.rho, axis1=1, axis2=2)
    np.testing.assert_allclose(tr, np.ones_like(tr), atol=1e-13)
    full = [st for st in r.stats if st.t + 1 >= dk]
    assert full and all(st.merged <= (M * M) ** len(mask) for st in full)


def test_post_merging_filtered_markov_map():
    c = FILTER_PIN
    U = _tls_propagator(c["delta"], c["dt"])
    hs = np.array([[0, c["delta"] / 2], [c["delta"] / 2, 0]], dtype=complex)
    rho0 = np.array(c["rho0"], dtype=complex)
    want, _, _ = filtered_markov(U, np.array(c["q"]), c["e0"], c["theta"], rho0, c["steps"])
    r = iquapi.propagate(2, c["q"], hs, c["dt"], np.array([c["e0"]]), 1, None, c["theta"], rho0, c["steps"],
                         scheme="post")
    assert np.abs(r.rho - want).max() <= 1e-14


# ---------------------------------------------------------------- symmetric splitting

def _random_Qh(seed, n):
    """Any sequence Q(j dt/2) with Q(0) = 0 defines coefficients both sides
    must agree on (the pins below need no bath)."""
    rng = np.random.default_rng(seed)
    j = np.arange(n)
    return (0.02 * j ** 1.5 * (1 + 0.1 * rng.normal(size=n))
            + 1j * 0.01 * j ** 2 * (1 + 0.1 * rng.normal(size=n))) * (j > 0)


def eta_from_Qh(Qh, dkmax):
    """Interior coefficients of full intervals from Q at half steps."""
    eta = np.zeros(dkmax, dtype=complex)
    eta[0] = Qh[2]
    for d in range(1, dkmax):
        eta[d] = Qh[2 * d + 2] - 2 * Qh[2 * d] + Qh[2 * d - 2]
    return eta


@pytest.mark.parametrize("M,dkmax,N,seed", [(2, 1, 4, 1), (2, 2, 5, 2), (2, 3, 5, 3), (2, 6, 5, 4), (2, 4, 6, 9),
                                            (3, 2, 4, 5), (3, 3, 3, 6)])
def test_symmetric_splitting_equals_brute_force(M, dkmax, N, seed):
    """The iterative propagation with the symmetric splitting's end points
    (point 0's half interval carried by the stored amplitudes, the newest
    point's half interval applied to rho(t) only) against the path sum
    over intervals, written independently from Q at the intervals' ends."""
    c = W.random_case(seed, M, dkmax)
    Qh = _random_Qh(seed, 2 * max(dkmax, N) + 4)
    eta = eta_from_Qh(Qh, dkmax)
    r = iquapi.propagate(M, c["q"], c["hs"], c["dt"], eta, dkmax, None, 0.0, c["rho0"], N, Qh=Qh)
    for n in range(1, N + 1):
        rb = brute.rho_by_enumeration_symmetric(M, c["q"], c["hs"], c["dt"], Qh, dkmax, c["rho0"], n)
        np.testing.assert_allclose(r.rho[n], rb, rtol=0, atol=2e-14)


@pytest.mark.parametrize("mask", [None, (0, 1, 3)])
def test_symmetric_splitting_pure_dephasing_exact(mask):
    """H_S = 0: the intervals tile [0, t], so within the memory the exact
    decoherence function exp(-(q_a-q_b)(q_a Q(t) - q_b Q*(t))) holds for the
    symmetric splitting too (it pins the end-point coefficients)."""
    alpha, wc, beta, dt, dkmax, steps = 0.1, 5.0, 5.0, 0.25, 7, 6
    bath = W.Bath(beta=beta, ohmic_alpha=alpha, ohmic_wc=wc)
    Qh = ohmic_Q_closed(alpha, wc, beta, 0.5 * dt * np.arange(2 * dkmax + 4))
    eta = eta_from_Qh(Qh, dkmax)
    for M, q in [(2, np.array([1.0, -1.0])), (3, np.array([-1.0, 0.0, 1.0]))]:
        rho0 = np.full((M, M), 1.0 / M, dtype=complex)
        r = iquapi.propagate(M, q, np.zeros((M, M)), dt, eta, dkmax, mask, 0.0, rho0, steps, Qh=Qh)
        for n in range(1, steps + 1):
            Q = ohmic_Q_closed(alpha, wc, beta, n * dt)
            expect = rho0 * np.exp(-(q[:, None] - q[None, :]) * (q[:, None] * Q - q[None, :] * np.conj(Q)))
            np.testing.assert_allclose(r.rho[n], expect, atol=1e-13)
    assert bath.beta == beta



def _splitting_order_ratios(bath, t_end, mod=iquapi, Ns=(2, 4, 8)):
    """rho(t_end) with the full memory (no truncation) at dt = t_end/N for
    N = 2, 4, 8, in the right-box reading and with the symmetric splitting;
    the ratio of successive differences, |rho_2 - rho_4| / |rho_4 - rho_8|,
    is 2^p for a method of order p in dt."""
    hs = np.array([[0, 0.5], [0.5, 0]], dtype=complex)
    q = np.array([1.0, -1.0])
    rho0 = np.array([[1, 0], [0, 0]], dtype=complex)
    res = {}
    for N in Ns:
        dt = t_end / N
        eta = B.eta_coefficients(bath, dt, N)
        Qh = B.Q_of_t(bath, 0.5 * dt * np.arange(2 * N + 3))
        res[N] = (mod.propagate(2, q, hs, dt, eta, N, None, 0.0, rho0, N).rho[N],
                  mod.propagate(2, q, hs, dt, eta, N, None, 0.0, rho0, N, Qh=Qh).rho[N])
    return [np.abs(res[Ns[0]][k] - res[Ns[1]][k]).max() / np.abs(res[Ns[1]][k] - res[Ns[2]][k]).max()
            for k in (0, 1)]


@pytest.mark.parametrize("alpha,wc,beta,t_end", [(0.05, 3.0, 2.0, 1.6), (0.02, 2.0, 1.0, 2.0), (0.1, 2.0, 0.5, 1.0)])
def test_symmetric_splitting_is_second_order_in_dt(alpha, wc, beta, t_end):
    """The splitting of the short-time propagator between H_S and the bath
    (Eq. quapi_red_rho) decides the order in dt of the exact-memory path sum:
    the right-box reading (R1: the system propagates over a step, the bath
    sees the new point over the whole step) is a one-sided splitting, first
    order; the symmetric splitting (R17: intervals centred on the points,
    half intervals at both ends) is second order.  The ratio of successive
    differences at dt, dt/2, dt/4 must show it (2 and 4 asymptotically; the
    steps here are coarse, so the bands are wide but do not overlap)."""
    bath = W.Bath(beta=beta, ohmic_alpha=alpha, ohmic_wc=wc)
    r_box, r_sym = _splitting_order_ratios(bath, t_end)
    assert 1.6 < r_box < 3.0, r_box
    assert 3.3 < r_sym < 6.0, r_sym

# ---------------------------------------------------------------- planted mistakes

MUTATIONS = {
    "dropped conjugate in history": ("- np.conj(eta[d]) * q[rsm[:, d - 1]]", "- eta[d] * q[rsm[:, d - 1]]"),
    "history index off by one": ("q[rsp[:, d - 1]]", "q[rsp[:, d]]"),
    "wrong sign of new-point term": ("(H + eta[0] * q[a] - np.conj(eta[0]) * q[b])",
                                     "(H - eta[0] * q[a] - np.conj(eta[0]) * q[b])"),
    "transposed propagator": ("prop = U[a, rsp[:, 0]] * np.conj(U[b, rsm[:, 0]])",
                              "prop = U[rsp[:, 0], a] * np.conj(U[b, rsm[:, 0]])"),
    "backward branch not conjugated": ("np.conj(U[b, rsm[:, 0]])", "U[b, rsm[:, 0]]"),
    "history misses the last lag": ("for d in range(1, n_act):", "for d in range(1, n_act - 1):"),
    "sum keeps one member per group": ("np.add.at(S, inv, paths.amp)", "S[inv] = paths.amp"),
    "new point enters the history sum": ("for d in range(1, n_act):", "for d in range(0, n_act):"),
    "theta not squared in the filter": ("keep = w2 >= th2", "keep = w2 >= theta"),
    "rho summed before the filter": ("rho[a, b] = child[keep].sum()", "rho[a, b] = child.sum()"),
    "pre-merge on P without the shift": ("return sorted(set([p - 1 for p in P if p >= 1] + [0]))",
                                         "return sorted(set(P))"),
}


def _mutant(src_old, src_new):
    import inspect
    src = inspect.getsource(iquapi)
    assert src_old in src, src_old
    import sys
    name = "iquapi_mutant"
    mod = types.ModuleType(name)
    sys.modules[name] = mod
    try:
        exec(compile(src.replace(src_old, src_new), name, "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod


def _pins_pass(mod):
    try:
        for (M, dkmax, N, seed) in [(2, 3, 5, 3), (3, 2, 4, 7), (2, 2, 5, 12)]:
            c = W.random_case(seed, M, dkmax)
            rb = brute.rho_by_enumeration(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, c["rho0"], N)
            r = mod.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, None, 0.0, c["rho0"], N)
            if np.abs(r.rho[N] - rb).max() > 2e-14:
                return False
        q, hs, eta, rho0 = _structured_case(2, 8)
        r = mod.propagate(2, q, hs, 0.2, eta, 8, (0, 1, 2, 5), 0.0, rho0, 16)
        if np.abs(np.trace(r.rho, axis1=1, axis2=2) - 1).max() > 1e-13:
            return False
        if _filter_pin_error(mod) > 1e-14:
            return False
        for theta, amps, kept in [(0.1, (0.2, 0.05j, -0.05j, 0.8), (0, 3)), (2.0, (1.5, 0.5j, -0.5j, 2.5), (3,))]:
            paths = mod.Paths(np.array([[0], [0], [1], [1]]), np.array([[0], [1], [0], [1]]),
                              np.array(amps, dtype=complex))
            _, rho, _ = mod.step(paths, 1, np.eye(2, dtype=complex), np.array([1.0, -1.0]), np.zeros(1), 1, [0],
                                 theta, 2)
            if not np.array_equal(np.diag(rho), [amps[0] if 0 in kept else 0, amps[3] if 3 in kept else 0]):
                return False
        return _prefix_pins_pass(mod, "pre")
    except Exception:
        return False


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    assert not _pins_pass(_mutant(old, new)), f"pins missed: {name}"


def test_unmutated_oracle_passes_mutation_harness():
    assert _pins_pass(iquapi)


POST_MUTATIONS = {
    "post: own history index off by one": ("q[paths.sp[:, d - 1]] - np.conj(eta[d]) * q[paths.sm[:, d - 1]]",
                                           "q[paths.sp[:, d]] - np.conj(eta[d]) * q[paths.sm[:, d]]"),
    "post: merged on one position too few": ("out, near_tie = merge_on(unmerged, sorted(P), M)",
                                             "out, near_tie = merge_on(unmerged, sorted(P)[:-1], M)"),
    "post: never merged": ("if L_child == dkmax and unmerged.amp.size:", "if False:"),
    "post: merged on P' instead of P": ("out, near_tie = merge_on(unmerged, sorted(P), M)",
                                        "out, near_tie = merge_on(unmerged, premerge_positions(P, dkmax), M)"),
    "post: backward branch not conjugated": ("prop = U[a, paths.sp[:, 0]] * np.conj(U[b, paths.sm[:, 0]])",
                                             "prop = U[a, paths.sp[:, 0]] * U[b, paths.sm[:, 0]]"),
    "post: rho summed before the filter": ("            rho[a, b] = child[keep].sum()\n            k = int(np.count_nonzero(keep))\n            new_sp.append(np.hstack([np.full",
                                           "            rho[a, b] = child.sum()\n            k = int(np.count_nonzero(keep))\n            new_sp.append(np.hstack([np.full"),
}


def _post_pins_pass(mod):
    try:
        for (M, dkmax, N, seed) in [(2, 3, 6, 3), (3, 2, 4, 7)]:
            c = W.random_case(seed, M, dkmax)
            rb = brute.rho_by_enumeration(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, c["rho0"], N)
            r = mod.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, None, 0.0, c["rho0"], N, scheme="post")
            if np.abs(r.rho[N] - rb).max() > 2e-14:
                return False
            if any(st.merged > (M * M) ** min(st.t + 1, dkmax) for st in r.stats):
                return False
        c = FILTER_PIN
        hs = np.array([[0, c["delta"] / 2], [c["delta"] / 2, 0]], dtype=complex)
        rho0 = np.array(c["rho0"], dtype=complex)
        want, _, _ = filtered_markov(_tls_propagator(c["delta"], c["dt"]), np.array(c["q"]), c["e0"], c["theta"],
                                     rho0, c["steps"])
        r = mod.propagate(2, c["q"], hs, c["dt"], np.array([c["e0"]]), 1, None, c["theta"], rho0, c["steps"],
                          scheme="post")
        return np.abs(r.rho - want).max() <= 1e-14 and _prefix_pins_pass(mod, "post")
    except Exception:
        return False


@pytest.mark.parametrize("name", sorted(POST_MUTATIONS))
def test_planted_post_merging_mistake_is_caught(name):
    old, new = POST_MUTATIONS[name]
    assert not _post_pins_pass(_mutant(old, new)), f"pins missed: {name}"


def test_unmutated_oracle_passes_post_merging_harness():
    assert _post_pins_pass(iquapi)


SYM_MUTATIONS = {
    "sym: point 0 without its half interval": ("        amp = amp * np.exp(-(q[a] - q[b]) * (ep.eta00 * q[a] - np.conj(ep.eta00) * q[b]))",
                                               "        amp = amp * 1.0"),
    "sym: no end-point correction of rho": ("                rho[a, b] = (child * corr)[keep].sum()", "                rho[a, b] = child[keep].sum()"),
    "sym: point 0 with the interior coefficient": ("            H += ep.eta0[t] * q[rsp[:, t - 1]] - np.conj(ep.eta0[t]) * q[rsm[:, t - 1]]",
                                                   "            H += eta[t] * q[rsp[:, t - 1]] - np.conj(eta[t]) * q[rsm[:, t - 1]]"),
    "sym: end point as interior for the history": ("            dE = ep.etaE[d] - eta[d]", "            dE = 0.0 * eta[d]"),
    "sym: half interval of the newest point ignored": ("        dS = ep.eta00 - eta[0]", "        dS = 0.0 * eta[0]"),
}


def _sym_pins_pass(mod):
    try:
        for (M, dkmax, N, seed) in [(2, 3, 5, 3), (3, 2, 4, 5), (2, 6, 4, 4)]:
            c = W.random_case(seed, M, dkmax)
            Qh = _random_Qh(seed, 2 * max(dkmax, N) + 4)
            r = mod.propagate(M, c["q"], c["hs"], c["dt"], eta_from_Qh(Qh, dkmax), dkmax, None, 0.0, c["rho0"], N, Qh=Qh)
            rb = brute.rho_by_enumeration_symmetric(M, c["q"], c["hs"], c["dt"], Qh, dkmax, c["rho0"], N)
            if np.abs(r.rho[N] - rb).max() > 2e-14:
                return False
        # second order in dt (a check of the reading itself, not of its code)
        r_sym = _splitting_order_ratios(W.Bath(beta=2.0, ohmic_alpha=0.05, ohmic_wc=3.0), 1.6, mod)[1]
        return 3.3 < r_sym < 6.0
    except Exception:
        return False


@pytest.mark.parametrize("name", sorted(SYM_MUTATIONS))
def test_planted_symmetric_splitting_mistake_is_caught(name):
    old, new = SYM_MUTATIONS[name]
    assert not _sym_pins_pass(_mutant(old, new)), f"pins missed: {name}"


def test_unmutated_oracle_passes_symmetric_harness():
    assert _sym_pins_pass(iquapi)


# ---------------------------------------------------------------- wide keys (M up to 8)

def _random_set(rng, M, L, n=3000):
    sp = rng.integers(0, M, size=(n, L))
    sm = rng.integers(0, M, size=(n, L))
    amp = rng.normal(size=n) + 1j * rng.normal(size=n)
    amp[::7] = 10.0 * amp[::7] / np.abs(amp[::7])   # equal largest weights: the tie rule decides
    return iquapi.Paths(sp, sm, amp)


def _same_premerge(a, b):
    ka = sorted(map(tuple, np.hstack([a[0], a[1]])))
    kb = sorted(map(tuple, np.hstack([b[0], b[1]])))
    return ka == kb and np.allclose(np.sort_complex(a[2]), np.sort_complex(b[2]), rtol=0, atol=1e-14)


@pytest.mark.parametrize("M,L,Pp", [(2, 6, [0, 1, 3]), (3, 5, [0, 1]), (4, 4, [0, 2]), (5, 4, [0, 1]),
                                    (6, 3, [0, 2]), (8, 3, [0])])
def test_premerge_without_packing_equals_packed_premerge(M, L, Pp):
    """premerge_rows (keys of any width) against the packed-key premerge
    where both apply: the same groups, sums and representatives, ties
    included."""
    rng = np.random.default_rng(M * 10 + L)
    P = _random_set(rng, M, L)
    assert _same_premerge(iquapi.premerge(P, Pp, M), iquapi.premerge_rows(P, Pp, M))


@pytest.mark.parametrize("M,dkmax,N,seed", [(5, 2, 3, 1), (5, 3, 3, 2), (6, 2, 3, 3)])
def test_iterative_equals_brute_force_larger_M(M, dkmax, N, seed):
    c = W.random_case(seed, M, dkmax)
    rb = brute.rho_by_enumeration(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, c["rho0"], N)
    r = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, None, 0.0, c["rho0"], N)
    assert np.abs(r.rho[N] - rb).max() <= 2e-14


def test_wide_keys_go_through_premerge_rows():
    """M = 8 at 11 points: 66 key bits, beyond a packed 64-bit key; the
    step uses premerge_rows and agrees with a run whose window columns are
    reordered (a relabelling that leaves the physics unchanged is not
    available, so the check is the equality of the two premerge forms on
    the step's own input)."""
    rng = np.random.default_rng(3)
    P = _random_set(rng, 8, 11, n=4000)
    a = iquapi.premerge(P, [0, 1], 8)
    assert _same_premerge(a, iquapi.premerge_rows(P, [0, 1], 8))
    # the packed form cannot hold these keys
    assert iquapi.state_bits(8)[1] * 11 > 64


ROWS_MUTATIONS = {
    "backward point before forward within a position reversed": ("keys += [paths.sp[idx, p], paths.sm[idx, p]]",
                                                                  "keys += [paths.sm[idx, p], paths.sp[idx, p]]"),
    "groups ignore the backward points": ("gk = np.concatenate([paths.sp[:, cols], paths.sm[:, cols]], axis=1)",
                                          "gk = np.concatenate([paths.sp[:, cols], paths.sp[:, cols]], axis=1)"),
    "newest position compared first": ("for p in range(L):\n        keys +=", "for p in reversed(range(L)):\n        keys +="),
}


@pytest.mark.parametrize("name", sorted(ROWS_MUTATIONS))
def test_planted_premerge_rows_mistake_is_caught(name):
    old, new = ROWS_MUTATIONS[name]
    mod = _mutant(old, new)
    rng = np.random.default_rng(11)
    caught = False
    for M, L, Pp in [(2, 6, [0, 1, 3]), (3, 5, [0, 1]), (5, 4, [0, 1])]:
        P = _random_set(rng, M, L)
        if not _same_premerge(iquapi.premerge(P, Pp, M), mod.premerge_rows(P, Pp, M)):
            caught = True
    assert caught
