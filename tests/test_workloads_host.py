"""The synthetic inputs (`workloads.py`) against facts that fix them
independently of how they are built (no GPU)."""
import math

import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("nvib", [2, 3, 4, 6])
def test_reaction_coordinate_basis_and_hamiltonian(nvib):
    """The model of Sec. 4.3 in the eigenbasis of the truncated position
    operator B + B^dagger: its eigenvalues are sqrt(2) times the roots of
    the Hermite polynomial H_nvib (the Gauss-Hermite nodes), each once per
    electronic state; H_S has the spectrum of the same Hamiltonian written
    in the number basis (a change of basis keeps it); rho0 is |up><up| times
    the mode's thermal state, Boltzmann populations of the number states."""
    w = W.reaction_coordinate(nvib=nvib)
    nodes, _ = np.polynomial.hermite.hermgauss(nvib)
    q = np.array(w.q)
    np.testing.assert_allclose(q[:nvib], math.sqrt(2.0) * np.sort(nodes), atol=1e-13)
    np.testing.assert_array_equal(q[:nvib], q[nvib:])
    # the same model in the number basis of the mode
    b = np.diag(np.sqrt(np.arange(1, nvib, dtype=float)), 1)
    delta, omega, g, kT = 1.0, 1.0, 0.18, 1.0
    sx, sz = np.array([[0.0, 1.0], [1.0, 0.0]]), np.diag([1.0, -1.0])
    h_num = 0.5 * delta * np.kron(sx, np.eye(nvib)) + g * np.kron(sz, b + b.T) + omega * np.kron(
        np.eye(2), np.diag(np.arange(nvib, dtype=float)))
    hs = w.hs_array()
    np.testing.assert_allclose(hs, hs.conj().T, atol=1e-14)
    np.testing.assert_allclose(np.linalg.eigvalsh(hs), np.linalg.eigvalsh(h_num), atol=1e-12)
    # rho0 back in the number basis: |up><up| x exp(-omega n / kT) / Z
    _, V = np.linalg.eigh(b + b.T)
    U = np.kron(np.eye(2), V)
    rho_num = U @ w.rho0_array() @ U.conj().T
    boltz = np.exp(-omega * np.arange(nvib) / kT)
    want = np.kron(np.diag([1.0, 0.0]), np.diag(boltz / boltz.sum()))
    np.testing.assert_allclose(rho_num, want, atol=1e-14)


def test_reaction_coordinate_bath_and_settings():
    """J = kappa w exp(-w/wc) with kappa = 0.056 written as (pi/2) alpha w
    exp(-w/wc); the converged settings of the paper's runs; Delta k_eff = 10."""
    w = W.reaction_coordinate()
    assert w.bath.ohmic_alpha * math.pi / 2 == pytest.approx(0.056)
    assert (w.M, w.dkmax, w.dt, w.theta, w.bath.ohmic_wc, w.bath.beta) == (8, 12, 0.06, 1e-9, 10.0, 1.0)
    assert len(w.mask) == 10 and set(w.mask) <= set(range(w.dkmax)) and {0, 1} <= set(w.mask)


def test_sweeps_draw_the_stated_distributions():
    """Resonance sweep: w0 in [0.5, 2], lambda cycling through 0.05, 0.1,
    0.2, width 0.05, one shared system; coupling sweep: the same instances
    with the ohmic coupling drawn log-uniform in [0.02, 0.8]."""
    rs = W.resonance_sweep(64)
    w0 = np.array([w.bath.res_w0 for w in rs])
    assert w0.min() >= 0.5 and w0.max() <= 2.0 and np.unique(w0).size == 64
    assert [w.bath.res_lambda for w in rs[:6]] == [0.05, 0.1, 0.2, 0.05, 0.1, 0.2]
    assert all(w.bath.res_gamma == 0.05 for w in rs)
    assert len({(w.M, w.q, w.hs, w.dt, w.dkmax, w.mask, w.theta, w.rho0) for w in rs}) == 1
    cs = W.coupling_sweep(64)
    alpha = np.array([w.bath.ohmic_alpha for w in cs])
    assert alpha.min() >= 0.02 and alpha.max() <= 0.8
    assert np.log(alpha).std() > 0.5                       # spread over the log range
    assert [w.bath.res_w0 for w in cs] == list(w0)          # same resonances as the resonance sweep
