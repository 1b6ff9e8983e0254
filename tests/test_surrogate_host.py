"""Host logic of the surrogate's checkpoint check (no GPU): which instances
fall back to the path update, and which errors are reported."""
import numpy as np
import pytest

from paper_2506_03127_gb300.surrogate import checkpoint_errors


def _rho(p_up, coh):
    return np.array([[p_up, coh], [np.conj(coh), 1.0 - p_up]], dtype=complex)


def test_fallback_on_trace_or_negative_eigenvalue_and_errors_reported():
    """Three instances, checkpoints 2 and 4: instance 0 is off by 0.01 and
    stays; instance 1's trace is off by 0.1 at t = 2 (beyond 0.05) and falls
    back; instance 2 is a unit-trace matrix with an eigenvalue of -0.05 at
    t = 4 (beyond -0.02) and falls back.  The raw errors include every
    instance, the combined ones only those that stay (the others take the
    path update's result, error 0)."""
    n, T = 3, 5
    plain = np.empty((T, n, 2, 2), dtype=complex)
    for t in range(T):
        for i in range(n):
            plain[t, i] = _rho(0.7 - 0.02 * t, 0.1j * (i + 1))
    sur = np.transpose(plain, (1, 0, 2, 3)).copy()
    sur[0, 2, 0, 1] += 0.01
    sur[0, 4, 1, 0] -= 0.01
    sur[1, 2] += np.diag([0.05, 0.05])            # trace 1.1
    sur[2, 4] = _rho(1.05, 0.0)                   # eigenvalues 1.05 and -0.05, trace 1
    combined, raw, fallback = checkpoint_errors(sur, plain, (2, 4))
    np.testing.assert_array_equal(fallback, [False, True, True])
    assert raw[2] == pytest.approx(0.05) and raw[4] == pytest.approx(np.abs(sur[2, 4] - plain[4, 2]).max())
    assert combined == pytest.approx({2: 0.01, 4: 0.01})


def test_within_tolerances_nothing_falls_back():
    n, T = 2, 3
    plain = np.empty((T, n, 2, 2), dtype=complex)
    for t in range(T):
        for i in range(n):
            plain[t, i] = _rho(0.5, 0.2)
    sur = np.transpose(plain, (1, 0, 2, 3)).copy()
    sur[0, 1] += np.diag([0.02, 0.02])            # trace off by 0.04 < 0.05
    sur[1, 2] = _rho(1.015, 0.0)                  # eigenvalue -0.015 > -0.02
    combined, raw, fallback = checkpoint_errors(sur, plain, (1, 2))
    assert not fallback.any()
    assert combined == raw
