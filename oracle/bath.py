"""Oracle: bath spectral densities and discretised influence coefficients.

TEST INFRASTRUCTURE (see oracle/__init__.py): never imported by the product.

The paper defers the explicit form of the influence coefficients eta_ij of
Eq. inf_fun to its references.  The oracle takes the standard reading:

  bath correlation  alpha(t) = (1/pi) int_0^inf J(w) [coth(beta w/2) cos wt - i sin wt] dw
                    (consistent with the normalisation of J in Eq. SD),
  double integral   Q(t) = int_0^t dt' int_0^t' dt'' alpha(t'')
                         = (1/pi) int J(w)/w^2 [coth(beta w/2)(1 - cos wt) - i (wt - sin wt)] dw,

and, with the path value q_k held over the box ((k-1) dt, k dt] (point 0
carries no box), the coefficient linking two points d steps apart is the
double integral of alpha over a pair of boxes:

  eta_0 = Q(dt),   eta_d = Q((d+1) dt) - 2 Q(d dt) + Q((d-1) dt)   (d >= 1).

Q(t) is evaluated by adaptive Gauss-Kronrod quadrature (scipy.quad_vec)
over all requested times at once.  Pins (tests/test_oracle_pins.py): closed
forms of Q for the ohmic density (log-Gamma series) and for the resonance of
Eq. sharpSD (pole and Matsubara expansion).
"""
from __future__ import annotations

import numpy as np
from scipy import integrate


def resonance_amplitude(w0: float, gamma: float, lam: float) -> float:
    """Amplitude alpha of Eq. sharpSD with Omega = w0, 2 pi kappa Omega = gamma,
    fixed by lambda = int J(w)/w dw = pi alpha Omega^2 / gamma."""
    return lam * gamma / (np.pi * w0 ** 2)


def spectral_density(bath, w):
    """J(w) of the workload's bath (sum of the ohmic part and the resonance part)."""
    w = np.asarray(w, dtype=np.float64)
    j = np.zeros_like(w)
    if bath.ohmic_alpha != 0.0:
        j = j + 0.5 * np.pi * bath.ohmic_alpha * w * np.exp(-w / bath.ohmic_wc)
    if bath.res_lambda != 0.0:
        a = resonance_amplitude(bath.res_w0, bath.res_gamma, bath.res_lambda)
        W = bath.res_w0
        j = j + 2.0 * a * w * W ** 4 / ((W ** 2 - w ** 2) ** 2 + (bath.res_gamma * w) ** 2)
    return j


def _x_minus_sin(x):
    """x - sin x without cancellation for small x."""
    x = np.asarray(x, dtype=np.float64)
    out = x - np.sin(x)
    small = np.abs(x) < 0.1
    if np.any(small):
        xs = x[small]
        x2 = xs * xs
        # Taylor series: x^3/3! - x^5/5! + x^7/7! - x^9/9! + x^11/11!
        s = xs * x2 / 6.0 * (1 - x2 / 20.0 * (1 - x2 / 42.0 * (1 - x2 / 72.0 * (1 - x2 / 110.0))))
        out[small] = s
    return out


def _breakpoints(bath):
    pts = []
    if bath.ohmic_alpha != 0.0:
        wc = bath.ohmic_wc
        pts += [0.5 * wc, wc, 2 * wc, 5 * wc, 10 * wc, 20 * wc, 40 * wc]
    if bath.res_lambda != 0.0:
        w0, g = bath.res_w0, bath.res_gamma
        for k in (0.0, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0, 32.0):
            pts += [w0 - k * g, w0 + k * g]
    return sorted(p for p in set(pts) if p > 0)


def Q_of_t(bath, ts) -> np.ndarray:
    """Q(t) for every t in ts, by quadrature of its spectral representation."""
    ts = np.atleast_1d(np.asarray(ts, dtype=np.float64))
    beta = bath.beta

    def integrand(w):
        jw = spectral_density(bath, w) / (w * w)
        coth = 1.0 / np.tanh(0.5 * beta * w)
        re = jw * coth * 2.0 * np.sin(0.5 * w * ts) ** 2
        im = -jw * _x_minus_sin(w * ts)
        return np.concatenate([re, im]) / np.pi

    if bath.res_lambda != 0.0:
        w_split = 40.0 * max(bath.res_w0 + 32 * bath.res_gamma, bath.ohmic_wc if bath.ohmic_alpha else 0.0)
    else:
        w_split = 60.0 * bath.ohmic_wc
    pts = [p for p in _breakpoints(bath) if p < w_split]
    edges = [0.0] + pts + [w_split]
    total = np.zeros(2 * ts.size)
    for a, b in zip(edges[:-1], edges[1:]):
        val, _err = integrate.quad_vec(integrand, a, b, epsabs=1e-16, epsrel=1e-12, limit=20000)
        total += val
    if bath.res_lambda != 0.0:
        # algebraic tail of the resonance (J ~ w^-3) beyond w_split
        val, _err = integrate.quad_vec(integrand, w_split, np.inf, epsabs=1e-17, epsrel=1e-12, limit=20000)
        total += val
    return total[: ts.size] + 1j * total[ts.size:]


def eta_coefficients(bath, dt: float, n: int) -> np.ndarray:
    """eta_0 .. eta_{n-1} for lags d = 0 .. n-1 (Toeplitz coefficients eta_{k,k-d})."""
    ts = dt * np.arange(0, n + 1)          # Q(0) = 0, Q(dt), ..., Q(n dt)
    q = Q_of_t(bath, ts[1:])
    qfull = np.concatenate([[0.0 + 0.0j], q])
    eta = np.empty(n, dtype=np.complex128)
    eta[0] = qfull[1]
    for d in range(1, n):
        eta[d] = qfull[d + 1] - 2.0 * qfull[d] + qfull[d - 1]
    return eta
