"""Seeded synthetic inputs for the MACGIC-iQUAPI path update.

This module holds the parameter sets of the workloads and the seeded random
draws used by tests and benchmarks, and nothing of the propagation method's
arithmetic: system Hamiltonians in the DVR basis, coupling eigenvalues, bath
parameters, time step, memory length, MACGIC mask, filter threshold and the
initial reduced density matrix.  Both the CUDA library's callers and the
oracle take their inputs from here.

Physical model (paper Sec. 2, Eq. tot_ham): H = H_S + H_B + H_SB with the
bath coupled through the diagonal operator sum_i q_i |q_i><q_i|.  Units:
hbar = 1, energies in units of the tunnelling splitting Delta.

Bath spectral densities are given by parameters only:
  * ohmic:     J(w) = (pi/2) * alpha * w * exp(-w / wc)
  * resonance: the sharp-resonance form of Eq. sharpSD with Omega = w0 and
               resonance width 2*pi*kappa*Omega = gamma; its amplitude is
               fixed by the reorganisation energy lambda = int J(w)/w dw.
The total J is the sum of the parts that are switched on (nonzero).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace
from typing import Optional, Tuple

import numpy as np


@dataclass(frozen=True)
class Bath:
    beta: float
    ohmic_alpha: float = 0.0
    ohmic_wc: float = 5.0
    res_w0: float = 0.0
    res_gamma: float = 0.0
    res_lambda: float = 0.0


@dataclass(frozen=True)
class Workload:
    name: str
    M: int
    q: Tuple[float, ...]
    hs: Tuple[Tuple[complex, ...], ...]     # M x M, row-major, Hermitian
    bath: Bath
    dt: float
    dkmax: int
    mask: Optional[Tuple[int, ...]]          # window positions at time t, 0 = newest; None = all
    theta: float                             # filter threshold on |amplitude|; 0 = keep all
    rho0: Tuple[Tuple[complex, ...], ...]
    steps: int

    def hs_array(self) -> np.ndarray:
        return np.array(self.hs, dtype=np.complex128)

    def rho0_array(self) -> np.ndarray:
        return np.array(self.rho0, dtype=np.complex128)

    def mask_list(self):
        return list(range(self.dkmax)) if self.mask is None else sorted(self.mask)


def _tls_hs(delta: float = 1.0):
    # H_S = (Delta/2) sigma_x in the sigma_z basis, state 0 = up (q = +1)
    return ((0.0, delta / 2), (delta / 2, 0.0))


_UP = ((1.0, 0.0), (0.0, 0.0))

# Spin-boson, ohmic bath, full memory of 8 steps, no mask, no filter:
# 4^8 = 65536 stored paths once the window is full; 100 steps.
SPIN_BOSON_OHMIC_DK8 = Workload(
    name="spin_boson_ohmic_dk8",
    M=2, q=(1.0, -1.0), hs=_tls_hs(),
    bath=Bath(beta=5.0, ohmic_alpha=0.1, ohmic_wc=5.0),
    dt=0.25, dkmax=8, mask=None, theta=0.0, rho0=_UP, steps=100)

# Spin-boson, ohmic background plus a sharp resonance, memory 16 steps,
# MACGIC mask: the last 8 lags fine, then 4-step blocks represented by their
# first lag (Delta k_eff = 10), filter 1e-9, 2000 steps.
STRUCTURED_MASK = (0, 1, 2, 3, 4, 5, 6, 7, 8, 12)
SPIN_BOSON_STRUCTURED_DK16 = Workload(
    name="spin_boson_structured_dk16",
    M=2, q=(1.0, -1.0), hs=_tls_hs(),
    bath=Bath(beta=10.0, ohmic_alpha=0.05, ohmic_wc=5.0,
              res_w0=1.0, res_gamma=0.05, res_lambda=0.1),
    dt=0.1, dkmax=16, mask=STRUCTURED_MASK, theta=1e-9, rho0=_UP, steps=2000)

# Three-level chain (coupling eigenvalues -1, 0, 1; neighbour couplings 1),
# the same structured bath, memory 12 steps with mask {0..8}, filter 1e-10.
CHAIN3_STRUCTURED_DK12 = Workload(
    name="chain3_structured_dk12",
    M=3, q=(-1.0, 0.0, 1.0),
    hs=((0.0, 1.0, 0.0), (1.0, 0.0, 1.0), (0.0, 1.0, 0.0)),
    bath=SPIN_BOSON_STRUCTURED_DK16.bath,
    dt=0.1, dkmax=12, mask=(0, 1, 2, 3, 4, 5, 6, 7, 8), theta=1e-10,
    rho0=((1.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0)), steps=300)

# The same chain with memory 7 and mask {0..5}: about 2.5e5 stored paths, a
# case whose merging steps the oracle runs in seconds.
CHAIN3_STRUCTURED_DK7 = replace(CHAIN3_STRUCTURED_DK12, name="chain3_structured_dk7", dkmax=7,
                                mask=(0, 1, 2, 3, 4, 5), steps=60)

# The paper's distributed-memory scaling model (Sec. 4.2): TLS with
# H_S = (Delta/2) sigma_x, ohmic J = (gamma/pi) w exp(-w/wc), gamma = 1/16,
# wc = 10, kT = 0.2, dt = 0.3, t_max = 35, full QUAPI (no mask, no filter),
# memory 14 steps -> 2^28 paths.  alpha below is the same J written in the
# (pi/2) alpha w convention: alpha = 2 gamma / pi^2.
def tls_ohmic_full(dkmax: int = 14) -> Workload:
    return Workload(
        name=f"tls_ohmic_full_dk{dkmax}",
        M=2, q=(1.0, -1.0), hs=_tls_hs(),
        bath=Bath(beta=5.0, ohmic_alpha=2.0 * (1.0 / 16.0) / math.pi ** 2, ohmic_wc=10.0),
        dt=0.3, dkmax=dkmax, mask=None, theta=0.0, rho0=_UP,
        steps=int(round(35.0 / 0.3)))


TLS_OHMIC_FULL_DK14 = tls_ohmic_full(14)

SWEEP_SEED = 2506031270


def resonance_sweep(n_instances: int = 64, seed: int = SWEEP_SEED, theta: float = 1e-7):
    """Frequency sweep: instances of the 8-step ohmic spin-boson model with an
    added resonance, w0 ~ U[0.5, 2.0] (seeded), lambda cycling through
    {0.05, 0.1, 0.2}, width 0.05, filter theta.  At theta = 1e-9 every
    instance keeps the same number of paths; at 1e-7 the counts differ from
    instance to instance (by about 1-2 %), which is the default."""
    rng = np.random.default_rng(seed)
    w0s = rng.uniform(0.5, 2.0, size=n_instances)
    lams = (0.05, 0.1, 0.2)
    out = []
    base = SPIN_BOSON_OHMIC_DK8
    for i in range(n_instances):
        bath = replace(base.bath, res_w0=float(w0s[i]), res_gamma=0.05, res_lambda=lams[i % 3])
        out.append(replace(base, name=f"sweep_{i:02d}", bath=bath, theta=theta))
    return out


def coupling_sweep(n_instances: int = 64, seed: int = SWEEP_SEED, theta: float = 1e-7):
    """Resonance and coupling sweep: the resonance sweep's instances with the
    ohmic coupling drawn as well, alpha log-uniform in [0.02, 0.8] (seeded).
    Stronger coupling damps more off-diagonal paths below the filter, so the
    instances keep from about 16 000 to 39 000 paths at theta = 1e-7: the
    work per instance differs by more than a factor of 2."""
    rng = np.random.default_rng(seed + 1)
    alphas = np.exp(rng.uniform(np.log(0.02), np.log(0.8), size=n_instances))
    out = []
    for i, w in enumerate(resonance_sweep(n_instances, seed, theta)):
        bath = replace(w.bath, ohmic_alpha=float(alphas[i]))
        out.append(replace(w, name=f"csweep_{i:02d}", bath=bath))
    return out


def reaction_coordinate(nvib: int = 4, dkmax: int = 12, mask=(0, 1, 2, 3, 4, 5, 6, 7, 8, 10), theta: float = 1e-9,
                        steps: int = 400) -> Workload:
    """The primary reaction-coordinate model of Sec. 4.3 (Eq. tot_TSS_HO):
    a bias-free TLS (H = Delta/2 sigma_x, Delta = 1) coupled by g sigma_z
    (B + B^dagger) to a primary mode of frequency Omega = Delta (resonance),
    truncated to nvib levels, which couples through its position B +
    B^dagger to an ohmic bath J = kappa w exp(-w/wc), kappa = 0.056, wc =
    10, kT = Delta; g = 0.18, dt = 0.06, Delta k_max = 12, Delta k_eff = 10,
    theta = 1e-9 (the converged settings of the paper's figure captions).
    The system basis is electronic state x the eigenbasis of the mode's
    position (where the bath coupling is diagonal): q = the position
    eigenvalues, once per electronic state; M = 2 nvib.  The mask is not
    printed in the paper: here the last nine positions fine and position 10
    (Delta k_eff = 10).  rho0 = |up><up| x the mode's thermal state.  J in
    the (pi/2) alpha w convention: alpha = 2 kappa / pi."""
    n = nvib
    Bm = np.diag(np.sqrt(np.arange(1, n, dtype=np.float64)), 1)     # annihilation, number basis
    X = Bm + Bm.T
    x, V = np.linalg.eigh(X)                                        # position eigenbasis
    Nx = V.T @ np.diag(np.arange(n, dtype=np.float64)) @ V          # B^dagger B there
    Delta, Omega, g, kT = 1.0, 1.0, 0.18, 1.0
    sx = np.array([[0.0, 1.0], [1.0, 0.0]])
    sz = np.diag([1.0, -1.0])
    H = 0.5 * Delta * np.kron(sx, np.eye(n)) + g * np.kron(sz, np.diag(x)) + Omega * np.kron(np.eye(2), Nx)
    q = tuple(float(v) for v in np.concatenate([x, x]))
    th = np.diag(np.exp(-Omega * np.arange(n) / kT))
    th = V.T @ (th / np.trace(th)) @ V
    rho0 = np.kron(np.diag([1.0, 0.0]), th)
    return Workload(
        name=f"reaction_coordinate_nvib{nvib}_dk{dkmax}",
        M=2 * n, q=q, hs=tuple(tuple(complex(v) for v in row) for row in H),
        bath=Bath(beta=1.0 / kT, ohmic_alpha=2.0 * 0.056 / math.pi, ohmic_wc=10.0),
        dt=0.06, dkmax=dkmax, mask=tuple(mask), theta=theta,
        rho0=tuple(tuple(complex(v) for v in row) for row in rho0), steps=steps)


# ---------------------------------------------------------------------------
# Small seeded random cases for tests: random Hermitian H_S, coupling
# eigenvalues and influence coefficients are drawn directly (the influence
# coefficients are an input of the path update).
# ---------------------------------------------------------------------------

def random_hermitian(rng: np.random.Generator, M: int, scale: float = 1.0) -> np.ndarray:
    a = rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))
    return scale * 0.5 * (a + a.conj().T)


def random_density_matrix(rng: np.random.Generator, M: int) -> np.ndarray:
    a = rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))
    r = a @ a.conj().T
    return r / np.trace(r).real


def random_eta(rng: np.random.Generator, n: int, scale: float = 0.05) -> np.ndarray:
    """Complex coefficients with a positive real part at lag 0 and decaying lags."""
    decay = np.exp(-0.4 * np.arange(n))
    re = scale * decay * (0.5 + rng.uniform(size=n))
    im = scale * decay * rng.normal(size=n)
    return re + 1j * im


def random_case(seed: int, M: int, dkmax: int):
    rng = np.random.default_rng(seed)
    hs = random_hermitian(rng, M)
    q = np.sort(rng.normal(size=M))
    eta = random_eta(rng, dkmax)
    rho0 = random_density_matrix(rng, M)
    dt = float(rng.uniform(0.1, 0.4))
    return dict(M=M, q=q, hs=hs, eta=eta, rho0=rho0, dt=dt, dkmax=dkmax)
