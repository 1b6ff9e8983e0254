"""GPU: the symmetric Trotter splitting (qp_set_end_points) on the
merge-table engine against the oracle's symmetric-splitting propagation.

The oracle's version is pinned by an independent path sum over intervals
and by exact pure dephasing (tests/test_oracle_pins.py).  Bar: FP64 rho(t)
within 1e-10, survivor counts equal and the surviving key set bit-exact;
complex64 within 1e-6 on a physical bath.  Q at half steps from a random sequence (any values
define coefficients both sides must agree on) and from a physical bath.
"""
import numpy as np
import pytest

import workloads as W
from oracle import bath as B
from oracle import iquapi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2506_03127_gb300 import Propagator, abi, build  # noqa: E402

build.build()

TOL = 1e-10


def random_Qh(seed, n):
    rng = np.random.default_rng(seed)
    j = np.arange(n)
    return (0.02 * j ** 1.5 * (1 + 0.1 * rng.normal(size=n))
            + 1j * 0.01 * j ** 2 * (1 + 0.1 * rng.normal(size=n))) * (j > 0)


def eta_from_Qh(Qh, dkmax):
    eta = np.zeros(dkmax, dtype=complex)
    eta[0] = Qh[2]
    for d in range(1, dkmax):
        eta[d] = Qh[2 * d + 2] - 2 * Qh[2 * d] + Qh[2 * d - 2]
    return eta


def run_sym(case, mask, theta, steps, Qh, precision="fp64"):
    M, dk = case["M"], case["dkmax"]
    p = Propagator(M, dk, case["dt"], case["q"], case["hs"], theta, precision, "auto", max_paths=1 << 20)
    p.set_eta(eta_from_Qh(Qh, dk))
    p.set_end_points(Qh)
    p.set_mask(mask)
    p.set_rho0(case["rho0"])
    p.step(steps)
    p.sync()
    assert p.tuning().engine == abi.QP_ENGINE_HASH     # the splitting runs on the merge-table engine
    out = (p.rho(0, steps + 1), p.stats(1, steps), *p.export_paths())
    p.close()
    return out


@pytest.mark.parametrize("M,dkmax,mask,theta,steps,seed", [
    (2, 1, None, 0.0, 6, 1), (2, 3, None, 0.0, 9, 2), (2, 6, (0, 1, 2, 4), 1e-5, 14, 3), (2, 8, None, 1e-6, 12, 4),
    (3, 3, None, 1e-6, 7, 5), (3, 4, (0, 1, 3), 1e-5, 9, 6), (4, 3, (0, 1), 1e-4, 6, 7)])
def test_symmetric_splitting_matches_oracle(M, dkmax, mask, theta, steps, seed):
    case = W.random_case(seed, M, dkmax)
    Qh = random_Qh(seed, 2 * dkmax + 3)
    rho, stats, keys, amps = run_sym(case, mask, theta, steps, Qh)
    o = iquapi.propagate(M, case["q"], case["hs"], case["dt"], eta_from_Qh(Qh, dkmax), dkmax, mask, theta,
                         case["rho0"], steps, Qh=Qh)
    assert np.abs(rho - o.rho).max() <= TOL, np.abs(rho - o.rho).max()
    assert [s[3] for s in stats] == [s.kept for s in o.stats]
    if not any(s.near_tie or s.near_theta for s in o.stats):
        ko = iquapi.packed_keys(o.paths.sp, o.paths.sm, M)
        np.testing.assert_array_equal(np.sort(keys), np.sort(ko))


def test_symmetric_splitting_with_a_bath_and_pure_dephasing():
    """The structured bath's Q at half steps from the library's quadrature;
    with H_S = 0 the decoherence function is exact within the memory."""
    w = W.SPIN_BOSON_STRUCTURED_DK16
    dk, steps = 10, 9
    Qh = abi.qp_Q_from_bath(w.bath, 0.5 * w.dt, 2 * dk + 3)
    q = np.array([1.0, -1.0])
    rho0 = np.full((2, 2), 0.5, dtype=complex)
    case = dict(M=2, dkmax=dk, dt=w.dt, q=q, hs=np.zeros((2, 2)), rho0=rho0)
    rho, *_ = run_sym(case, None, 0.0, steps, Qh)
    Qt = B.Q_of_t(w.bath, w.dt * np.arange(1, steps + 1))
    for n in range(1, steps + 1):
        Q = Qt[n - 1]
        expect = rho0 * np.exp(-(q[:, None] - q[None, :]) * (q[:, None] * Q - q[None, :] * np.conj(Q)))
        assert np.abs(rho[n] - expect).max() <= 1e-12
    # a full propagation with tunnelling against the oracle
    case = dict(M=2, dkmax=dk, dt=w.dt, q=q, hs=w.hs_array(), rho0=w.rho0_array())
    rho, *_ = run_sym(case, (0, 1, 2, 3, 4, 5, 7), 1e-8, 24, Qh)
    o = iquapi.propagate(2, q, w.hs_array(), w.dt, eta_from_Qh(Qh, dk), dk, (0, 1, 2, 3, 4, 5, 7), 1e-8,
                         w.rho0_array(), 24, Qh=Qh)
    assert np.abs(rho - o.rho).max() <= TOL
    # complex64 (the random sequences above reach amplitudes of order 10 with
    # exponents far from physical ones; the bath's stay below 1)
    rho_c, *_ = run_sym(case, (0, 1, 2, 3, 4, 5, 7), 1e-8, 24, Qh, precision="c64")
    assert np.abs(rho_c - o.rho).max() <= 1e-6, np.abs(rho_c - o.rho).max()


def test_set_eta_returns_to_the_right_box_reading():
    case = W.random_case(8, 2, 4)
    Qh = random_Qh(8, 11)
    p = Propagator(2, 4, case["dt"], case["q"], case["hs"], 0.0, max_paths=1 << 14)
    p.set_eta(case["eta"])
    p.set_end_points(Qh)
    p.set_eta(case["eta"])
    p.set_rho0(case["rho0"])
    p.step(6)
    o = iquapi.propagate(2, case["q"], case["hs"], case["dt"], case["eta"], 4, None, 0.0, case["rho0"], 6)
    assert np.abs(p.rho(0, 7) - o.rho).max() <= TOL
    p.close()
    p = Propagator(2, 4, case["dt"], case["q"], case["hs"], 0.0, engine="stream", max_paths=1 << 14)
    p.set_eta(case["eta"])
    with pytest.raises(abi.QPError) as e:
        p.set_end_points(Qh)
    assert e.value.status == abi.QP_ERR_STATE
    p.close()
