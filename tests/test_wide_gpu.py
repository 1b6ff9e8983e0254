"""GPU: the path update with keys of up to 128 bits (qp_wide_*, M up to 8).

Each case must reproduce the oracle (FP64: rho within 1e-10, per-step
counts equal, the stored key sets equal), including windows whose keys do
not fit 64 bits (M = 8 at 11 and 12 points: the oracle pre-merges them
without packing), and agree with the narrow engines where both apply
(M <= 4).  complex64 within a stated bound.
"""
import numpy as np
import pytest

import workloads as W
from oracle import iquapi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2506_03127_gb300 import Propagator, WidePropagator, abi, build  # noqa: E402

build.build()

TOL = 1e-10


def _wide_keys_of(sp, sm):
    """Oracle paths -> (lo, hi) of the wide layout: one byte per position."""
    lo = np.zeros(sp.shape[0], dtype=np.uint64)
    hi = np.zeros(sp.shape[0], dtype=np.uint64)
    for p in range(sp.shape[1]):
        code = (sp[:, p] | (sm[:, p] << 4)).astype(np.uint64)
        if p < 8:
            lo |= code << np.uint64(8 * p)
        else:
            hi |= code << np.uint64(8 * (p - 8))
    return set(zip(lo.tolist(), hi.tolist()))


def _case(seed, M, dkmax, diag=True, scale=0.3):
    rng = np.random.default_rng(seed)
    hs = W.random_hermitian(rng, M, scale)
    if diag:   # diagonal-dominant: few significant paths (long windows at M = 8)
        hs = hs + np.diag(np.linspace(-1.0, 1.0, M))
    q = np.sort(rng.normal(size=M))
    eta = W.random_eta(rng, dkmax, 0.05)
    rho0 = W.random_density_matrix(rng, M)
    return dict(M=M, dkmax=dkmax, hs=hs, q=q, eta=eta, rho0=rho0, dt=0.2)


def _run_wide(c, mask, theta, steps, precision="fp64", max_paths=1 << 20):
    p = WidePropagator(c["M"], c["dkmax"], c["dt"], c["q"], c["hs"], theta, precision, max_paths=max_paths)
    p.set_eta(c["eta"])
    p.set_mask(mask)
    p.set_rho0(c["rho0"])
    p.step(steps)
    rho = p.rho(0, steps + 1)
    stats = p.stats(1, steps)
    keys, amps = p.export_paths()
    p.close()
    return rho, stats, keys, amps


CASES = [
    (5, 3, None, 0.0, 5, 1),
    (6, 3, (0, 1), 1e-4, 6, 2),
    (8, 2, None, 1e-3, 5, 3),
    (8, 3, (0, 1), 1e-3, 6, 4),
    (3, 4, (0, 1, 3), 1e-6, 8, 5),
    (8, 11, (0, 1, 2), 1e-3, 13, 6),           # 88-bit keys, the oracle beyond 64 bits
    (8, 12, tuple(range(10)), 1e-3, 14, 7),    # the production shape: Delta k_max 12, Delta k_eff 10
    (7, 11, (0, 1, 2, 5), 1e-4, 13, 8),
]


@pytest.mark.parametrize("M,dkmax,mask,theta,steps,seed", CASES)
def test_wide_matches_oracle(M, dkmax, mask, theta, steps, seed):
    c = _case(seed, M, dkmax, diag=dkmax > 4)
    rho, stats, keys, amps = _run_wide(c, mask, theta, steps)
    o = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, mask, theta, c["rho0"], steps)
    err = np.abs(rho - o.rho).max()
    assert err <= TOL, err
    assert [s[3] for s in stats] == [s.kept for s in o.stats]
    assert [s[1] for s in stats] == [s.groups for s in o.stats]
    got = set(zip(keys[:, 0].tolist(), keys[:, 1].tolist()))
    assert got == _wide_keys_of(o.paths.sp, o.paths.sm)
    if dkmax >= 11:
        assert int(keys[:, 1].max()) > 0   # keys past 64 bits are in use


@pytest.mark.parametrize("M,dkmax,mask,theta,steps", [(2, 8, (0, 1, 2, 5), 1e-6, 14), (3, 5, None, 1e-7, 9),
                                                      (4, 3, (0, 1), 1e-5, 6)])
def test_wide_agrees_with_narrow_engine(M, dkmax, mask, theta, steps):
    """M <= 4: the wide context and the merge-table engine on the same
    problem give the same rho, counts and key sets (keys converted from the
    narrow packing)."""
    c = _case(40 + M, M, dkmax, diag=False)
    rho, stats, keys, _ = _run_wide(c, mask, theta, steps)
    p = Propagator(M, dkmax, c["dt"], c["q"], c["hs"], theta, "fp64", engine="hash", max_paths=1 << 20)
    p.set_eta(c["eta"])
    p.set_mask(mask)
    p.set_rho0(c["rho0"])
    p.step(steps)
    rn = p.rho(0, steps + 1)
    sn = p.stats(1, steps)
    kn, _ = p.export_paths()
    p.close()
    assert np.abs(rho - rn).max() <= 1e-12
    assert [s[3] for s in stats] == [s[3] for s in sn]
    bs, b = iquapi.state_bits(M)
    L = min(steps + 1, dkmax)
    sp = np.zeros((kn.size, L), dtype=np.int64)
    sm = np.zeros((kn.size, L), dtype=np.int64)
    for pos in range(L):
        code = (kn >> np.uint64(b * pos)) & np.uint64((1 << b) - 1)
        sp[:, pos] = (code & np.uint64((1 << bs) - 1)).astype(np.int64)
        sm[:, pos] = (code >> np.uint64(bs)).astype(np.int64)
    assert set(zip(keys[:, 0].tolist(), keys[:, 1].tolist())) == _wide_keys_of(sp, sm)


def test_wide_complex64_within_bound():
    """complex64 amplitudes (FP32 history exponent with Kahan additions,
    FP32 hi/lo propagator table, FP64 merge sums and rho) against the FP64
    oracle: within 1e-5 on an 8-level case through the window fill and
    merging steps."""
    c = _case(6, 8, 11)
    steps = 13
    rho, stats, _, _ = _run_wide(c, (0, 1, 2), 1e-3, steps, precision="c64")
    o = iquapi.propagate(8, c["q"], c["hs"], c["dt"], c["eta"], 11, (0, 1, 2), 1e-3, c["rho0"], steps)
    assert np.abs(rho - o.rho).max() <= 1e-5
    kept_o = [s.kept for s in o.stats]
    assert all(abs(a[3] - b) <= max(2, b // 100) for a, b in zip(stats, kept_o))


def test_wide_capacity_error_and_restart():
    c = _case(9, 6, 3, diag=False)
    p = WidePropagator(6, 3, c["dt"], c["q"], c["hs"], 0.0, "fp64", max_paths=256)
    p.set_eta(c["eta"])
    p.set_mask(None)
    p.set_rho0(c["rho0"])
    p.step(3)
    with pytest.raises(abi.QPError) as e:
        p.current()
    assert e.value.status == abi.QP_ERR_CAPACITY
    with pytest.raises(abi.QPError) as e:
        p.step(1)
    assert e.value.status == abi.QP_ERR_STATE
    pure = np.zeros((6, 6), dtype=complex)
    pure[0, 0] = 1.0
    p.set_rho0(pure)                                  # 36 children at the first step
    p.step(1)
    assert p.current() == (1, 36)
    p.close()


def test_wide_mask_limits():
    """P' beyond ten positions (a 64-bit group key of 6 bits each) is refused;
    so is a rho0 before a usable mask on a long window."""
    c = _case(10, 8, 13)
    p = WidePropagator(8, 13, c["dt"], c["q"], c["hs"], 1e-3, "fp64", max_paths=1 << 16)
    p.set_eta(c["eta"])
    with pytest.raises(abi.QPError) as e:
        p.set_rho0(c["rho0"])                         # the default full mask: P' of 12 positions
    assert e.value.status == abi.QP_ERR_STATE
    with pytest.raises(abi.QPError) as e:
        p.set_mask(tuple(range(13)))
    assert e.value.status == abi.QP_ERR_ARG
    p.set_mask((0, 1, 2, 3))
    p.set_rho0(c["rho0"])
    p.step(2)
    p.close()


@pytest.mark.parametrize("precision,tol,tie", [("fp64", TOL, None), ("c64", 1e-5, 1e-6)])
def test_wide_reaction_coordinate_matches_oracle(precision, tol, tie, monkeypatch):
    """The reaction-coordinate model of Sec. 4.3 (M = 8, the production mask
    at Delta k_max = 12: 96-bit keys; its position eigenvalues come in equal
    pairs, so the children's influence factors are tabulated per distinct
    coupling difference), at theta = 1e-4 so that the oracle runs it; eta
    from each side's own quadrature (they agree to 1e-13).  This model has
    group members whose weights agree to between 1e-12 and 1e-9: the
    complex64 form, whose tie window is 1e-6 (reading R11), is compared with
    the oracle run with the same window (the oracle with its FP64 window of
    1e-12 resolves those groups by weight and differs from either by 2e-3)."""
    if tie is not None:
        monkeypatch.setattr(iquapi, "TIE_REL", tie)
    from oracle.bath import eta_coefficients
    from paper_2506_03127_gb300 import eta_from_bath

    w = W.reaction_coordinate(theta=1e-4)
    steps = 14
    p = WidePropagator(w.M, w.dkmax, w.dt, w.q, w.hs_array(), w.theta, precision, max_paths=1 << 20)
    p.set_eta(eta_from_bath(w.bath, w.dt, w.dkmax))
    p.set_mask(w.mask)
    p.set_rho0(w.rho0_array())
    p.step(steps)
    rho = p.rho(0, steps + 1)
    stats = p.stats(1, steps)
    keys, _ = p.export_paths()
    p.close()
    o = iquapi.propagate(w.M, w.q, w.hs_array(), w.dt, eta_coefficients(w.bath, w.dt, w.dkmax), w.dkmax, w.mask,
                         w.theta, w.rho0_array(), steps)
    assert np.abs(rho - o.rho).max() <= tol
    if precision == "fp64":
        assert [s[3] for s in stats] == [s.kept for s in o.stats]
        assert set(zip(keys[:, 0].tolist(), keys[:, 1].tolist())) == _wide_keys_of(o.paths.sp, o.paths.sm)
        assert int(keys[:, 1].max()) > 0
