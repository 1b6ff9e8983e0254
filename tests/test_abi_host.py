"""Host-side checks of libqp that need no GPU: the library loads, exports
every symbol include/qp.h declares, validates configurations, and its host
eta quadrature agrees with the oracle's (an independent formula: box
integrals vs second differences of Q(t))."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2506_03127_gb300 import build as qp_build

qp_build.build()

from paper_2506_03127_gb300 import abi  # noqa: E402
import workloads as W  # noqa: E402
from oracle import bath as B  # noqa: E402

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "qp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qp_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(abi.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def declared_prototypes():
    """{name: number of parameters} of every function include/qp.h declares."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\b(qp_[a-z0-9_]+)\s*\(([^;{}]*?)\)\s*;", src, flags=re.S):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_matches_every_declared_prototype():
    """The ctypes binding gives every entry point of the C ABI as many
    argument types as its prototype has parameters."""
    protos = declared_prototypes()
    assert set(protos) == set(declared_functions())
    wrong = {}
    for name, n in protos.items():
        f = getattr(abi.lib, name)
        if f.argtypes is None or len(f.argtypes) != n:
            wrong[name] = (n, None if f.argtypes is None else len(f.argtypes))
    assert not wrong, wrong


def test_version_and_status_strings():
    assert abi.lib.qp_version() >= 100
    assert abi.lib.qp_status_string(abi.QP_ERR_CAPACITY).decode() == "capacity exceeded"


def _cfg(**kw):
    args = dict(M=2, dkmax=8, dt=0.25, q=[1, -1], hs=np.array([[0, 0.5], [0.5, 0]]), theta=0.0)
    args.update(kw)
    return abi.make_config(**args)


def test_workspace_size_grows_with_capacity():
    c1, k1 = _cfg(max_paths=1 << 12)
    c2, k2 = _cfg(max_paths=1 << 16)
    assert abi.qp_workspace_size(c2) > abi.qp_workspace_size(c1) > 0


@pytest.mark.parametrize("precision,amp_bytes", [(abi.QP_C64, 8), (abi.QP_FP64, 16)])
def test_stream_only_workspace_holds_little_beyond_the_path_buffers(precision, amp_bytes):
    """With the stream engine asked for, the merge table is not allocated:
    per path, two buffers of key + amplitude and a small look-back share."""
    n = 1 << 22
    cs, ks = _cfg(max_paths=n, precision=precision, engine=abi.QP_ENGINE_STREAM)
    ca, ka = _cfg(max_paths=n, precision=precision, engine=abi.QP_ENGINE_AUTO)
    ws, wa = abi.qp_workspace_size(cs), abi.qp_workspace_size(ca)
    assert 2 * (8 + amp_bytes) * n <= ws <= (2 * (8 + amp_bytes) + 1) * n
    assert wa > ws + 16 * n   # AUTO keeps the merge table as well


@pytest.mark.parametrize("bad", [dict(M=1), dict(M=5), dict(dkmax=0), dict(M=2, dkmax=33), dict(M=3, q=[1, 0, -1],
                                 hs=np.eye(3), dkmax=17), dict(dt=-1.0), dict(theta=-1.0), dict(max_paths=0),
                                 dict(hs=np.array([[0, 0.5], [0.2, 0]])), dict(precision=7), dict(engine=9)])
def test_invalid_configs_rejected(bad):
    cfg, keep = _cfg(**bad)
    n = ctypes.c_size_t()
    assert abi.lib.qp_workspace_size(ctypes.byref(cfg), ctypes.byref(n)) == abi.QP_ERR_ARG


def test_create_rejects_small_or_misaligned_workspace():
    cfg, keep = _cfg()
    h = ctypes.c_void_p()
    need = abi.qp_workspace_size(cfg)
    assert abi.lib.qp_create(ctypes.byref(cfg), ctypes.c_void_p(256 * 1000), need - 256, None,
                             ctypes.byref(h)) == abi.QP_ERR_OOM
    assert abi.lib.qp_create(ctypes.byref(cfg), ctypes.c_void_p(256 * 1000 + 8), need, None,
                             ctypes.byref(h)) == abi.QP_ERR_ARG
    assert abi.lib.qp_create(ctypes.byref(cfg), None, need, None, ctypes.byref(h)) == abi.QP_ERR_ARG


@pytest.mark.parametrize("w", [W.SPIN_BOSON_OHMIC_DK8, W.SPIN_BOSON_STRUCTURED_DK16, W.CHAIN3_STRUCTURED_DK12,
                               W.TLS_OHMIC_FULL_DK14, W.resonance_sweep(3)[2]], ids=lambda w: w.name)
def test_library_eta_matches_oracle(w):
    el = abi.qp_eta_from_bath(w.bath, w.dt, w.dkmax)
    eo = B.eta_coefficients(w.bath, w.dt, w.dkmax)
    np.testing.assert_allclose(el, eo, rtol=0, atol=1e-13)


def test_eta_from_bath_rejects_bad_bath():
    b = abi.qp_bath(beta=-1.0, ohmic_alpha=0.1, ohmic_wc=5.0)
    re, im = np.zeros(4), np.zeros(4)
    assert abi.lib.qp_eta_from_bath(ctypes.byref(b), 0.1, 4, abi._ptr(re), abi._ptr(im)) == abi.QP_ERR_ARG


@pytest.mark.parametrize("w", [W.SPIN_BOSON_OHMIC_DK8, W.SPIN_BOSON_STRUCTURED_DK16], ids=lambda w: w.name)
def test_library_Q_at_half_steps_matches_oracle(w):
    """Q(j dt/2), the input of the symmetric splitting, by the library's host
    quadrature against the oracle's (scipy) quadrature."""
    n = 2 * w.dkmax + 2
    ql = abi.qp_Q_from_bath(w.bath, 0.5 * w.dt, n)
    qo = np.concatenate([[0.0], B.Q_of_t(w.bath, 0.5 * w.dt * np.arange(1, n))])
    np.testing.assert_allclose(ql, qo, rtol=0, atol=1e-13)


def _wcfg(**kw):
    M = kw.pop("M", 8)
    args = dict(M=M, dkmax=12, dt=0.06, q=np.arange(M, dtype=float), hs=np.eye(M), theta=1e-9, max_paths=1 << 16)
    args.update(kw)
    return abi.make_config(**args)


def test_wide_workspace_size_follows_capacity_and_precision():
    """Wide keys: the workspace grows with max_paths; complex64 amplitudes
    save 8 bytes per entry in each of the two ping-pong amplitude buffers;
    per path at least the two buffers of a 16-byte key and an FP64
    amplitude plus a merge table of 32-byte slots for twice the groups."""
    (a, ka), (b, kb), (c, kc) = _wcfg(max_paths=1 << 12), _wcfg(), _wcfg(precision=abi.QP_C64)
    sa, sb, sc = abi.qp_wide_workspace_size(a), abi.qp_wide_workspace_size(b), abi.qp_wide_workspace_size(c)
    assert 0 < sa < sb
    assert sb - sc == 2 * 8 * (1 << 16)
    big, kbig = _wcfg(max_paths=1 << 20)
    assert abi.qp_wide_workspace_size(big) >= (2 * (16 + 16) + 2 * 32) * (1 << 20)


@pytest.mark.parametrize("bad", [dict(M=1, q=[0.0], hs=np.eye(1)), dict(M=9, q=np.arange(9.0), hs=np.eye(9)),
                                 dict(dkmax=0), dict(dkmax=17), dict(dt=0.0), dict(theta=-1.0), dict(precision=5),
                                 dict(max_paths=8), dict(n_inst=2), dict(scheme=abi.QP_POSTMERGE)],
                         ids=lambda d: ",".join(d))
def test_wide_config_checks(bad):
    cfg, keep = _wcfg(**bad)
    n = ctypes.c_size_t()
    assert abi.lib.qp_wide_workspace_size(ctypes.byref(cfg), ctypes.byref(n)) == abi.QP_ERR_ARG


def test_wide_create_rejects_small_or_missing_workspace():
    """Refused before any device call: a workspace one byte short
    (QP_ERR_OOM) or none (QP_ERR_ARG); no context is returned."""
    cfg, keep = _wcfg()
    need = abi.qp_wide_workspace_size(cfg)
    h = ctypes.c_void_p()
    assert abi.lib.qp_wide_create(ctypes.byref(cfg), ctypes.c_void_p(256 * 1000), need - 1, None,
                                  ctypes.byref(h)) == abi.QP_ERR_OOM
    assert abi.lib.qp_wide_create(ctypes.byref(cfg), None, need, None, ctypes.byref(h)) == abi.QP_ERR_ARG
    assert h.value is None


def test_mlp_workspace_size_and_checks():
    """The surrogate's workspace grows with the batch and holds at least the
    FP32 parameters, their gradient and the two Adam moments; dimensions
    out of range, a short or misaligned workspace are refused before any
    device call."""
    s1, s2 = abi.qp_mlp_workspace_size(258, 256, 8, 64), abi.qp_mlp_workspace_size(258, 256, 8, 4096)
    npar = 258 * 256 + 256 + 256 * 256 + 256 + 256 * 8 + 8
    assert 4 * 4 * npar <= s1 < s2
    n = ctypes.c_size_t()
    for bad in [(0, 256, 8, 64), (258, 0, 8, 64), (258, 256, 0, 64), (258, 256, 8, 0), (5000, 256, 8, 64),
                (258, 256, 8, (1 << 20) + 1)]:
        assert abi.lib.qp_mlp_workspace_size(*bad, ctypes.byref(n)) == abi.QP_ERR_ARG
    h = ctypes.c_void_p()
    assert abi.lib.qp_mlp_create(258, 256, 8, 64, ctypes.c_void_p(256 * 1000), s1 - 1, None,
                                 ctypes.byref(h)) == abi.QP_ERR_OOM
    assert abi.lib.qp_mlp_create(258, 256, 8, 64, ctypes.c_void_p(256 * 1000 + 8), s1, None,
                                 ctypes.byref(h)) == abi.QP_ERR_ARG


def test_capacity_limits_as_documented():
    """max_paths up to 2^40; beyond 2^30 paths the merge table needs an
    explicit max_groups (at most 2^30) unless the stream engine, which has
    none, is asked for; the post-merging order keeps max_paths below 2^32."""
    def size(**kw):
        cfg, keep = _cfg(**kw)
        n = ctypes.c_size_t()
        st = abi.lib.qp_workspace_size(ctypes.byref(cfg), ctypes.byref(n))
        return st, n.value

    assert size(max_paths=1 << 32, engine=abi.QP_ENGINE_AUTO)[0] == abi.QP_ERR_ARG
    assert size(max_paths=1 << 32, engine=abi.QP_ENGINE_HASH, max_groups=1 << 28)[0] == abi.QP_OK
    assert size(max_paths=1 << 32, engine=abi.QP_ENGINE_HASH, max_groups=(1 << 30) + 1)[0] == abi.QP_ERR_ARG
    st, n = size(max_paths=1 << 40, engine=abi.QP_ENGINE_STREAM, precision=abi.QP_C64)
    assert st == abi.QP_OK and n >= 2 * (8 + 8) * (1 << 40)       # 64-bit sizes, no overflow
    assert size(max_paths=(1 << 40) + 1, engine=abi.QP_ENGINE_STREAM)[0] == abi.QP_ERR_ARG
    assert size(max_paths=1 << 32, scheme=abi.QP_POSTMERGE)[0] == abi.QP_ERR_ARG
    assert size(max_paths=(1 << 32) - 1, scheme=abi.QP_POSTMERGE, max_groups=1 << 20)[0] == abi.QP_OK
    assert size(rho_history=(1 << 24) + 1)[0] == abi.QP_ERR_ARG


EXTREME_BATHS = [dict(beta=100.0, ohmic_alpha=0.1, ohmic_wc=5.0), dict(beta=0.05, ohmic_alpha=0.1, ohmic_wc=5.0),
                 dict(beta=5.0, ohmic_alpha=0.1, ohmic_wc=50.0), dict(beta=5.0, ohmic_alpha=0.1, ohmic_wc=0.5),
                 dict(beta=50.0, res_w0=1.0, res_gamma=0.01, res_lambda=0.1),
                 dict(beta=0.2, res_w0=3.0, res_gamma=0.5, res_lambda=0.3)]


# (the hot broad resonance at the long step only at dt = 0.02: the oracle's
# adaptive quadrature takes tens of seconds there)
@pytest.mark.parametrize("kw,dt", [(kw, dt) for kw in EXTREME_BATHS for dt in (0.02, 0.25)
                                   if not (kw["beta"] == 0.2 and dt == 0.25)],
                         ids=lambda x: ",".join(f"{k}={v}" for k, v in x.items()) if isinstance(x, dict) else str(x))
def test_library_eta_matches_oracle_at_extreme_baths(kw, dt):
    """Cold and hot baths, wide and narrow cut-offs, a sharp and a broad
    resonance: the library's quadrature and the oracle's agree to 1e-11
    relative (measured at most 3e-12 for eta)."""
    bath = W.Bath(**kw)
    lib = abi.qp_eta_from_bath(bath, dt, 16)
    orc = B.eta_coefficients(bath, dt, 16)
    assert np.abs(lib - orc).max() <= 1e-11 * np.abs(orc).max()
    # Q at half steps (the symmetric splitting's input): measured at most 8e-13
    ql = abi.qp_Q_from_bath(bath, 0.5 * dt, 35)
    qo = B.Q_of_t(bath, 0.5 * dt * np.arange(35))
    assert np.abs(ql - qo).max() <= 1e-11 * np.abs(qo).max()
