"""The step entry point that allocates nothing (qp_step_noalloc), against
the context-based qp_step.

qp_step_noalloc serves callers that cannot allocate device memory (a plug-in
inside a host program that owns the GPU memory, a real-time loop that may not
call cudaMalloc, a process under a hard memory quota): its scratch is one
fixed array inside the library.  Two calls in a row, t -> t+1 -> t+2, starting
from a stored set produced by a context, must give the same rho and the same
stored paths as two more qp_step calls on that context, within the FP64
parity tolerance of the other GPU tests.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2506_03127_gb300 import Propagator, abi, build  # noqa: E402

build.build()

TOL = 1e-10


def _summed_by_key(keys, amps):
    u, inv = np.unique(keys, return_inverse=True)
    s = np.zeros(u.size, dtype=complex)
    np.add.at(s, inv, amps)
    return u, s


@pytest.mark.parametrize("M,dkmax,mask,theta,t0,seed", [(2, 6, (0, 1, 2, 4), 1e-5, 8, 2506),
                                                         (3, 4, None, 0.0, 5, 7),
                                                         (4, 3, (0, 1), 1e-6, 4, 11)])
def test_noalloc_step_matches_context_step_twice(M, dkmax, mask, theta, t0, seed):
    case = W.random_case(seed, M, dkmax)
    p = Propagator(M, dkmax, case["dt"], case["q"], case["hs"], theta, max_paths=1 << 18)
    p.set_eta(case["eta"])
    p.set_mask(mask)
    p.set_rho0(case["rho0"])
    p.step(t0)
    keys, amps = p.export_paths()
    dev = torch.device("cuda", torch.cuda.current_device())
    cap = 1 << 18
    k_in = torch.from_numpy(keys.view(np.int64).copy()).to(dev)
    a_in = torch.from_numpy(np.stack([amps.real, amps.imag], axis=1).reshape(-1).copy()).to(dev)
    n_in = keys.size
    cfg, keep = abi.make_config(M, dkmax, case["dt"], case["q"], case["hs"], theta)
    t = t0
    for call in range(2):
        k_out = torch.empty(cap, dtype=torch.int64, device=dev)
        a_out = torch.empty(2 * cap, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        n_out, rho = abi.qp_step_noalloc(cfg, case["eta"], mask, t, k_in.data_ptr(), a_in.data_ptr(), n_in,
                                         k_out.data_ptr(), a_out.data_ptr(), cap)
        p.step(1)
        t += 1
        rho_ctx = p.rho(t, 1)[0]
        assert np.abs(rho - rho_ctx).max() <= TOL, (call, np.abs(rho - rho_ctx).max())
        kc, ac = p.export_paths()
        assert n_out == kc.size
        kn = k_out[:n_out].cpu().numpy().view(np.uint64)
        an = a_out[:2 * n_out].cpu().numpy()
        an = an[0::2] + 1j * an[1::2]
        u1, s1 = _summed_by_key(kn, an)
        u2, s2 = _summed_by_key(kc, ac)
        np.testing.assert_array_equal(u1, u2)
        assert np.abs(s1 - s2).max() <= TOL
        k_in, a_in, n_in = k_out, a_out, n_out
    p.close()


def test_noalloc_rejects_inputs_beyond_its_fixed_scratch():
    case = W.random_case(3, 2, 4)
    cfg, keep = abi.make_config(2, 4, case["dt"], case["q"], case["hs"], 0.0)
    with pytest.raises(abi.QPError) as e:
        abi.qp_step_noalloc(cfg, case["eta"], None, 3, 1 << 20, 1 << 21, (1 << 20) + 1, 1 << 22, 1 << 23, 16)
    assert e.value.status == abi.QP_ERR_ARG
    big, keepb = abi.make_config(2, 17, case["dt"], case["q"], case["hs"], 0.0)
    with pytest.raises(abi.QPError) as e2:
        abi.qp_step_noalloc(big, np.zeros(17), None, 3, 1 << 20, 1 << 21, 4, 1 << 22, 1 << 23, 16)
    assert e2.value.status == abi.QP_ERR_ARG


def _device_set(keys, amps, dev):
    k = torch.from_numpy(np.asarray(keys, dtype=np.uint64).view(np.int64).copy()).to(dev)
    a = torch.from_numpy(np.stack([np.real(amps), np.imag(amps)], axis=1).reshape(-1).copy()).to(dev)
    return k, a


def _compare_sets(k_out, a_out, n_out, kc, ac):
    kn = k_out[:n_out].cpu().numpy().view(np.uint64)
    an = a_out[:2 * n_out].cpu().numpy()
    u1, s1 = _summed_by_key(kn, an[0::2] + 1j * an[1::2])
    u2, s2 = _summed_by_key(kc, ac)
    np.testing.assert_array_equal(u1, u2)
    assert np.abs(s1 - s2).max() <= TOL


def test_noalloc_chain_from_the_initial_state_through_the_window_fill():
    """From t = 0 (one stored path per nonzero element of rho(0)) through
    the steps while the window fills, where every stored path is expanded
    on its own, into the first merging steps: each call against qp_step."""
    M, dkmax, mask, theta, steps = 2, 5, (0, 1, 3), 1e-6, 9
    case = W.random_case(19, M, dkmax)
    p = Propagator(M, dkmax, case["dt"], case["q"], case["hs"], theta, max_paths=1 << 18)
    p.set_eta(case["eta"])
    p.set_mask(mask)
    p.set_rho0(case["rho0"])
    a, b = np.nonzero(case["rho0"])
    dev = torch.device("cuda", torch.cuda.current_device())
    k_in, a_in = _device_set(a | (b << 1), case["rho0"][a, b], dev)
    n_in = a.size
    cfg, keep = abi.make_config(M, dkmax, case["dt"], case["q"], case["hs"], theta)
    cap = 1 << 16
    for t in range(steps):
        k_out = torch.empty(cap, dtype=torch.int64, device=dev)
        a_out = torch.empty(2 * cap, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        n_out, rho = abi.qp_step_noalloc(cfg, case["eta"], mask, t, k_in.data_ptr(), a_in.data_ptr(), n_in,
                                         k_out.data_ptr(), a_out.data_ptr(), cap)
        p.step(1)
        assert np.abs(rho - p.rho(t + 1, 1)[0]).max() <= TOL, t
        kc, ac = p.export_paths()
        assert n_out == kc.size
        _compare_sets(k_out, a_out, n_out, kc, ac)
        k_in, a_in, n_in = k_out, a_out, n_out
    p.close()


def test_noalloc_capacity_error_then_a_clean_call():
    """More survivors than cap_out: QP_ERR_CAPACITY with *n_out = 0.  The
    next call with room for the survivors starts from cleared scratch and
    matches qp_step."""
    M, dkmax, mask, theta, t0 = 2, 6, (0, 1, 2, 4), 1e-5, 8
    case = W.random_case(2506, M, dkmax)
    p = Propagator(M, dkmax, case["dt"], case["q"], case["hs"], theta, max_paths=1 << 18)
    p.set_eta(case["eta"])
    p.set_mask(mask)
    p.set_rho0(case["rho0"])
    p.step(t0)
    keys, amps = p.export_paths()
    dev = torch.device("cuda", torch.cuda.current_device())
    k_in, a_in = _device_set(keys, amps, dev)
    cfg, keep = abi.make_config(M, dkmax, case["dt"], case["q"], case["hs"], theta)
    eta = np.asarray(case["eta"], dtype=np.complex128)
    er, ei = np.ascontiguousarray(eta.real), np.ascontiguousarray(eta.imag)
    m = np.array(mask, dtype=np.int32)
    cap = 1 << 16
    k_out = torch.empty(cap, dtype=torch.int64, device=dev)
    a_out = torch.empty(2 * cap, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    n_out = ctypes.c_int64(-1)
    rr, ri = np.zeros(M * M), np.zeros(M * M)
    dp = ctypes.POINTER(ctypes.c_double)
    st = abi.lib.qp_step_noalloc(ctypes.byref(cfg), er.ctypes.data_as(dp), ei.ctypes.data_as(dp), eta.size,
                                 m.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), m.size, t0,
                                 ctypes.c_void_p(k_in.data_ptr()), ctypes.c_void_p(a_in.data_ptr()), keys.size,
                                 ctypes.c_void_p(k_out.data_ptr()), ctypes.c_void_p(a_out.data_ptr()), 8,
                                 ctypes.byref(n_out), rr.ctypes.data_as(dp), ri.ctypes.data_as(dp), None)
    assert st == abi.QP_ERR_CAPACITY and n_out.value == 0
    n_ok, rho = abi.qp_step_noalloc(cfg, case["eta"], mask, t0, k_in.data_ptr(), a_in.data_ptr(), keys.size,
                                    k_out.data_ptr(), a_out.data_ptr(), cap)
    p.step(1)
    assert np.abs(rho - p.rho(t0 + 1, 1)[0]).max() <= TOL
    kc, ac = p.export_paths()
    assert n_ok == kc.size
    _compare_sets(k_out, a_out, n_ok, kc, ac)
    p.close()
