"""ctypes binding of libqp (include/qp.h): same names, argument marshalling only.

Every computation of the path update runs in the library's CUDA kernels.
Importing this module loads the in-tree libqp.so and fails loudly if it is
missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqp.so")

QP_OK, QP_ERR_ARG, QP_ERR_OOM, QP_ERR_CUDA, QP_ERR_CAPACITY, QP_ERR_TIMEOUT, QP_ERR_STATE = range(7)
QP_FP64, QP_C64 = 0, 1
QP_ENGINE_AUTO, QP_ENGINE_HASH, QP_ENGINE_STREAM = 0, 1, 2
QP_LAUNCH_GRAPH, QP_LAUNCH_PERSISTENT = 0, 1
QP_PREMERGE, QP_POSTMERGE = 0, 1
QP_ROLLOUT_AUTO, QP_ROLLOUT_GRAPH, QP_ROLLOUT_FUSED = 0, 1, 2

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)


class qp_config(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("dkmax", ctypes.c_int), ("dt", ctypes.c_double),
                ("q", _dp), ("hs_re", _dp), ("hs_im", _dp),
                ("precision", ctypes.c_int), ("engine", ctypes.c_int), ("theta", ctypes.c_double),
                ("max_paths", ctypes.c_int64), ("max_groups", ctypes.c_int64), ("rho_history", ctypes.c_int),
                ("n_inst", ctypes.c_int), ("scheme", ctypes.c_int)]


class qp_tuning(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("insert_blocks_per_sm", ctypes.c_int), ("expand_blocks_per_sm", ctypes.c_int),
                ("persistent_blocks", ctypes.c_int), ("graph_steps", ctypes.c_int), ("table_log2", ctypes.c_int),
                ("engine", ctypes.c_int), ("stream_tile", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class qp_bath(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("ohmic_alpha", ctypes.c_double), ("ohmic_wc", ctypes.c_double),
                ("res_w0", ctypes.c_double), ("res_gamma", ctypes.c_double), ("res_lambda", ctypes.c_double)]


class qp_step_stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int64), ("groups", ctypes.c_int64), ("extended", ctypes.c_int64),
                ("kept", ctypes.c_int64), ("intermediate", ctypes.c_int64)]


class QPError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{lib.qp_status_string(status).decode()} ({status}): {msg}")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libqp.so not built at {LIB_PATH}; run `python -m paper_2506_03127_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "qp_version": (ctypes.c_int, []),
        "qp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "qp_workspace_size": (ctypes.c_int, [ctypes.POINTER(qp_config), ctypes.POINTER(ctypes.c_size_t)]),
        "qp_create": (ctypes.c_int, [ctypes.POINTER(qp_config), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_void_p)]),
        "qp_destroy": (None, [ctypes.c_void_p]),
        "qp_eta_from_bath": (ctypes.c_int, [ctypes.POINTER(qp_bath), ctypes.c_double, ctypes.c_int, _dp, _dp]),
        "qp_set_eta": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, ctypes.c_int]),
        "qp_set_mask": (ctypes.c_int, [ctypes.c_void_p, _ip, ctypes.c_int]),
        "qp_set_rho0": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
        "qp_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
        "qp_sync": (ctypes.c_int, [ctypes.c_void_p]),
        "qp_current": (ctypes.c_int, [ctypes.c_void_p, _i64p, _i64p]),
        "qp_read_rho": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, _dp, _dp]),
        "qp_read_rho_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]),
        "qp_read_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                         ctypes.POINTER(qp_step_stats)]),
        "qp_export_paths": (ctypes.c_int, [ctypes.c_void_p, _u64p, _dp, ctypes.c_int64, _i64p]),
        "qp_profile_steps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int]),
        "qp_set_eta_instance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp, _dp, ctypes.c_int]),
        "qp_read_instance_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _i64p]),
        "qp_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
        "qp_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
        "qp_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, _dp]),
        "qp_test_stall_barrier": (ctypes.c_int, [ctypes.c_void_p]),
        "qp_test_stall_lookback": (ctypes.c_int, [ctypes.c_void_p]),
        "qp_Q_from_bath": (ctypes.c_int, [ctypes.POINTER(qp_bath), ctypes.c_double, ctypes.c_int, _dp, _dp]),
        "qp_set_end_points": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, ctypes.c_int]),
        "qp_partition_paths": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_int64, _i64p]),
        "qp_import_paths": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
        "qp_test_widen": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
        "qp_mlp_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_size_t)]),
        "qp_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
        "qp_mlp_destroy": (None, [ctypes.c_void_p]),
        "qp_mlp_num_params": (ctypes.c_int, [ctypes.c_void_p, _i64p]),
        "qp_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
        "qp_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
        "qp_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
        "qp_mlp_gradients": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_float), _dp]),
        "qp_mlp_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                             ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _dp]),
        "qp_mlp_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
        "qp_surrogate_windows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
        "qp_surrogate_rollout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
        "qp_mlp_set_rollout_mode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
        "qp_wide_workspace_size": (ctypes.c_int, [ctypes.POINTER(qp_config), ctypes.POINTER(ctypes.c_size_t)]),
        "qp_wide_create": (ctypes.c_int, [ctypes.POINTER(qp_config), ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
        "qp_wide_destroy": (None, [ctypes.c_void_p]),
        "qp_wide_set_eta": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, ctypes.c_int]),
        "qp_wide_set_mask": (ctypes.c_int, [ctypes.c_void_p, _ip, ctypes.c_int]),
        "qp_wide_set_rho0": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
        "qp_wide_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
        "qp_wide_current": (ctypes.c_int, [ctypes.c_void_p, _i64p, _i64p]),
        "qp_wide_read_rho": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, _dp, _dp]),
        "qp_wide_read_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                              ctypes.POINTER(qp_step_stats)]),
        "qp_wide_export_paths": (ctypes.c_int, [ctypes.c_void_p, _u64p, _dp, ctypes.c_int64, _i64p]),
        "qp_wide_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
        "qp_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
        "qp_step_noalloc": (ctypes.c_int, [ctypes.POINTER(qp_config), _dp, _dp, ctypes.c_int, _ip, ctypes.c_int,
                                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, _i64p, _dp, _dp,
                                           ctypes.c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _arr(x, dtype=np.float64):
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def check(status, ctx=None):
    if status != QP_OK:
        msg = lib.qp_last_error(ctx).decode() if ctx else ""
        raise QPError(status, msg)


def make_config(M, dkmax, dt, q, hs, theta=0.0, precision=QP_FP64, engine=QP_ENGINE_AUTO,
                max_paths=1 << 20, max_groups=0, rho_history=4096, n_inst=1, scheme=QP_PREMERGE):
    """qp_config plus the numpy arrays it points into (keep both alive)."""
    q = _arr(q)
    hs = np.asarray(hs, dtype=np.complex128)
    hre, him = _arr(hs.real), _arr(hs.imag)
    cfg = qp_config(M=M, dkmax=dkmax, dt=dt, q=_ptr(q), hs_re=_ptr(hre), hs_im=_ptr(him),
                    precision=precision, engine=engine, theta=theta, max_paths=max_paths,
                    max_groups=max_groups, rho_history=rho_history, n_inst=n_inst, scheme=scheme)
    return cfg, (q, hre, him)


def qp_workspace_size(cfg) -> int:
    n = ctypes.c_size_t(0)
    check(lib.qp_workspace_size(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def qp_create(cfg, d_workspace: int, nbytes: int, stream: int):
    h = ctypes.c_void_p()
    check(lib.qp_create(ctypes.byref(cfg), ctypes.c_void_p(d_workspace), nbytes, ctypes.c_void_p(stream),
                        ctypes.byref(h)))
    return h


def qp_destroy(ctx):
    lib.qp_destroy(ctx)


def qp_eta_from_bath(bath, dt: float, n: int) -> np.ndarray:
    b = qp_bath(beta=bath.beta, ohmic_alpha=bath.ohmic_alpha, ohmic_wc=bath.ohmic_wc,
                res_w0=bath.res_w0, res_gamma=bath.res_gamma, res_lambda=bath.res_lambda)
    re, im = np.zeros(n), np.zeros(n)
    check(lib.qp_eta_from_bath(ctypes.byref(b), dt, n, _ptr(re), _ptr(im)))
    return re + 1j * im


def qp_set_eta(ctx, eta):
    eta = np.asarray(eta, dtype=np.complex128)
    re, im = _arr(eta.real), _arr(eta.imag)
    check(lib.qp_set_eta(ctx, _ptr(re), _ptr(im), eta.size), ctx)


def qp_set_mask(ctx, positions):
    if positions is None:
        check(lib.qp_set_mask(ctx, None, 0), ctx)
        return
    p = _arr(list(positions), np.int32)
    check(lib.qp_set_mask(ctx, _ptr(p, _ip), p.size), ctx)


def qp_set_rho0(ctx, rho0):
    r = np.asarray(rho0, dtype=np.complex128)
    re, im = _arr(r.real), _arr(r.imag)
    check(lib.qp_set_rho0(ctx, _ptr(re), _ptr(im)), ctx)


def qp_step(ctx, nsteps: int = 1):
    check(lib.qp_step(ctx, nsteps), ctx)


def qp_sync(ctx):
    check(lib.qp_sync(ctx), ctx)


def qp_current(ctx):
    t, n = ctypes.c_int64(), ctypes.c_int64()
    check(lib.qp_current(ctx, ctypes.byref(t), ctypes.byref(n)), ctx)
    return t.value, n.value


def qp_read_rho(ctx, t0: int, count: int, M: int, n_inst: int = 1) -> np.ndarray:
    """rho(t0 .. t0+count-1): shape (count, M, M), or (count, n_inst, M, M) for a batch."""
    re, im = np.zeros(count * n_inst * M * M), np.zeros(count * n_inst * M * M)
    check(lib.qp_read_rho(ctx, t0, count, _ptr(re), _ptr(im)), ctx)
    r = (re + 1j * im)
    return r.reshape(count, M, M) if n_inst == 1 else r.reshape(count, n_inst, M, M)


def qp_read_rho_async(ctx, t0: int, count: int, dst_addr: int):
    """Enqueue the copy of rho(t0 .. t0+count-1) to host memory at dst_addr
    (complex128 [count][n_inst][M*M]); in place after qp_sync."""
    check(lib.qp_read_rho_async(ctx, t0, count, ctypes.c_void_p(dst_addr)), ctx)


def qp_set_eta_instance(ctx, inst: int, eta):
    eta = np.asarray(eta, dtype=np.complex128)
    re, im = _arr(eta.real), _arr(eta.imag)
    check(lib.qp_set_eta_instance(ctx, inst, _ptr(re), _ptr(im), eta.size), ctx)


def qp_read_instance_counts(ctx, t: int, n_inst: int) -> np.ndarray:
    kept = np.zeros(n_inst, dtype=np.int64)
    check(lib.qp_read_instance_counts(ctx, t, _ptr(kept, _i64p)), ctx)
    return kept


def qp_get_tuning(ctx) -> qp_tuning:
    t = qp_tuning()
    check(lib.qp_get_tuning(ctx, ctypes.byref(t)), ctx)
    return t


def qp_set_tuning(ctx, t: qp_tuning):
    check(lib.qp_set_tuning(ctx, ctypes.byref(t)), ctx)


def qp_autotune(ctx, trial_steps: int = 8, use_cache: bool = True):
    t = qp_tuning()
    ms = ctypes.c_double()
    check(lib.qp_autotune(ctx, trial_steps, 1 if use_cache else 0, ctypes.byref(t), ctypes.byref(ms)), ctx)
    return t, ms.value


def qp_test_stall_barrier(ctx):
    check(lib.qp_test_stall_barrier(ctx), ctx)


def qp_Q_from_bath(bath, h: float, n: int) -> np.ndarray:
    """Q(j h), j = 0 .. n-1 (host quadrature in libqp)."""
    b = qp_bath(beta=bath.beta, ohmic_alpha=bath.ohmic_alpha, ohmic_wc=bath.ohmic_wc, res_w0=bath.res_w0,
                res_gamma=bath.res_gamma, res_lambda=bath.res_lambda)
    re, im = np.zeros(n), np.zeros(n)
    check(lib.qp_Q_from_bath(ctypes.byref(b), h, n, _ptr(re), _ptr(im)))
    return re + 1j * im


def qp_set_end_points(ctx, Qh):
    Qh = np.asarray(Qh, dtype=np.complex128)
    re, im = _arr(Qh.real), _arr(Qh.imag)
    check(lib.qp_set_end_points(ctx, _ptr(re), _ptr(im), Qh.size), ctx)


def qp_test_stall_lookback(ctx):
    check(lib.qp_test_stall_lookback(ctx), ctx)


def qp_partition_paths(ctx, n_ranks: int, d_keys: int, d_amps: int, cap: int):
    """Stored set grouped by owner rank into device buffers; counts per rank."""
    counts = np.zeros(n_ranks, dtype=np.int64)
    check(lib.qp_partition_paths(ctx, n_ranks, ctypes.c_void_p(d_keys), ctypes.c_void_p(d_amps), cap,
                                 _ptr(counts, _i64p)), ctx)
    return counts


def qp_import_paths(ctx, d_keys: int, d_amps: int, n: int):
    check(lib.qp_import_paths(ctx, ctypes.c_void_p(d_keys), ctypes.c_void_p(d_amps), n), ctx)


def qp_test_widen(in_ptr: int, out_ptr: int, n: int, stream: int = 0):
    """Device FP32 -> FP64 widening of the step kernels over n entries."""
    check(lib.qp_test_widen(in_ptr, out_ptr, n, stream), None)



def qp_read_stats(ctx, t0: int, count: int):
    arr = (qp_step_stats * count)()
    check(lib.qp_read_stats(ctx, t0, count, arr), ctx)
    return [(s.t, s.groups, s.extended, s.kept, s.intermediate) for s in arr]


def qp_export_paths(ctx, cap: int):
    keys = np.zeros(cap, dtype=np.uint64)
    amps = np.zeros(2 * cap, dtype=np.float64)
    n = ctypes.c_int64()
    check(lib.qp_export_paths(ctx, _ptr(keys, _u64p), _ptr(amps), cap, ctypes.byref(n)), ctx)
    k = n.value
    return keys[:k].copy(), amps[0:2 * k:2] + 1j * amps[1:2 * k:2]


def qp_profile_steps(ctx, nsteps: int) -> np.ndarray:
    """Per-kernel milliseconds summed over nsteps steps (insert, tie-break, expand, finalise)."""
    ms = np.zeros(4)
    check(lib.qp_profile_steps(ctx, nsteps, _ptr(ms), 4), ctx)
    return ms


def qp_last_error(ctx) -> str:
    return lib.qp_last_error(ctx).decode()


def qp_step_noalloc(cfg, eta, mask, t, d_keys_in, d_amps_in, n_in, d_keys_out, d_amps_out, cap_out, stream=0):
    """One step without allocation or context (see include/qp.h).  Device
    buffers are passed as integer addresses; returns (n_out, rho(t+1))."""
    f = lib.qp_step_noalloc
    M = cfg.M
    eta = np.asarray(eta, dtype=np.complex128)
    er, ei = _arr(eta.real), _arr(eta.imag)
    m = None if mask is None else _arr(list(mask), np.int32)
    n_out = ctypes.c_int64()
    rr, ri = np.zeros(M * M), np.zeros(M * M)
    check(f(ctypes.byref(cfg), _ptr(er), _ptr(ei), eta.size, None if m is None else _ptr(m, _ip),
            0 if m is None else m.size, t, ctypes.c_void_p(d_keys_in), ctypes.c_void_p(d_amps_in), n_in,
            ctypes.c_void_p(d_keys_out), ctypes.c_void_p(d_amps_out), cap_out, ctypes.byref(n_out),
            _ptr(rr), _ptr(ri), ctypes.c_void_p(stream)))
    return n_out.value, (rr + 1j * ri).reshape(M, M)


# ----------------------------------------------------------------- surrogate MLP

_fp = ctypes.POINTER(ctypes.c_float)


def mcheck(status, m=None):
    if status != QP_OK:
        raise QPError(status, lib.qp_mlp_last_error(m).decode() if m else "")


def qp_mlp_workspace_size(d_in, width, d_out, max_batch) -> int:
    n = ctypes.c_size_t()
    mcheck(lib.qp_mlp_workspace_size(d_in, width, d_out, max_batch, ctypes.byref(n)))
    return n.value


def qp_mlp_create(d_in, width, d_out, max_batch, d_ws, nbytes, stream):
    h = ctypes.c_void_p()
    mcheck(lib.qp_mlp_create(d_in, width, d_out, max_batch, ctypes.c_void_p(d_ws), nbytes, ctypes.c_void_p(stream),
                             ctypes.byref(h)))
    return h


def qp_mlp_num_params(m) -> int:
    n = ctypes.c_int64()
    mcheck(lib.qp_mlp_num_params(m, ctypes.byref(n)), m)
    return n.value


def qp_mlp_set_params(m, params):
    p = _arr(params, np.float32)
    mcheck(lib.qp_mlp_set_params(m, _ptr(p, _fp)), m)


def qp_mlp_get_params(m, n):
    p = np.zeros(n, dtype=np.float32)
    mcheck(lib.qp_mlp_get_params(m, _ptr(p, _fp)), m)
    return p


def qp_mlp_forward(m, d_x, batch, d_y):
    mcheck(lib.qp_mlp_forward(m, ctypes.c_void_p(d_x), batch, ctypes.c_void_p(d_y)), m)


def qp_mlp_gradients(m, d_x, d_t, batch, n):
    g = np.zeros(n, dtype=np.float32)
    loss = ctypes.c_double()
    mcheck(lib.qp_mlp_gradients(m, ctypes.c_void_p(d_x), ctypes.c_void_p(d_t), batch, _ptr(g, _fp),
                                ctypes.byref(loss)), m)
    return loss.value, g


def qp_mlp_train_step(m, d_x, d_t, batch, lr, beta1=0.9, beta2=0.999, eps=1e-8, want_loss=False):
    loss = ctypes.c_double()
    mcheck(lib.qp_mlp_train_step(m, ctypes.c_void_p(d_x), ctypes.c_void_p(d_t), batch, lr, beta1, beta2, eps,
                                 ctypes.byref(loss) if want_loss else None), m)
    return loss.value if want_loss else None


def qp_surrogate_windows(d_rho, n_inst, L, d_par, n_par, t_begin, t_end, inst0, ninst_used, out_scale, d_x, d_t,
                         stream):
    check(lib.qp_surrogate_windows(ctypes.c_void_p(d_rho), n_inst, L, ctypes.c_void_p(d_par), n_par, t_begin, t_end,
                                   inst0, ninst_used, out_scale, ctypes.c_void_p(d_x), ctypes.c_void_p(d_t),
                                   ctypes.c_void_p(stream)))


def qp_mlp_set_rollout_mode(m, mode: int):
    mcheck(lib.qp_mlp_set_rollout_mode(m, mode), m)


def qp_surrogate_rollout(m, d_hist, n, T, L, d_par, n_par, t_from, t_to, out_scale, d_xbuf, d_ybuf):
    mcheck(lib.qp_surrogate_rollout(m, ctypes.c_void_p(d_hist), n, T, L, ctypes.c_void_p(d_par), n_par, t_from, t_to,
                                    out_scale, ctypes.c_void_p(d_xbuf), ctypes.c_void_p(d_ybuf)), m)


# ---------------------------------------------------------------- wide keys (M up to 8, 128-bit keys)

def wcheck(status, w=None):
    if status != QP_OK:
        raise QPError(status, lib.qp_wide_last_error(w).decode() if w else "")


def qp_wide_workspace_size(cfg) -> int:
    n = ctypes.c_size_t()
    wcheck(lib.qp_wide_workspace_size(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def qp_wide_create(cfg, d_workspace: int, nbytes: int, stream: int):
    h = ctypes.c_void_p()
    wcheck(lib.qp_wide_create(ctypes.byref(cfg), ctypes.c_void_p(d_workspace), nbytes, ctypes.c_void_p(stream),
                              ctypes.byref(h)))
    return h


def qp_wide_set_eta(w, eta):
    e = np.ascontiguousarray(np.asarray(eta, dtype=np.complex128))
    re, im = np.ascontiguousarray(e.real), np.ascontiguousarray(e.imag)
    wcheck(lib.qp_wide_set_eta(w, _ptr(re), _ptr(im), e.size), w)


def qp_wide_set_mask(w, positions):
    if positions is None:
        wcheck(lib.qp_wide_set_mask(w, None, 0), w)
        return
    p = np.ascontiguousarray(np.asarray(positions, dtype=np.int32))
    wcheck(lib.qp_wide_set_mask(w, _ptr(p, _ip), p.size), w)


def qp_wide_set_rho0(w, rho0):
    r = np.asarray(rho0, dtype=np.complex128)
    re, im = np.ascontiguousarray(r.real.ravel()), np.ascontiguousarray(r.imag.ravel())
    wcheck(lib.qp_wide_set_rho0(w, _ptr(re), _ptr(im)), w)


def qp_wide_step(w, nsteps: int):
    wcheck(lib.qp_wide_step(w, nsteps), w)


def qp_wide_current(w):
    t, n = ctypes.c_int64(), ctypes.c_int64()
    wcheck(lib.qp_wide_current(w, ctypes.byref(t), ctypes.byref(n)), w)
    return t.value, n.value


def qp_wide_read_rho(w, t0: int, count: int, M: int) -> np.ndarray:
    re, im = np.zeros(count * M * M), np.zeros(count * M * M)
    wcheck(lib.qp_wide_read_rho(w, t0, count, _ptr(re), _ptr(im)), w)
    return (re + 1j * im).reshape(count, M, M)


def qp_wide_read_stats(w, t0: int, count: int):
    arr = (qp_step_stats * count)()
    wcheck(lib.qp_wide_read_stats(w, t0, count, arr), w)
    return [(s.t, s.groups, s.extended, s.kept, s.intermediate) for s in arr]


def qp_wide_export_paths(w, cap: int):
    """(keys [n, 2] uint64 as (lo, hi), amplitudes [n] complex128)."""
    keys = np.zeros(2 * cap, dtype=np.uint64)
    amps = np.zeros(2 * cap, dtype=np.float64)
    n = ctypes.c_int64()
    wcheck(lib.qp_wide_export_paths(w, _ptr(keys, _u64p), _ptr(amps), cap, ctypes.byref(n)), w)
    k = n.value
    return keys[:2 * k].reshape(k, 2).copy(), amps[0:2 * k:2] + 1j * amps[1:2 * k:2]
