"""GB300-native MACGIC-iQUAPI per-step path update.

The propagation runs in libqp (hand-written sm_103a CUDA behind the C ABI of
include/qp.h).  This package holds the ctypes binding (``abi``), the build
script (``build``) and ``Propagator``, a convenience wrapper that takes the
device workspace and the CUDA stream from PyTorch.  PyTorch is used only for
device memory and streams.
"""
from __future__ import annotations

import importlib

import numpy as np

__all__ = ["abi", "Propagator", "WidePropagator", "eta_from_bath", "batch_from_workloads"]


def _abi():
    return importlib.import_module(".abi", __name__)


def __getattr__(name):
    # the binding loads libqp.so; import it on first use so that the build
    # script (a submodule) can run before the library exists
    if name == "abi":
        return importlib.import_module(".abi", __name__)
    raise AttributeError(name)


def eta_from_bath(bath, dt: float, n: int) -> np.ndarray:
    """Influence coefficients eta_0..eta_{n-1} (host FP64 quadrature in libqp)."""
    return _abi().qp_eta_from_bath(bath, dt, n)


class Propagator:
    """One propagation context: owns a device workspace tensor and a stream."""

    def __init__(self, M, dkmax, dt, q, hs, theta=0.0, precision="fp64", engine="auto",
                 max_paths=1 << 20, max_groups=0, rho_history=4096, device=None, stream=None, n_inst=1,
                 scheme="pre"):
        import torch
        from . import abi
        if not torch.cuda.is_available():
            raise RuntimeError("Propagator needs a CUDA device")
        self.M = M
        self.dkmax = dkmax
        self.n_inst = n_inst
        prec = {"fp64": abi.QP_FP64, "c64": abi.QP_C64}[precision]
        eng = {"auto": abi.QP_ENGINE_AUTO, "hash": abi.QP_ENGINE_HASH, "stream": abi.QP_ENGINE_STREAM}[engine]
        sch = {"pre": abi.QP_PREMERGE, "post": abi.QP_POSTMERGE}[scheme]
        self._cfg, self._keep = abi.make_config(M, dkmax, dt, q, hs, theta, prec, eng, max_paths, max_groups,
                                                rho_history, n_inst, sch)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self.nbytes = _abi().qp_workspace_size(self._cfg)
            self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
            self.ctx = _abi().qp_create(self._cfg, self.workspace.data_ptr(), self.nbytes, self.stream.cuda_stream)

    @classmethod
    def from_workload(cls, w, precision="fp64", engine="auto", max_paths=1 << 20, max_groups=0, **kw):
        p = cls(w.M, w.dkmax, w.dt, w.q, w.hs_array(), w.theta, precision, engine, max_paths, max_groups, **kw)
        p.set_eta(eta_from_bath(w.bath, w.dt, w.dkmax))
        p.set_mask(w.mask)
        p.set_rho0(w.rho0_array())
        return p

    def set_eta(self, eta):
        _abi().qp_set_eta(self.ctx, eta)

    def set_end_points(self, Qh):
        """Symmetric Trotter splitting from Q at multiples of dt/2 (see qp.h)."""
        _abi().qp_set_end_points(self.ctx, Qh)

    def set_mask(self, positions):
        _abi().qp_set_mask(self.ctx, positions)

    def set_rho0(self, rho0):
        _abi().qp_set_rho0(self.ctx, rho0)

    def step(self, nsteps=1):
        _abi().qp_step(self.ctx, nsteps)

    def sync(self):
        _abi().qp_sync(self.ctx)

    def current(self):
        return _abi().qp_current(self.ctx)

    def rho(self, t0, count=1):
        """rho(t0..t0+count-1): (count, M, M), or (count, n_inst, M, M) for a batch."""
        return _abi().qp_read_rho(self.ctx, t0, count, self.M, self.n_inst)

    def rho_async(self, t0, out, count=1):
        """Enqueue the copy of rho(t0 .. t0+count-1) into out, a contiguous
        page-locked complex128 tensor of at least count * n_inst * M * M
        elements (torch.empty(..., dtype=torch.complex128, pin_memory=True));
        the values are in place after sync()."""
        import torch

        need = count * self.n_inst * self.M * self.M
        if out.dtype != torch.complex128 or not out.is_contiguous() or out.numel() < need or out.device.type != "cpu":
            raise ValueError("out: a contiguous host complex128 tensor of at least %d elements" % need)
        _abi().qp_read_rho_async(self.ctx, t0, count, out.data_ptr())

    def set_eta_instance(self, inst, eta):
        _abi().qp_set_eta_instance(self.ctx, inst, eta)

    def instance_counts(self, t):
        return _abi().qp_read_instance_counts(self.ctx, t, self.n_inst)

    def tuning(self):
        return _abi().qp_get_tuning(self.ctx)

    def set_tuning(self, **kw):
        t = _abi().qp_get_tuning(self.ctx)
        for k, v in kw.items():
            setattr(t, k, v)
        _abi().qp_set_tuning(self.ctx, t)

    def autotune(self, trial_steps=8, use_cache=True):
        return _abi().qp_autotune(self.ctx, trial_steps, use_cache)

    def stats(self, t0, count=1):
        return _abi().qp_read_stats(self.ctx, t0, count)

    def profile(self, nsteps):
        """Run nsteps steps kernel by kernel; per-kernel milliseconds (CUDA events)."""
        return _abi().qp_profile_steps(self.ctx, nsteps)

    def export_paths(self, cap=None):
        if cap is None:
            cap = self.current()[1]
        return _abi().qp_export_paths(self.ctx, cap)

    def close(self):
        if getattr(self, "ctx", None):
            # work still queued on the context's stream uses the workspace,
            # which PyTorch may hand out again once this object is gone
            self.stream.synchronize()
            _abi().qp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_from_workloads(ws, precision="c64", max_paths=1 << 22, engine="auto", **kw):
    """One batched Propagator over instances that differ only in their bath
    (e.g. workloads.resonance_sweep): eta per instance from libqp.  "auto"
    takes the stream engine when P' is a prefix of the window."""
    w0 = ws[0]
    for w in ws[1:]:
        if (w.M, w.q, w.hs, w.dt, w.dkmax, w.mask, w.theta, w.rho0) != (w0.M, w0.q, w0.hs, w0.dt, w0.dkmax, w0.mask,
                                                                         w0.theta, w0.rho0):
            raise ValueError("batched instances must share everything but the bath")
    p = Propagator(w0.M, w0.dkmax, w0.dt, w0.q, w0.hs_array(), w0.theta, precision, engine, max_paths,
                   n_inst=len(ws), **kw)
    p.set_eta(eta_from_bath(w0.bath, w0.dt, w0.dkmax))
    for i, w in enumerate(ws):
        p.set_eta_instance(i, eta_from_bath(w.bath, w.dt, w.dkmax))
    p.set_mask(w0.mask)
    p.set_rho0(w0.rho0_array())
    return p


class WidePropagator:
    """The path update with keys of up to 128 bits (M up to 8, windows up to
    16 points): a qp_wide context (see qp.h) with its device workspace and
    stream from PyTorch.  Single problems, pre-merging order."""

    def __init__(self, M, dkmax, dt, q, hs, theta=0.0, precision="fp64", max_paths=1 << 20, max_groups=0,
                 rho_history=4096, device=None, stream=None):
        import torch
        from . import abi
        if not torch.cuda.is_available():
            raise RuntimeError("WidePropagator needs a CUDA device")
        self.M, self.dkmax = M, dkmax
        prec = {"fp64": abi.QP_FP64, "c64": abi.QP_C64}[precision]
        self._cfg, self._keep = abi.make_config(M, dkmax, dt, q, hs, theta, prec, abi.QP_ENGINE_HASH, max_paths,
                                                max_groups, rho_history, 1, abi.QP_PREMERGE)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self.nbytes = abi.qp_wide_workspace_size(self._cfg)
            self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
            self.ctx = abi.qp_wide_create(self._cfg, self.workspace.data_ptr(), self.nbytes, self.stream.cuda_stream)

    def set_eta(self, eta):
        _abi().qp_wide_set_eta(self.ctx, eta)

    def set_mask(self, positions):
        _abi().qp_wide_set_mask(self.ctx, positions)

    def set_rho0(self, rho0):
        _abi().qp_wide_set_rho0(self.ctx, rho0)

    def step(self, nsteps=1):
        _abi().qp_wide_step(self.ctx, nsteps)

    def current(self):
        return _abi().qp_wide_current(self.ctx)

    def rho(self, t0, count=1):
        return _abi().qp_wide_read_rho(self.ctx, t0, count, self.M)

    def stats(self, t0, count=1):
        return _abi().qp_wide_read_stats(self.ctx, t0, count)

    def export_paths(self, cap=None):
        if cap is None:
            cap = self.current()[1]
        return _abi().qp_wide_export_paths(self.ctx, cap)

    def close(self):
        if getattr(self, "ctx", None):
            self.stream.synchronize()   # queued work still uses the workspace
            _abi().lib.qp_wide_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
