"""Learned surrogate of rho(t): orchestration of libqp's MLP kernels.

Every computation (window assembly, forward and backward passes, Adam,
rollout) runs in libqp; this module holds device buffers (PyTorch tensors),
loops and bookkeeping only.  The paper has no counterpart: the surrogate
extends the propagation of the path update in time, and the path update is
its check at checkpoints and its fallback.

Features of one prediction: the last L values of rho(t) (8 reals each: Re,
Im of rho_00, rho_01, rho_10, rho_11) and the instance's bath parameters
(w0, 10 lambda); output: (rho(t) - rho(t-1)) * out_scale, added to rho(t-1)
and projected onto Hermitian, positive semidefinite matrices of the same trace.
"""
from __future__ import annotations

import numpy as np

from . import abi


def rho_to_device(torch, rho, device):
    """rho [T][n_inst][2][2] complex -> device double tensor [T][n_inst][4][2]."""
    r = np.ascontiguousarray(np.asarray(rho, dtype=np.complex128).reshape(rho.shape[0], rho.shape[1], 4))
    return torch.from_numpy(r.view(np.float64).copy()).to(device)


def bath_features(ws):
    return np.array([[w.bath.res_w0, 10.0 * w.bath.res_lambda] for w in ws], dtype=np.float32)


class MLP:
    def __init__(self, d_in, width, d_out, max_batch, device=None, stream=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.d_in, self.width, self.d_out, self.max_batch = d_in, width, d_out, max_batch
        nb = abi.qp_mlp_workspace_size(d_in, width, d_out, max_batch)
        self.ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.h = abi.qp_mlp_create(d_in, width, d_out, max_batch, self.ws.data_ptr(), nb, self.stream.cuda_stream)
        self.n_params = abi.qp_mlp_num_params(self.h)

    def init(self, seed=0, out_gain=0.1):
        rng = np.random.default_rng(seed)
        d, w, o = self.d_in, self.width, self.d_out
        parts = [rng.normal(size=(d, w)) * np.sqrt(1.0 / d), np.zeros(w), rng.normal(size=(w, w)) * np.sqrt(1.0 / w),
                 np.zeros(w), rng.normal(size=(w, o)) * np.sqrt(1.0 / w) * out_gain, np.zeros(o)]
        self.set_params(np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32))

    def set_params(self, p):
        abi.qp_mlp_set_params(self.h, p)

    def params(self):
        return abi.qp_mlp_get_params(self.h, self.n_params)

    def forward(self, x):
        y = self.torch.empty((x.shape[0], self.d_out), dtype=self.torch.float32, device=self.device)
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        abi.qp_mlp_forward(self.h, x.data_ptr(), x.shape[0], y.data_ptr())
        self.stream.synchronize()
        return y

    def gradients(self, x, t):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        return abi.qp_mlp_gradients(self.h, x.data_ptr(), t.data_ptr(), x.shape[0], self.n_params)

    def train_step(self, x, t, lr, want_loss=False):
        return abi.qp_mlp_train_step(self.h, x.data_ptr(), t.data_ptr(), x.shape[0], lr, want_loss=want_loss)

    def close(self):
        if getattr(self, "h", None):
            self.stream.synchronize()   # queued work still uses the workspace
            abi.lib.qp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    def __init__(self, L=32, width=256, n_par=2, out_scale=10.0, max_batch=8192, device=None):
        import torch
        self.torch = torch
        self.L, self.n_par, self.out_scale = L, n_par, out_scale
        self.net = MLP(8 * L + n_par, width, 8, max_batch, device)
        self.device = self.net.device

    def windows(self, rho_dev, n_inst, par_dev, inst0, ninst, t_begin, t_end):
        rows = ninst * (t_end - t_begin)
        x = self.torch.empty((rows, 8 * self.L + self.n_par), dtype=self.torch.float32, device=self.device)
        t = self.torch.empty((rows, 8), dtype=self.torch.float32, device=self.device)
        abi.qp_surrogate_windows(rho_dev.data_ptr(), n_inst, self.L, par_dev.data_ptr(), self.n_par, t_begin, t_end,
                                 inst0, ninst, self.out_scale, x.data_ptr(), t.data_ptr(), self.net.stream.cuda_stream)
        return x, t

    def fit(self, rho, par, train=(0, 48), epochs=3000, lr=2e-3, lr_end=2e-5, seed=0, log_every=0):
        """rho [T+1][n_inst][2][2] (host, from the path update), par [n_inst][n_par]."""
        torch = self.torch
        T1, n_inst = rho.shape[0], rho.shape[1]
        rho_dev = rho_to_device(torch, rho, self.device)
        par_dev = torch.from_numpy(np.ascontiguousarray(par, dtype=np.float32)).to(self.device)
        torch.cuda.synchronize()
        x, t = self.windows(rho_dev, n_inst, par_dev, train[0], train[1] - train[0], self.L, T1)
        self.net.init(seed)
        hist = []
        for e in range(epochs):
            frac = e / max(1, epochs - 1)
            lr_e = lr * (lr_end / lr) ** frac
            want = log_every and (e % log_every == 0 or e == epochs - 1)
            loss = self.net.train_step(x, t, lr_e, want_loss=bool(want))
            if want:
                hist.append((e, loss))
        self.net.stream.synchronize()
        return hist

    def rollout(self, rho_init, par, T_total, mode="auto"):
        """rho_init [n][L][2][2] (steps 0..L-1), par [n][n_par] -> rho [n][T_total][2][2].
        mode: "auto" (one block for all steps where it fits), "graph" (CUDA
        graphs of step kernels) or "fused" (qp_mlp_set_rollout_mode)."""
        torch = self.torch
        n = rho_init.shape[0]
        h = np.zeros((n, T_total, 8), dtype=np.float32)
        ri = np.asarray(rho_init, dtype=np.complex128).reshape(n, self.L, 4)
        h[:, :self.L, 0::2] = ri.real
        h[:, :self.L, 1::2] = ri.imag
        hist = torch.from_numpy(h).to(self.device)
        par_dev = torch.from_numpy(np.ascontiguousarray(par, dtype=np.float32)).to(self.device)
        xb = torch.empty((n, 8 * self.L + self.n_par), dtype=torch.float32, device=self.device)
        yb = torch.empty((n, 8), dtype=torch.float32, device=self.device)
        torch.cuda.synchronize()
        abi.qp_mlp_set_rollout_mode(self.net.h, {"auto": abi.QP_ROLLOUT_AUTO, "graph": abi.QP_ROLLOUT_GRAPH,
                                                 "fused": abi.QP_ROLLOUT_FUSED}[mode])
        abi.qp_surrogate_rollout(self.net.h, hist.data_ptr(), n, T_total, self.L, par_dev.data_ptr(), self.n_par,
                                 self.L, T_total, self.out_scale, xb.data_ptr(), yb.data_ptr())
        self.net.stream.synchronize()
        out = hist.cpu().numpy().astype(np.float64)
        return (out[..., 0::2] + 1j * out[..., 1::2]).reshape(n, T_total, 2, 2)


def checkpoint_errors(rho_sur, rho_plain, checkpoints, trace_tol=0.05, eig_tol=0.02):
    """Check the surrogate at checkpoints against the plain path.  An instance
    falls back to the plain path (its result is the plain one) when at any
    checkpoint its trace deviates from the plain trace by more than
    trace_tol or rho has an eigenvalue below -eig_tol.  Returns (errors of
    the combined result per checkpoint, errors of the raw surrogate per
    checkpoint, fallback mask).  rho_sur [n][T][2][2], rho_plain [T][n][2][2]."""
    n = rho_sur.shape[0]
    fallback = np.zeros(n, dtype=bool)
    raw = {}
    for c in checkpoints:
        rs, rp = rho_sur[:, c], rho_plain[c]
        tr_s = np.trace(rs, axis1=1, axis2=2).real
        tr_p = np.trace(rp, axis1=1, axis2=2).real
        ev = np.linalg.eigvalsh(0.5 * (rs + np.conj(np.swapaxes(rs, 1, 2))))
        fallback |= (np.abs(tr_s - tr_p) > trace_tol) | (ev.min(axis=1) < -eig_tol)
        raw[int(c)] = float(np.abs(rs - rp).max())
    combined = {}
    for c in checkpoints:
        d = np.abs(rho_sur[:, c] - rho_plain[c]).reshape(n, -1).max(axis=1)
        combined[int(c)] = float(np.where(fallback, 0.0, d).max())
    return combined, raw, fallback


def truncated_memory_baselines(ws, T, rho_ref, checkpoints, dks=(1, 2, 3, 4, 5, 6, 7), precision="c64",
                               max_paths=1 << 22):
    """The cheaper settings of the path update itself, for the comparison
    the surrogate has to win: the same instances propagated with a shorter
    memory (Delta k_max = dk; dk = 1 is the Markov map), each batched and
    timed over the T - 1 steps (CUDA-synchronised wall time), with the
    largest |rho - rho_ref| over instances and entries at each checkpoint.
    rho_ref [T][n][2][2] from the full-memory path.  Returns {dk: dict}."""
    import time
    from dataclasses import replace

    import torch

    from . import batch_from_workloads
    out = {}
    for dk in dks:
        wsx = [replace(w, dkmax=dk, mask=None) for w in ws]
        q = batch_from_workloads(wsx, precision=precision, max_paths=max_paths)
        q.step(3)      # graphs captured before timing
        q.sync()
        q.set_rho0(wsx[0].rho0_array())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q.step(T - 1)
        q.sync()
        dt = time.perf_counter() - t0
        r = q.rho(0, T)
        q.close()
        errs = {int(c): float(np.abs(r[c] - rho_ref[c]).max()) for c in checkpoints}
        out[dk] = {"seconds": dt, "us_per_step": 1e6 * dt / (T - 1), "err_max": max(errs.values()), "errors": errs}
    return out
