"""Sharded propagation of one problem over several ranks (one GPU each).

The paper distributes the stored paths over MPI processes and merges them
across processes by sequential broadcast rounds (Sec. 3.2).  Here every
stored path lives on the rank that owns its next pre-merge group (a hash of
the masked key, computed by libqp's qp_partition_paths), so each rank's
pre-merge sees complete groups and a step needs one exchange of paths (an
all-to-all) and one sum of the ranks' parts of rho(t) (an all-reduce of
M*M values):

    local step (pre-merge, extension, filter, the rank's part of rho(t))
    -> partition the stored set by owner -> all-to-all -> import
    -> rho(t) = sum over ranks.

This module holds the driver and the exchanges (marshalling only): the
local step, the partition and the import run in libqp.  ``TorchExchange``
uses torch.distributed (NCCL for device tensors, gloo for host tensors);
``step_in_process`` runs several shards held by one process (one GPU), the
exchange done by copies between the shards' buffers, no collective and no
kernel that waits on another.
"""
from __future__ import annotations

import numpy as np


class ContextShard:
    """One rank's part: a libqp context on the merge-table engine."""

    def __init__(self, prop, n_ranks, rank):
        import torch
        from . import abi
        self.torch, self.abi = torch, abi
        self.p = prop
        self.n_ranks, self.rank = n_ranks, rank
        self.M = prop.M
        self.c64 = prop._cfg.precision == abi.QP_C64
        self.t = 0

    def start(self):
        """t = 0: the initial paths stay on rank 0 only (each context set
        one path per nonzero element of rho(0))."""
        if self.rank != 0:
            self.import_paths(*self.empty())
        self.t = 0

    def empty(self):
        torch = self.torch
        dev = self.p.device
        return (torch.empty(0, dtype=torch.int64, device=dev),
                torch.empty(0, dtype=torch.float32 if self.c64 else torch.float64, device=dev))

    def step(self):
        self.p.step(1)
        self.t += 1

    def partition(self):
        """The stored set grouped by owner rank: (keys, amps (re, im)
        interleaved), counts per rank."""
        torch = self.torch
        n = self.p.current()[1]
        cap = max(n, 1)
        keys = torch.empty(cap, dtype=torch.int64, device=self.p.device)
        amps = torch.empty(2 * cap, dtype=torch.float32 if self.c64 else torch.float64, device=self.p.device)
        counts = self.abi.qp_partition_paths(self.p.ctx, self.n_ranks, keys.data_ptr(), amps.data_ptr(), cap)
        return keys[:n], amps[:2 * n], counts

    def import_paths(self, keys, amps):
        keys = keys.contiguous()
        amps = amps.contiguous()
        self.abi.qp_import_paths(self.p.ctx, keys.data_ptr(), amps.data_ptr(), keys.numel())

    def rho(self):
        """This rank's part of rho(t) after the last step (M x M complex)."""
        return self.p.rho(self.t, 1)[0]


class TorchExchange:
    """Exchange through torch.distributed (the default process group or
    ``group``): counts, then keys and amplitudes, by all_to_all_single;
    rho by all_reduce."""

    def __init__(self, group=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.group = torch, dist, group
        self.size = dist.get_world_size(group)

    def all_to_all(self, keys, amps, counts):
        torch, dist = self.torch, self.dist
        dev = keys.device
        c_in = torch.as_tensor(np.asarray(counts, dtype=np.int64), device=dev)
        c_out = torch.empty_like(c_in)
        dist.all_to_all_single(c_out, c_in, group=self.group)
        rc = c_out.cpu().tolist()
        sc = [int(x) for x in counts]
        rk = torch.empty(sum(rc), dtype=keys.dtype, device=dev)
        ra = torch.empty(2 * sum(rc), dtype=amps.dtype, device=dev)
        dist.all_to_all_single(rk, keys.contiguous(), rc, sc, group=self.group)
        dist.all_to_all_single(ra, amps.contiguous(), [2 * x for x in rc], [2 * x for x in sc], group=self.group)
        return rk, ra

    def all_reduce(self, rho):
        torch = self.torch
        r = torch.as_tensor(np.ascontiguousarray(rho, dtype=np.complex128).view(np.float64))
        dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
        r = r.to(dev)
        self.dist.all_reduce(r, group=self.group)
        return r.cpu().numpy().view(np.complex128).reshape(np.shape(rho))


class ShardedPropagation:
    """The step loop of one rank: local step, partition, exchange, import,
    rho(t) summed over ranks."""

    def __init__(self, shard, exchange, rho0):
        self.shard, self.ex = shard, exchange
        self.rho_hist = [np.asarray(rho0, dtype=np.complex128)]
        self.kept = []
        shard.start()
        self._route()

    def _route(self):
        keys, amps, counts = self.shard.partition()
        rk, ra = self.ex.all_to_all(keys, amps, counts)
        self.shard.import_paths(rk, ra)
        return int(rk.numel())

    def step(self, nsteps=1):
        for _ in range(nsteps):
            self.shard.step()
            self.rho_hist.append(self.ex.all_reduce(self.shard.rho()))
            self.kept.append(self._route())
        return self.rho_hist


def step_in_process(shards, rho0, nsteps):
    """Several shards of one problem held by one process (on one GPU): the
    same steps as ShardedPropagation, the all-to-all done by copies between
    the shards' tensors and rho(t) summed on the host.  Returns rho(0..n)
    and the stored paths per shard after each step."""
    import torch

    def route():
        parts = [s.partition() for s in shards]
        n = len(shards)
        kept = []
        for dst, s in enumerate(shards):
            ks, as_ = [], []
            for keys, amps, counts in parts:
                off = np.concatenate([[0], np.cumsum(counts)])
                ks.append(keys[off[dst]:off[dst + 1]])
                as_.append(amps[2 * off[dst]:2 * off[dst + 1]])
            k = torch.cat(ks) if ks else s.empty()[0]
            a = torch.cat(as_) if as_ else s.empty()[1]
            s.import_paths(k, a)
            kept.append(int(k.numel()))
        assert n == len(kept)
        return kept

    for s in shards:
        s.start()
    route()
    rho = [np.asarray(rho0, dtype=np.complex128)]
    kept = []
    for _ in range(nsteps):
        for s in shards:
            s.step()
        rho.append(sum(s.rho() for s in shards))
        kept.append(route())
    return np.array(rho), kept
