"""Sharded propagation over ranks, on the CPU with gloo (world size 2 and 3).

The driver of paper_2506_03127_gb300/ranks.py (owner routing, the
all-to-all of paths with uneven counts, the all-reduce of rho) runs here
with a stand-in for libqp's local step built from the oracle: each rank
steps the paths it owns, partitions them by the owner of their next
pre-merge group (the formula qp_partition_paths states), and the exchange
goes through torch.distributed.  rho(t) summed over ranks must equal the
single-process oracle: the pre-merge groups are complete on their owners,
so sharding changes nothing but the order of sums.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

GOLDEN_MULT = 0x9E3779B97F4A7C15


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class OracleShard:
    """The rank's part of the problem stepped by the oracle (test stand-in
    for a libqp context on the merge-table engine)."""

    def __init__(self, case, mask, theta, n_ranks, rank):
        from oracle import iquapi
        self.iq = iquapi
        self.c, self.theta, self.n_ranks, self.rank = case, theta, n_ranks, rank
        self.M, self.dk = case["M"], case["dkmax"]
        P = iquapi.check_mask(range(self.dk) if mask is None else mask, self.dk)
        self.Pp = iquapi.premerge_positions(P, self.dk)
        self.U = iquapi.short_time_propagator(case["hs"], case["dt"])
        self.bs, self.b = iquapi.state_bits(self.M)
        self.pmask = np.uint64(sum(((1 << self.b) - 1) << (self.b * p) for p in self.Pp))
        self.paths = iquapi.initial_paths(case["rho0"])
        self.t = 0
        self.last_rho = None

    def start(self):
        if self.rank != 0:
            self.import_paths(*self.empty())

    def empty(self):
        return torch.empty(0, dtype=torch.int64), torch.empty(0, dtype=torch.float64)

    def step(self):
        self.t += 1
        self.paths, self.last_rho, _ = self.iq.step(self.paths, self.t, self.U, np.asarray(self.c["q"]), self.c["eta"],
                                                    self.dk, self.Pp, self.theta, self.M)

    def owners(self, keys):
        with np.errstate(over="ignore"):
            h = ((keys & self.pmask) * np.uint64(GOLDEN_MULT)) >> np.uint64(32)
        return (h % np.uint64(self.n_ranks)).astype(np.int64)

    def partition(self):
        keys = self.iq.packed_keys(self.paths.sp, self.paths.sm, self.M)
        own = self.owners(keys)
        order = np.argsort(own, kind="stable")
        counts = np.bincount(own, minlength=self.n_ranks)
        amps = np.stack([self.paths.amp.real, self.paths.amp.imag], axis=1)[order].reshape(-1)
        return (torch.from_numpy(keys[order].view(np.int64).copy()), torch.from_numpy(amps.copy()), counts)

    def import_paths(self, keys, amps):
        k = keys.numpy().view(np.uint64)
        L = min(self.t + 1, self.dk)
        sp = np.zeros((k.size, L), dtype=np.int64)
        sm = np.zeros((k.size, L), dtype=np.int64)
        for p in range(L):
            code = (k >> np.uint64(self.b * p)) & np.uint64((1 << self.b) - 1)
            sp[:, p] = (code & np.uint64((1 << self.bs) - 1)).astype(np.int64)
            sm[:, p] = (code >> np.uint64(self.bs)).astype(np.int64)
        a = amps.numpy()
        self.paths = self.iq.Paths(sp, sm, a[0::2] + 1j * a[1::2])

    def rho(self):
        return self.last_rho


CASES = [(2, 6, (0, 1, 2, 4), 1e-6, 12, 61), (3, 4, None, 1e-6, 7, 62), (2, 8, None, 0.0, 11, 63)]


def _rank(rank, world, port, out_dir, case_idx):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads as W
    from paper_2506_03127_gb300.ranks import ShardedPropagation, TorchExchange
    M, dk, mask, theta, steps, seed = CASES[case_idx]
    case = W.random_case(seed, M, dk)
    shard = OracleShard(case, mask, theta, world, rank)
    sp = ShardedPropagation(shard, TorchExchange(), case["rho0"])
    rho = np.array(sp.step(steps))
    np.save(os.path.join(out_dir, f"rho{rank}.npy"), rho)
    np.save(os.path.join(out_dir, f"kept{rank}.npy"), np.array(sp.kept))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case_idx", range(len(CASES)))
def test_sharded_propagation_equals_one_process(tmp_path, world, case_idx):
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path), case_idx), nprocs=world, join=True,
                       start_method="spawn")
    sys.path.insert(0, ROOT)
    import workloads as W
    from oracle import iquapi
    M, dk, mask, theta, steps, seed = CASES[case_idx]
    case = W.random_case(seed, M, dk)
    ref = iquapi.propagate(M, case["q"], case["hs"], case["dt"], case["eta"], dk, mask, theta, case["rho0"], steps)
    kept = sum(np.load(tmp_path / f"kept{r}.npy") for r in range(world))
    for r in range(world):
        rho = np.load(tmp_path / f"rho{r}.npy")
        np.testing.assert_allclose(rho, ref.rho, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(kept, [s.kept for s in ref.stats])
