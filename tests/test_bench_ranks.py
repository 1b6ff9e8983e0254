"""The bench's multi-rank path (independent replicas, one per rank, no data
exchange): the whole-job time is the slowest rank's and the units are summed
over ranks.  Run here as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate_over_ranks(10.0 + 5.0 * rank, 1000.0 * (rank + 1))
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{t} {u}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_sum_the_units(tmp_path):
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        t, u = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert t == 15.0 and u == 3000.0


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(7.5, 42) == (7.5, 42.0)
