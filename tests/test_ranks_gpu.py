"""GPU: sharded propagation with libqp's own partition and import, several
shards held by one process on one GPU (the exchange done by copies between
the shards' buffers; no collective, no kernel that waits on another).

Each shard is a context on the merge-table engine holding the paths whose
next pre-merge group its rank owns; rho(t) summed over the shards must equal
the single-context result and the oracle within the FP64 parity bar, and the
stored paths summed over shards must equal the single context's.  The
partition must place every path with the owner the header's formula gives.
"""
import numpy as np
import pytest

import workloads as W
from oracle import iquapi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2506_03127_gb300 import Propagator, build  # noqa: E402

build.build()
from paper_2506_03127_gb300.ranks import ContextShard, step_in_process  # noqa: E402

TOL = 1e-10


def _ctx(case, mask, theta, precision="fp64"):
    p = Propagator(case["M"], case["dkmax"], case["dt"], case["q"], case["hs"], theta, precision, "hash",
                   max_paths=1 << 20)
    p.set_eta(case["eta"])
    p.set_mask(mask)
    p.set_rho0(case["rho0"])
    return p


@pytest.mark.parametrize("n_ranks", [2, 3])
@pytest.mark.parametrize("M,dkmax,mask,theta,steps,seed", [(2, 6, (0, 1, 2, 4), 1e-6, 14, 71),
                                                            (3, 4, None, 1e-6, 8, 72), (2, 9, None, 0.0, 12, 73)])
def test_shards_on_one_gpu_equal_one_context(n_ranks, M, dkmax, mask, theta, steps, seed):
    case = W.random_case(seed, M, dkmax)
    shards = [ContextShard(_ctx(case, mask, theta), n_ranks, r) for r in range(n_ranks)]
    rho, kept = step_in_process(shards, case["rho0"], steps)
    one = _ctx(case, mask, theta)
    one.step(steps)
    one.sync()
    rho1 = one.rho(0, steps + 1)
    kept1 = [s[3] for s in one.stats(1, steps)]
    assert np.abs(rho - rho1).max() <= TOL
    assert [sum(k) for k in kept] == kept1
    o = iquapi.propagate(M, case["q"], case["hs"], case["dt"], case["eta"], dkmax, mask, theta, case["rho0"], steps)
    assert np.abs(rho - o.rho).max() <= TOL
    if steps > dkmax:
        assert min(min(k) for k in kept[dkmax:]) > 0   # every rank holds paths
    # the partition places every path with the owner of the stated formula
    Pp = iquapi.premerge_positions(iquapi.check_mask(range(dkmax) if mask is None else mask, dkmax), dkmax)
    bs, b = iquapi.state_bits(M)
    pmask = np.uint64(sum(((1 << b) - 1) << (b * p) for p in Pp))
    keys, amps, counts = shards[0].partition()
    k = keys.cpu().numpy().view(np.uint64)
    with np.errstate(over="ignore"):
        own = (((k & pmask) * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(32)) % np.uint64(n_ranks)
    np.testing.assert_array_equal(own, np.repeat(np.arange(n_ranks), counts))
    for s in shards:
        s.p.close()
    one.close()
