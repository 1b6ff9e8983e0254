"""GPU: the batched form on the stream engine.

A batch keeps its stored set in n_inst * M^2 regions (instance, newest
point); one ticket order runs over the tiles of all regions, so an
instance's tiles are consecutive and each tile's look-back stops at its
instance's first tile; every tile reads its own instance's history tables
and propagator table and adds its children to its instance's rho.  Each
instance must reproduce, within the FP64 parity bar, the oracle run of that
instance alone (rho, per-instance path counts), in graph launches and in one
persistent launch for all steps, and store the same key set as the
merge-table engine's batch.
"""
import numpy as np
import pytest

import workloads as W
from oracle import bath as B
from oracle import iquapi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2506_03127_gb300 import Propagator, abi, batch_from_workloads, build  # noqa: E402

build.build()

TOL = 1e-10


def _batch(case, etas, mask, theta, precision="fp64", engine="auto", tuning=None, max_paths=1 << 20):
    M, dk = case["M"], case["dkmax"]
    p = Propagator(M, dk, case["dt"], case["q"], case["hs"], theta, precision, engine=engine, max_paths=max_paths,
                   n_inst=len(etas))
    p.set_eta(etas[0])
    for i, e in enumerate(etas):
        p.set_eta_instance(i, e)
    p.set_mask(mask)
    p.set_rho0(case["rho0"])
    if tuning:
        p.set_tuning(**tuning)
    return p


def _oracle(case, eta, mask, theta, steps):
    return iquapi.propagate(case["M"], case["q"], case["hs"], case["dt"], eta, case["dkmax"], mask, theta,
                            case["rho0"], steps)


CASES = [(2, 6, None, 1e-5, 14, 5), (2, 7, (0, 1, 2, 3), 1e-6, 12, 3), (3, 4, None, 1e-6, 8, 3),
         (4, 3, None, 1e-6, 6, 2), (2, 8, None, 0.0, 11, 4)]
LAUNCHES = {
    "graph512": dict(stream_tile=512),
    "graph1024": dict(stream_tile=1024, expand_blocks_per_sm=1),
    "persistent": dict(mode=abi.QP_LAUNCH_PERSISTENT, persistent_blocks=152, stream_tile=1024),
    "persistent3": dict(mode=abi.QP_LAUNCH_PERSISTENT, persistent_blocks=3, stream_tile=512),
}


@pytest.mark.parametrize("M,dkmax,mask,theta,steps,ninst", CASES)
@pytest.mark.parametrize("launch", list(LAUNCHES), ids=list(LAUNCHES))
def test_batch_stream_matches_oracle(M, dkmax, mask, theta, steps, ninst, launch):
    case = W.random_case(200 + 10 * M + dkmax, M, dkmax)
    rng = np.random.default_rng(11)
    etas = [W.random_eta(rng, dkmax, 0.03 + 0.04 * i) for i in range(ninst)]
    p = _batch(case, etas, mask, theta, tuning=LAUNCHES[launch])
    assert p.tuning().engine == abi.QP_ENGINE_STREAM
    # two calls (the persistent kernel runs each call's steps in one launch)
    p.step(steps // 2)
    p.step(steps - steps // 2)
    p.sync()
    rho = p.rho(0, steps + 1)
    counts = np.array([p.instance_counts(t) for t in range(steps + 1)])
    stats = p.stats(1, steps)
    p.close()
    total = np.zeros(steps + 1, dtype=np.int64)
    for i, e in enumerate(etas):
        o = _oracle(case, e, mask, theta, steps)
        err = np.abs(rho[:, i] - o.rho).max()
        assert err <= TOL, (i, err)
        kept_o = [int(np.count_nonzero(case["rho0"]))] + [s.kept for s in o.stats]
        np.testing.assert_array_equal(counts[:, i], kept_o)
        total += np.array(kept_o)
    assert [s[3] for s in stats] == list(total[1:])


@pytest.mark.parametrize("M,dkmax,theta,steps", [(2, 6, 1e-5, 12), (3, 4, 1e-6, 7)])
def test_batch_stream_key_sets_match_merge_table_batch(M, dkmax, theta, steps):
    """Same instances on both engines: per instance the same stored keys
    (with the instance index above the path bits) and amplitudes."""
    case = W.random_case(300 + M, M, dkmax)
    rng = np.random.default_rng(5)
    etas = [W.random_eta(rng, dkmax, 0.05 + 0.03 * i) for i in range(4)]
    out = {}
    for engine in ("stream", "hash"):
        p = _batch(case, etas, None, theta, engine=engine)
        p.step(steps)
        keys, amps = p.export_paths()
        out[engine] = dict(zip(keys.tolist(), amps.tolist()))
        p.close()
    assert set(out["stream"]) == set(out["hash"])
    d = max(abs(out["stream"][k] - out["hash"][k]) for k in out["hash"])
    assert d <= 1e-12


def test_batch_stream_empty_instances():
    """A filter that removes every child: all instances empty from the first
    step on, later steps run on the empty set, rho is zero."""
    case = W.random_case(401, 2, 5)
    rng = np.random.default_rng(3)
    etas = [W.random_eta(rng, 5, 0.05) for _ in range(3)]
    p = _batch(case, etas, None, 10.0)
    p.step(4)
    p.sync()
    assert p.current() == (4, 0)
    assert all((p.instance_counts(t) == 0).all() for t in range(1, 5))
    rho = p.rho(1, 4)
    assert np.abs(rho).max() == 0.0
    p.close()


def test_coupling_sweep_c64_against_oracle():
    """Three instances of the 64-instance coupling sweep (path counts
    differ by more than 2x) in complex64 on the stream engine, 100 steps,
    against the FP64 oracle of each instance: within the complex64 bound of
    the single-problem engine on the same model (2e-6)."""
    ws = W.coupling_sweep(64)
    p = batch_from_workloads(ws, precision="c64", max_paths=1 << 23)
    assert p.tuning().engine == abi.QP_ENGINE_STREAM
    p.set_tuning(mode=abi.QP_LAUNCH_PERSISTENT, persistent_blocks=304, stream_tile=1024)
    p.step(100)
    rb = p.rho(0, 101)
    counts = p.instance_counts(100)
    p.close()
    assert counts.max() >= 2 * counts.min()
    for i in (0, 2, 3):
        w = ws[i]
        o = iquapi.propagate_workload(w, eta=B.eta_coefficients(w.bath, w.dt, w.dkmax), steps=100)
        err = np.abs(rb[:, i] - o.rho).max()
        assert err <= 2e-6, (i, err)
        assert abs(int(counts[i]) - o.stats[-1].kept) <= max(2, o.stats[-1].kept // 200)


def test_coupling_sweep_fp64_instances_against_oracle():
    ws = W.coupling_sweep(64)
    p = batch_from_workloads(ws, precision="fp64", max_paths=1 << 23)
    p.step(40)
    rb = p.rho(0, 41)
    counts = p.instance_counts(40)
    p.close()
    for i in (0, 1, 2, 63):
        w = ws[i]
        o = iquapi.propagate_workload(w, eta=B.eta_coefficients(w.bath, w.dt, w.dkmax), steps=40)
        assert np.abs(rb[:, i] - o.rho).max() <= TOL
        assert counts[i] == o.stats[-1].kept


def test_batch_stream_autotune_keeps_parity():
    case = W.random_case(501, 2, 6)
    rng = np.random.default_rng(8)
    etas = [W.random_eta(rng, 6, 0.04 + 0.02 * i) for i in range(6)]
    p = _batch(case, etas, None, 1e-6)
    p.step(6)
    best, ms = p.autotune(trial_steps=3, use_cache=False)
    assert best.mode in (abi.QP_LAUNCH_GRAPH, abi.QP_LAUNCH_PERSISTENT) and best.stream_tile in (512, 1024)
    assert ms > 0
    t, _ = p.current()
    p.step(4)
    rho = p.rho(0, t + 5)
    p.close()
    for i, e in enumerate(etas):
        o = _oracle(case, e, None, 1e-6, t + 4)
        assert np.abs(rho[:, i] - o.rho).max() <= TOL


def test_batch_stream_persistent_barrier_wait_is_bounded():
    """The persistent batch kernel's grid barrier cannot complete: every
    block gives up after its bound, QP_ERR_TIMEOUT, usable after
    qp_set_rho0."""
    case = W.random_case(601, 2, 5)
    rng = np.random.default_rng(2)
    etas = [W.random_eta(rng, 5, 0.05) for _ in range(2)]
    p = _batch(case, etas, None, 0.0, tuning=dict(mode=abi.QP_LAUNCH_PERSISTENT, persistent_blocks=152))
    p.step(2)
    p.sync()
    abi.qp_test_stall_barrier(p.ctx)
    p.step(3)
    with pytest.raises(abi.QPError) as e:
        p.sync()
    assert e.value.status == abi.QP_ERR_TIMEOUT
    p.set_rho0(case["rho0"])
    p.step(4)
    p.sync()
    assert p.current()[0] == 4
    rho = p.rho(0, 5)
    p.close()
    for i, eta in enumerate(etas):
        o = _oracle(case, eta, None, 0.0, 4)
        assert np.abs(rho[:, i] - o.rho).max() <= TOL


def test_batch_stream_lookback_wait_is_bounded():
    """The first tile of a step publishes nothing: the other tiles of its
    instance give up after their bound, the step is not published,
    QP_ERR_TIMEOUT, usable after qp_set_rho0."""
    case = W.random_case(701, 2, 6)
    rng = np.random.default_rng(4)
    etas = [W.random_eta(rng, 6, 0.05) for _ in range(3)]
    p = _batch(case, etas, None, 0.0)
    p.step(5)
    p.sync()
    abi.qp_test_stall_lookback(p.ctx)
    p.step(1)
    with pytest.raises(abi.QPError) as e:
        p.sync()
    assert e.value.status == abi.QP_ERR_TIMEOUT
    p.set_rho0(case["rho0"])
    p.step(3)
    p.sync()
    rho = p.rho(0, 4)
    p.close()
    for i, eta in enumerate(etas):
        assert np.abs(rho[:, i] - _oracle(case, eta, None, 0.0, 3).rho).max() <= TOL
