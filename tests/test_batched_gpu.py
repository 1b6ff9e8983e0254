"""GPU: the batched form (several independent instances in one context),
the launch-shape autotuner and the bounded waits of the persistent kernel.
"auto" runs batches whose P' is a prefix of the window on the stream
engine (tests/test_batched_stream_gpu.py covers it in depth), the others on
the merge-table engine; "hash" forces the merge-table engine.

Each instance of a batch must reproduce, within the FP64 parity bar, the
oracle run of that instance alone, with the same per-instance path counts;
a batch must also agree with separate single-instance contexts.
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

from paper_2506_03127_gb300 import Propagator, abi, batch_from_workloads, build, eta_from_bath  # noqa: E402

build.build()

TOL = 1e-10


def _batch(case, etas, mask, theta, steps, precision="fp64", launch=None, engine="auto"):
    M, dk = case["M"], case["dkmax"]
    p = Propagator(M, dk, case["dt"], case["q"], case["hs"], theta, precision, engine=engine, max_paths=1 << 20,
                   n_inst=len(etas))
    p.set_eta(etas[0])
    for i, e in enumerate(etas):
        p.set_eta_instance(i, e)
    p.set_mask(mask)
    if launch:
        p.set_tuning(**launch)
    p.set_rho0(case["rho0"])
    p.step(steps)
    p.sync()
    rho = p.rho(0, steps + 1)
    counts = np.array([p.instance_counts(t) for t in range(steps + 1)])
    stats = p.stats(1, steps)
    p.close()
    return rho, counts, stats


@pytest.mark.parametrize("M,dkmax,mask,theta,steps,ninst", [(2, 6, (0, 1, 2, 4), 1e-5, 12, 5),
                                                            (3, 4, None, 1e-6, 8, 3), (2, 8, None, 0.0, 11, 4)])
@pytest.mark.parametrize("launch", [None, dict(mode=abi.QP_LAUNCH_PERSISTENT)], ids=["graph", "persistent"])
@pytest.mark.parametrize("engine", ["hash", "auto"])
def test_batch_instances_match_oracle(M, dkmax, mask, theta, steps, ninst, launch, engine):
    case = W.random_case(100 + M + dkmax, M, dkmax)
    rng = np.random.default_rng(7)
    etas = [W.random_eta(rng, dkmax, 0.05 + 0.02 * i) for i in range(ninst)]
    if launch:
        launch = dict(launch, persistent_blocks=152)
    rho, counts, stats = _batch(case, etas, mask, theta, steps, launch=launch, engine=engine)
    total_kept = np.zeros(steps + 1, dtype=np.int64)
    for i, e in enumerate(etas):
        o = iquapi.propagate(M, case["q"], case["hs"], case["dt"], e, dkmax, mask, theta, case["rho0"], steps)
        assert np.abs(rho[:, i] - o.rho).max() <= TOL, (i, np.abs(rho[:, i] - o.rho).max())
        kept_o = [int(np.count_nonzero(case["rho0"]))] + [s.kept for s in o.stats]
        np.testing.assert_array_equal(counts[:, i], kept_o)
        total_kept += np.array(kept_o)
    assert [s[3] for s in stats] == list(total_kept[1:])


def test_batch_agrees_with_single_contexts_c64():
    ws = W.resonance_sweep(6)
    p = batch_from_workloads(ws, precision="c64", max_paths=1 << 20)
    p.step(30)
    rb = p.rho(0, 31)
    cb = p.instance_counts(30)
    p.close()
    for i, w in enumerate(ws):
        q = Propagator.from_workload(w, precision="c64", max_paths=1 << 18)
        q.step(30)
        r1 = q.rho(0, 31)
        assert np.abs(rb[:, i] - r1).max() < 1e-6
        assert abs(int(cb[i]) - q.current()[1]) <= max(2, q.current()[1] // 1000)
        q.close()


def test_resonance_sweep_instances_against_oracle():
    """Three instances of the 64-instance sweep, FP64, 40 steps, against the
    oracle run of each instance (its own eta by quadrature)."""
    ws = W.resonance_sweep(64)
    p = batch_from_workloads(ws, precision="fp64", max_paths=1 << 22)
    p.step(40)
    rb = p.rho(0, 41)
    counts = p.instance_counts(40)
    assert len(set(counts.tolist())) > 32          # path counts differ across the sweep
    p.close()
    for i in (0, 21, 63):
        w = ws[i]
        o = iquapi.propagate_workload(w, eta=B.eta_coefficients(w.bath, w.dt, w.dkmax), steps=40)
        assert np.abs(rb[:, i] - o.rho).max() <= TOL
        assert counts[i] == o.stats[-1].kept


def test_autotune_picks_a_valid_shape_and_keeps_parity():
    case = W.random_case(5, 2, 8)
    mask, theta = (0, 1, 2, 5), 1e-6
    p = Propagator(2, 8, case["dt"], case["q"], case["hs"], theta, engine="hash", max_paths=1 << 18)
    p.set_eta(case["eta"])
    p.set_mask(mask)
    p.set_rho0(case["rho0"])
    p.step(10)
    best, ms = p.autotune(trial_steps=3, use_cache=False)
    assert best.mode in (abi.QP_LAUNCH_GRAPH, abi.QP_LAUNCH_PERSISTENT) and ms > 0
    t, _ = p.current()
    p.step(5)
    rho = p.rho(0, t + 6)
    p.close()
    o = iquapi.propagate(2, case["q"], case["hs"], case["dt"], case["eta"], 8, mask, theta, case["rho0"], t + 5)
    assert np.abs(rho - o.rho).max() <= TOL
    # cached choice is applied without trials
    p2 = Propagator(2, 8, case["dt"], case["q"], case["hs"], theta, engine="hash", max_paths=1 << 18)
    p2.set_eta(case["eta"])
    p2.set_mask(mask)
    p2.set_rho0(case["rho0"])
    p2.step(10)
    best2, ms2 = p2.autotune(trial_steps=3, use_cache=True)
    assert ms2 == -1.0 and best2.as_dict() == best.as_dict()
    p2.close()


def test_tuning_is_validated():
    case = W.random_case(6, 2, 6)
    p = Propagator(2, 6, case["dt"], case["q"], case["hs"], 0.0, max_paths=1 << 14)
    for bad in [dict(mode=7), dict(insert_blocks_per_sm=0), dict(graph_steps=0), dict(table_log2=63),
                dict(mode=abi.QP_LAUNCH_PERSISTENT, persistent_blocks=1 << 20)]:
        with pytest.raises(abi.QPError) as e:
            p.set_tuning(**bad)
        assert e.value.status == abi.QP_ERR_ARG
    p.close()


def test_persistent_barrier_wait_is_bounded():
    """A grid barrier that cannot complete: every block stops waiting after
    its bound, the step is not applied, the context reports QP_ERR_TIMEOUT and
    is usable again after qp_set_rho0."""
    case = W.random_case(8, 2, 5)
    p = Propagator(2, 5, case["dt"], case["q"], case["hs"], 0.0, engine="hash", max_paths=1 << 14)
    p.set_eta(case["eta"])
    p.set_mask(None)
    p.set_rho0(case["rho0"])
    p.set_tuning(mode=abi.QP_LAUNCH_PERSISTENT, persistent_blocks=152)
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
    o = iquapi.propagate(2, case["q"], case["hs"], case["dt"], case["eta"], 5, None, 0.0, case["rho0"], 4)
    assert np.abs(p.rho(0, 5) - o.rho).max() <= TOL
    p.close()
