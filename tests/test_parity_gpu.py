"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar (FP64 path): every rho(t) within 1e-10 max-abs of the oracle's, per-step
group and survivor counts equal, and the surviving key set bit-exact with
amplitudes within 1e-10 -- the key comparison is made only where the
oracle reports no decision within rounding distance of the tie window or of
the filter threshold (reported as near_tie / near_theta).
"""
import numpy as np
import pytest

import workloads as W
from oracle import iquapi
from tests.golden.make_golden import load as load_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2506_03127_gb300 import Propagator, abi, build, eta_from_bath  # noqa: E402

build.build()

RHO_TOL = 1e-10


def gpu_run(M, q, hs, dt, eta, dkmax, mask, theta, rho0, steps, precision="fp64", max_paths=1 << 20,
            max_groups=0, engine="auto"):
    p = Propagator(M, dkmax, dt, q, hs, theta, precision, engine, max_paths, max_groups)
    p.set_eta(eta)
    p.set_mask(mask)
    p.set_rho0(rho0)
    p.step(steps)
    p.sync()
    rho = p.rho(0, steps + 1)
    stats = p.stats(1, steps) if steps else []
    keys, amps = p.export_paths()
    p.close()
    return rho, stats, keys, amps


def compare(res_gpu, res_or, M, check_keys=True, tol=RHO_TOL):
    rho, stats, keys, amps = res_gpu
    assert np.abs(rho - res_or.rho).max() <= tol, np.abs(rho - res_or.rho).max()
    for s_g, s_o in zip(stats, res_or.stats):
        assert s_g[0] == s_o.t
        assert (s_g[1], s_g[3]) == (s_o.groups, s_o.kept), (s_g, s_o)
    ambiguous = any(s.near_tie or s.near_theta for s in res_or.stats)
    if check_keys and not ambiguous:
        ko = iquapi.packed_keys(res_or.paths.sp, res_or.paths.sm, M)
        assert keys.size == ko.size
        # with dkmax = 1 children of different groups share a key until the
        # next pre-merge, so compare the amplitude summed per distinct key
        ug, ig = np.unique(keys, return_inverse=True)
        uo, io = np.unique(ko, return_inverse=True)
        np.testing.assert_array_equal(ug, uo)
        sg = np.zeros(ug.size, dtype=complex)
        so = np.zeros(uo.size, dtype=complex)
        np.add.at(sg, ig, amps)
        np.add.at(so, io, res_or.paths.amp)
        assert np.abs(sg - so).max() <= tol
    return ambiguous


def run_both(case, mask, theta, steps, **kw):
    M, dk = case["M"], case["dkmax"]
    g = gpu_run(M, case["q"], case["hs"], case["dt"], case["eta"], dk, mask, theta, case["rho0"], steps, **kw)
    o = iquapi.propagate(M, case["q"], case["hs"], case["dt"], case["eta"], dk, mask, theta, case["rho0"], steps)
    return g, o


ENGINES = ["stream", "hash"]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("M,dkmax,steps,seed", [(2, 1, 10, 1), (2, 2, 12, 2), (2, 5, 14, 3), (2, 8, 12, 4),
                                                (3, 1, 8, 5), (3, 3, 8, 6), (3, 4, 7, 7), (4, 2, 6, 8), (4, 3, 5, 9)])
def test_unmasked_unfiltered_matches_oracle(M, dkmax, steps, seed, engine):
    case = W.random_case(seed, M, dkmax)
    g, o = run_both(case, None, 0.0, steps, engine=engine)
    compare(g, o, M)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("precision", ["fp64", "c64"])
@pytest.mark.parametrize("M,dkmax,mask,theta,steps,seed", [(3, 4, (0, 1, 2), 1e-6, 9, 51), (4, 3, None, 1e-5, 6, 52),
                                                            (2, 6, (0, 1, 2, 4), 1e-6, 14, 53)])
def test_equally_spaced_couplings_match_oracle(M, dkmax, mask, theta, steps, seed, precision, engine):
    """Coupling eigenvalues q_a = q_0 + a s: the kernels form the children's
    influence factors as powers of exp(-s H) instead of one exponential per
    distinct difference.  FP64 at the parity bar; complex64 within 1e-6."""
    case = W.random_case(seed, M, dkmax)
    case["q"] = np.array([-0.7 + 0.45 * a for a in range(M)])
    g, o = run_both(case, mask, theta, steps, engine=engine, precision=precision)
    if precision == "fp64":
        compare(g, o, M)
    else:
        assert np.abs(g[0] - o.rho).max() <= 1e-6


@pytest.mark.parametrize("M,dkmax,mask,theta,steps,seed", [
    (2, 8, (0, 1, 2, 5), 1e-4, 20, 11),
    (2, 10, (0, 1, 2, 3, 4, 5, 6, 8), 1e-6, 24, 12),
    (2, 9, (0, 1, 2, 3, 5, 8), 0.0, 14, 13),
    (2, 12, (0, 1, 2, 3, 4, 6, 9), 1e-5, 30, 14),
    (3, 5, (0, 1, 3), 1e-5, 12, 15),
    (3, 6, (0, 1, 2, 3), 0.0, 9, 16),
    (4, 4, (0, 1, 3), 1e-4, 8, 17),
])
@pytest.mark.parametrize("engine", ["auto", "hash"])
def test_masked_filtered_matches_oracle(M, dkmax, mask, theta, steps, seed, engine):
    """auto: the stream engine wherever P' is a prefix plus at most one extra
    position (M = 2), the merge table otherwise."""
    case = W.random_case(seed, M, dkmax)
    g, o = run_both(case, mask, theta, steps, engine=engine)
    compare(g, o, M)


def test_hashed_table_index_matches_oracle():
    """dkmax 11 without mask: 20 masked-key bits exceed a 2^17-slot table, so
    the merge table hashes (linear probing) instead of indexing directly."""
    case = W.random_case(21, 2, 11)
    g, o = run_both(case, None, 1e-7, 18, max_groups=1 << 16)
    compare(g, o, 2)


@pytest.mark.parametrize("engine", ENGINES)
def test_spin_boson_ohmic_dk8_trajectory_against_stored_oracle(engine):
    w = W.SPIN_BOSON_OHMIC_DK8
    eta = eta_from_bath(w.bath, w.dt, w.dkmax)
    rho, stats, keys, amps = gpu_run(w.M, w.q, w.hs_array(), w.dt, eta, w.dkmax, w.mask, w.theta,
                                     w.rho0_array(), w.steps, engine=engine)
    t, n, rho_o = load_golden("spin_boson_ohmic_dk8_rho.txt")
    assert np.abs(rho - rho_o).max() <= RHO_TOL
    assert [s[3] for s in stats] == list(n[1:])
    assert keys.size == 65536


def test_spin_boson_structured_dk16_first_40_steps_against_stored_oracle():
    w = W.SPIN_BOSON_STRUCTURED_DK16
    eta = eta_from_bath(w.bath, w.dt, w.dkmax)
    for engine in ("stream", "hash"):
        rho, stats, keys, amps = gpu_run(w.M, w.q, w.hs_array(), w.dt, eta, w.dkmax, w.mask, w.theta,
                                         w.rho0_array(), 40, max_paths=1 << 21, engine=engine)
        t, n, rho_o = load_golden("spin_boson_structured_dk16_rho40.txt")
        assert np.abs(rho - rho_o).max() <= RHO_TOL, engine
        assert [s[3] for s in stats] == list(n[1:]), engine
    rho, stats, keys, amps = gpu_run(w.M, w.q, w.hs_array(), w.dt, eta, w.dkmax, w.mask, w.theta,
                                     w.rho0_array(), 40, max_paths=1 << 21)
    t, n, rho_o = load_golden("spin_boson_structured_dk16_rho40.txt")
    assert np.abs(rho - rho_o).max() <= RHO_TOL
    assert [s[3] for s in stats] == list(n[1:])


@pytest.mark.parametrize("precision", ["fp64", "c64"])
def test_stream_engine_rerun_and_launch_shapes_agree(precision):
    """Look-back words carry the step number, which restarts with every
    qp_set_rho0: a second propagation on the same context, and the same
    propagation with every tile size and grid, give the same survivor counts
    and rho (up to rounding: the groups of runs longer than 32 paths, while the
    window fills, are summed with FP64 atomics in no fixed order)."""
    w = W.SPIN_BOSON_STRUCTURED_DK16
    p = Propagator.from_workload(w, precision=precision, engine="stream", max_paths=1 << 21)
    runs = []
    for tile, bps in [(512, 4), (512, 4), (256, 2), (1024, 1), (512, 8)]:
        p.set_rho0(w.rho0_array())
        p.set_tuning(stream_tile=tile, expand_blocks_per_sm=bps)
        p.step(60)
        p.sync()
        runs.append((p.rho(0, 61), [s[3] for s in p.stats(1, 60)]))
    tol = 1e-12 if precision == "fp64" else 1e-6
    for rho, kept in runs[1:]:
        assert kept == runs[0][1]
        assert np.abs(rho - runs[0][0]).max() <= tol
    if precision == "fp64":
        t, n, rho_o = load_golden("spin_boson_structured_dk16_rho40.txt")
        assert np.abs(runs[-1][0][:41] - rho_o).max() <= RHO_TOL
    p.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("c64", 1e-6)])
def test_stream_rho_read_every_step_equals_history_read_at_the_end(precision, tol):
    """A stream-engine step publishes its counters; its rho is summed from the
    blocks' partials when the next step starts or when it is read.  Reading
    rho after every step and reading the whole history once at the end give
    the same values (up to the order of the FP64 atomic sums of long runs)."""
    w = W.SPIN_BOSON_STRUCTURED_DK16
    p1 = Propagator.from_workload(w, precision=precision, engine="stream", max_paths=1 << 21)
    per_step = []
    for t in range(1, 41):
        p1.step(1)
        per_step.append(p1.rho(t, 1)[0])
    p1.close()
    p2 = Propagator.from_workload(w, precision=precision, engine="stream", max_paths=1 << 21)
    p2.step(40)
    at_end = p2.rho(1, 40)
    p2.close()
    assert np.abs(np.array(per_step) - at_end).max() <= tol
    if precision == "fp64":
        t, n, rho_o = load_golden("spin_boson_structured_dk16_rho40.txt")
        assert np.abs(at_end - rho_o[1:]).max() <= RHO_TOL


@pytest.mark.parametrize("engine,precision,pinned", [("stream", "c64", True), ("stream", "fp64", True),
                                                     ("hash", "fp64", True), ("stream", "c64", False)])
def test_async_rho_reads_equal_the_history(engine, precision, pinned):
    """qp_read_rho_async after every step (stream-ordered; page-locked memory
    is written by the finalising kernel itself, other memory is copied), one
    synchronisation at the end, gives the rows a synchronous read of the
    history gives; a step not yet taken, or one older than the history ring,
    is rejected without a copy."""
    w = W.SPIN_BOSON_STRUCTURED_DK16
    p = Propagator.from_workload(w, precision=precision, engine=engine, max_paths=1 << 21, rho_history=64)
    buf = torch.empty((100, 2, 2), dtype=torch.complex128, pin_memory=pinned)
    for t in range(1, 101):
        p.step(1)
        p.rho_async(t, buf[t - 1])
    p.sync()
    assert np.array_equal(buf.numpy()[40:], p.rho(41, 60))
    if precision == "fp64":
        t, n, rho_o = load_golden("spin_boson_structured_dk16_rho40.txt")
        assert np.abs(buf.numpy()[:40] - rho_o[1:]).max() <= RHO_TOL
    for bad in (101, 36):   # not taken yet / no longer in the ring of 64
        with pytest.raises(abi.QPError):
            p.rho_async(bad, buf[0])
    p.close()


def test_c64_group_sums_agree_with_fp64_sums_rounded():
    """Reading of the complex64 group sum: the stream engine forms it as an
    error-free FP32 pair rounded once, the merge-table engine adds the members
    in FP64 and rounds.  Both expand with the same arithmetic, so the stored
    sets agree bit for bit before the first merge; after the first merging
    step the survivors are the same and the amplitudes agree bit for bit
    except where an exact sum lies next to an FP32 rounding midpoint (then
    within a few units in the last place)."""
    w = W.SPIN_BOSON_STRUCTURED_DK16
    for steps in (w.dkmax - 1, w.dkmax):
        got = []
        for engine in ("stream", "hash"):
            p = Propagator.from_workload(w, precision="c64", engine=engine, max_paths=1 << 21)
            p.step(steps)
            p.sync()
            k, a = p.export_paths()
            p.close()
            o = np.argsort(k)
            got.append((k[o], a[o]))
        (ks, a_s), (kh, a_h) = got
        np.testing.assert_array_equal(ks, kh)
        if steps < w.dkmax:
            assert np.array_equal(a_s, a_h)
        else:
            diff = a_s != a_h
            assert diff.mean() <= 1e-3, diff.mean()
            assert np.all(np.abs(a_s - a_h)[diff] <= 2.0 ** -21 * np.abs(a_h)[diff])


def test_spin_boson_structured_dk16_full_length_properties():
    """All 2000 steps at full size: properties that hold at any size.  The
    trace is conserved by merging and propagation, so it changes only through
    the filter: its real part stays at or below 1 and its loss, like its
    imaginary part (the filtered paths carry complex weight), stays small.
    Counts stay below M^(2 dk_eff).  With a mask rho need not be Hermitian."""
    w = W.SPIN_BOSON_STRUCTURED_DK16
    p = Propagator.from_workload(w, max_paths=1 << 21)
    p.step(w.steps)
    p.sync()
    t, n = p.current()
    assert t == w.steps and 0 < n <= 4 ** 10
    rho = p.rho(w.steps - 999, 1000)
    tr = np.trace(rho, axis1=1, axis2=2)
    assert np.all(tr.real <= 1 + 1e-12) and np.all(tr.real > 0.95)
    assert np.abs(tr.imag).max() < 1e-3 and (1 - tr.real).max() < 1e-2
    d = np.diagonal(rho, axis1=1, axis2=2)
    assert d.real.min() > -1e-6
    p.close()


def test_all_paths_filtered_leaves_empty_set():
    case = W.random_case(31, 2, 4)
    g, o = run_both(case, None, 10.0, 6)
    rho, stats, keys, amps = g
    assert keys.size == 0 and np.abs(rho[1:]).max() == 0.0
    assert all(s[3] == 0 for s in stats)


def test_capacity_overflow_is_reported_and_recoverable():
    case = W.random_case(41, 2, 6)
    p = Propagator(2, 6, case["dt"], case["q"], case["hs"], 0.0, max_paths=300)
    p.set_eta(case["eta"])
    p.set_mask(None)
    p.set_rho0(case["rho0"])
    p.step(8)
    with pytest.raises(abi.QPError) as e:
        p.sync()
    assert e.value.status == abi.QP_ERR_CAPACITY
    with pytest.raises(abi.QPError) as e2:
        p.step(1)
    assert e2.value.status == abi.QP_ERR_STATE
    p.set_rho0(case["rho0"])       # restart clears the error
    p.step(3)
    p.sync()
    assert p.current()[0] == 3
    p.close()


def test_invalid_mask_rejected():
    case = W.random_case(42, 2, 6)
    p = Propagator(2, 6, case["dt"], case["q"], case["hs"], 0.0, max_paths=1 << 12)
    for bad in [(0, 2), (1, 2), (0, 1, 6), (-1, 0, 1)]:
        with pytest.raises(abi.QPError) as e:
            p.set_mask(bad)
        assert e.value.status == abi.QP_ERR_ARG
    with pytest.raises(abi.QPError) as e:
        p.step(1)                  # no rho0 yet
    assert e.value.status == abi.QP_ERR_STATE
    p.close()


def test_device_widening_is_exact_for_every_float_class():
    """The FP32 -> FP64 widening the step kernels apply (integer field
    arithmetic) equals IEEE conversion bit for bit: signed zeros, every
    subnormal leading-one position, normals over the whole exponent range,
    the largest float, infinities; NaNs stay NaNs."""
    rng = np.random.default_rng(7)
    bits = [0, 0x80000000, 1, 0x80000001, 0x007FFFFF, 0x807FFFFF, 0x00400000, 0x00000100, 0x00800000,
            0x7F7FFFFF, 0xFF7FFFFF, 0x7F800000, 0xFF800000, 0x7FC00000, 0x7F800001, 0x3F800000, 0xBF800000]
    bits += [1 << k for k in range(23)] + [(1 << k) | 0x80000000 for k in range(23)]
    x = np.concatenate([np.array(bits, dtype=np.uint32),
                        rng.integers(0, 2 ** 32, size=200000, dtype=np.uint64).astype(np.uint32)]).view(np.float32)
    xin = torch.from_numpy(x.copy()).cuda()
    out = torch.empty(x.size, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    abi.qp_test_widen(xin.data_ptr(), out.data_ptr(), x.size, 0)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    with np.errstate(invalid="ignore"):   # signalling NaNs among the random patterns
        ref = x.astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint64), ref[~nan].view(np.uint64))



def test_stream_lookback_wait_is_bounded():
    """A tile that never publishes its survivor counts: the step's other
    tiles give up waiting after their bound and write nothing, the step is
    not applied, the context reports QP_ERR_TIMEOUT, refuses to step
    (QP_ERR_STATE) and propagates correctly again after qp_set_rho0."""
    case = W.random_case(43, 2, 8)
    mask, theta = None, 1e-7            # about 26 000 stored paths from t = 10
    p = Propagator(2, 8, case["dt"], case["q"], case["hs"], theta, engine="stream", max_paths=1 << 18)
    p.set_eta(case["eta"])
    p.set_mask(mask)
    p.set_rho0(case["rho0"])
    p.set_tuning(stream_tile=256, expand_blocks_per_sm=1)
    p.step(10)
    p.sync()
    t_before, n_before = p.current()
    assert n_before > 8 * 256          # several tiles in the next step
    abi.qp_test_stall_lookback(p.ctx)
    p.step(2)
    with pytest.raises(abi.QPError) as e:
        p.sync()
    assert e.value.status == abi.QP_ERR_TIMEOUT
    with pytest.raises(abi.QPError) as e2:
        p.step(1)
    assert e2.value.status == abi.QP_ERR_STATE
    p.set_rho0(case["rho0"])
    p.step(12)
    p.sync()
    o = iquapi.propagate(2, case["q"], case["hs"], case["dt"], case["eta"], 8, mask, theta, case["rho0"], 12)
    assert np.abs(p.rho(0, 13) - o.rho).max() <= RHO_TOL
    p.close()
