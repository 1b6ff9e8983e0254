"""GPU: the complex64 precision form against the FP64 oracle.

The complex64 form (complex64 amplitudes, the influence exponent summed in
FP32 with compensated additions, group sums of FP32 members rounded once
from an error-free pair, FP64 eta and rho) is compared with trajectories the
oracle wrote (tests/golden/, make_golden.py calls only oracle/), on every
stream kernel and on the merge-table engine:

  * spin_boson_ohmic_dk8, full length, and the full-memory TLS model at
    memory 8 and 10 (no mask, no filter): the regular stream kernel;
  * spin_boson_structured_dk16, 200 steps (mask with one extra pre-merge
    position, filter): the tile kernel with sub-groups;
  * the three-level chain with memory 7 (merging steps) and memory 12 (the
    window filling, up to 1.6e7 stored paths): the M = 3 tile kernel.

Each case asserts its own bound on max_t max_ab |rho_c64(t) - rho_oracle(t)|,
the bound the design document states for that configuration, and that the
survivor counts stay within a small fraction of the oracle's (filter
decisions on sums of nearly cancelling members may differ).  The same trajectories
also bound the FP64 path at the parity tolerance of the other GPU tests.
"""
import numpy as np
import pytest

import workloads as W
from tests.golden.make_golden import load as load_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2506_03127_gb300 import Propagator, build  # noqa: E402

build.build()

RHO_TOL_FP64 = 1e-10

# (case id, workload, steps, golden file, max_paths, complex64 bound).  The
# bounds: FP32 unit roundoff u = 2^-24 ~ 6e-8 per operation, a few tens of
# roundings per amplitude and step, unbiased (the propagator table's own
# rounding error is carried, so no error enters every step with one sign):
# rho errors grow like a random walk over the steps.  Measured worst cases
# are 2e-7 (100 steps of the 8-step model), 4.5e-7 (200 structured steps),
# 2.3e-7 (chain), 1.2e-6 (117 steps, 65536 paths); each bound is about four
# times the measured value.
CASES = [
    ("cfg1", W.SPIN_BOSON_OHMIC_DK8, 100, "spin_boson_ohmic_dk8_rho.txt", 1 << 20, 1e-6),
    ("cfg2_200", W.SPIN_BOSON_STRUCTURED_DK16, 200, "spin_boson_structured_dk16_rho200.txt", 1 << 21, 2e-6),
    ("chain3_dk7", W.CHAIN3_STRUCTURED_DK7, 60, "chain3_structured_dk7_rho60.txt", 1 << 22, 1e-6),
    ("chain3_dk12_t10", W.CHAIN3_STRUCTURED_DK12, 10, "chain3_structured_dk12_rho10.txt", 1 << 26, 1e-6),
    ("tls_dk8", W.tls_ohmic_full(8), 117, "tls_ohmic_full_dk8_rho117.txt", 1 << 18, 5e-6),
    ("tls_dk10", W.tls_ohmic_full(10), 30, "tls_ohmic_full_dk10_rho30.txt", 1 << 21, 1e-6),
]


def run(w, steps, precision, engine, max_paths):
    p = Propagator.from_workload(w, precision=precision, engine=engine, max_paths=max_paths)
    p.step(steps)
    p.sync()
    rho = p.rho(0, steps + 1)
    kept = [s[3] for s in p.stats(1, steps)]
    p.close()
    return rho, np.array(kept)


@pytest.mark.parametrize("engine", ["stream", "hash"])
@pytest.mark.parametrize("cid,w,steps,fname,max_paths,bound", CASES, ids=[c[0] for c in CASES])
def test_complex64_within_stated_bound_of_oracle(cid, w, steps, fname, max_paths, bound, engine):
    t, n, rho_o = load_golden(fname)
    rho, kept = run(w, steps, "c64", engine, max_paths)
    err = np.abs(rho - rho_o).max(axis=(1, 2))
    print(f"{cid} {engine} c64: max err {err.max():.3e} at t={int(err.argmax())}")
    assert err.max() <= bound, (cid, engine, err.max(), int(err.argmax()))
    # filter decisions on sums of nearly cancelling members (whose relative
    # complex64 error is large) may differ: survivor counts within 0.5 %
    rel = np.abs(kept - n[1:]) / np.maximum(n[1:], 1)
    print(f"{cid} {engine} c64: survivor counts within {rel.max():.2e} of the oracle's")
    assert rel.max() <= 5e-3, (cid, engine, rel.max())


@pytest.mark.parametrize("engine", ["stream", "hash"])
@pytest.mark.parametrize("cid,w,steps,fname,max_paths,bound",
                         [c for c in CASES if c[0] != "cfg1"], ids=[c[0] for c in CASES if c[0] != "cfg1"])
def test_fp64_on_the_same_trajectories(cid, w, steps, fname, max_paths, bound, engine):
    t, n, rho_o = load_golden(fname)
    rho, kept = run(w, steps, "fp64", engine, max_paths)
    assert np.abs(rho - rho_o).max() <= RHO_TOL_FP64, (cid, engine, np.abs(rho - rho_o).max())
    np.testing.assert_array_equal(kept, n[1:])
