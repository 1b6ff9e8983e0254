"""Write the stored oracle trajectories used by the GPU parity tests.

Calls only oracle/ (and the input module workloads.py).  Each file holds one
line per time step t: t, the number of stored paths after the step, then
Re and Im of rho(t) row-major.  Regenerate with

    python tests/golden/make_golden.py [file ...]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import bath, iquapi  # noqa: E402


def write(w, steps, fname):
    eta = bath.eta_coefficients(w.bath, w.dt, w.dkmax)
    r = iquapi.propagate_workload(w, eta=eta, steps=steps)
    counts = [int(np.count_nonzero(w.rho0_array()))] + [s.kept for s in r.stats]
    with open(os.path.join(HERE, fname), "w") as f:
        f.write(f"# oracle trajectory of workload {w.name}, {steps} steps; "
                f"columns: t n_paths Re/Im rho row-major (M={w.M})\n")
        for t in range(steps + 1):
            vals = []
            for z in r.rho[t].reshape(-1):
                vals += [z.real, z.imag]
            f.write(f"{t} {counts[t]} " + " ".join(f"{v:.17e}" for v in vals) + "\n")


def load(fname):
    rows = np.loadtxt(os.path.join(HERE, fname), comments="#")
    t = rows[:, 0].astype(int)
    n = rows[:, 1].astype(np.int64)
    v = rows[:, 2:]
    rho = v[:, 0::2] + 1j * v[:, 1::2]
    M = int(round(np.sqrt(rho.shape[1])))
    return t, n, rho.reshape(-1, M, M)


# (workload, steps, file): the trajectories the GPU tests compare with.  The
# three-level chain with memory 12 stops at t = 10 (1.6e7 stored paths; the
# window fills at t = 12 with about 1e8, beyond what the oracle finishes in
# seconds); its memory-7 variant covers that model's merging steps.
GOLDEN = [
    (W.SPIN_BOSON_OHMIC_DK8, W.SPIN_BOSON_OHMIC_DK8.steps, "spin_boson_ohmic_dk8_rho.txt"),
    (W.SPIN_BOSON_STRUCTURED_DK16, 40, "spin_boson_structured_dk16_rho40.txt"),
    (W.SPIN_BOSON_STRUCTURED_DK16, 200, "spin_boson_structured_dk16_rho200.txt"),
    (W.CHAIN3_STRUCTURED_DK7, W.CHAIN3_STRUCTURED_DK7.steps, "chain3_structured_dk7_rho60.txt"),
    (W.CHAIN3_STRUCTURED_DK12, 10, "chain3_structured_dk12_rho10.txt"),
    (W.tls_ohmic_full(8), W.tls_ohmic_full(8).steps, "tls_ohmic_full_dk8_rho117.txt"),
    (W.tls_ohmic_full(10), 30, "tls_ohmic_full_dk10_rho30.txt"),
    # the first 10 steps of the memory-14 model (4^11 stored paths at t = 10);
    # while the window fills (t < memory) the trajectory does not depend on
    # the memory length, so these are also the first 10 steps at memory 13
    (W.tls_ohmic_full(14), 10, "tls_ohmic_full_dk14_rho10.txt"),
]

if __name__ == "__main__":
    only = set(sys.argv[1:])
    for w, steps, fname in GOLDEN:
        if not only or fname in only:
            write(w, steps, fname)
