"""Plain FP64 CPU oracle for the MACGIC-iQUAPI per-step path update.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import or run anything in this package.  The CUDA library never calls it and
shares no code with it; the two meet only in the seeded inputs of
``workloads.py``.

Contents
  bath.py    spectral densities, Q(t) by quadrature, influence coefficients
             eta_d as second differences of Q (paper Eq. inf_fun; the
             formulas themselves are deferred by the paper to its refs).
  iquapi.py  the iterative path algorithm: pre-merging on the shifted mask
             (Sec. 3.1, Schemes merging/propagation), extension by the M^2 new
             forward/backward points with the bare propagator (Eqs. SysP0,
             SysP) and the influence factor (Eq. inf_fun), filtering
             (Sec. 2.1) and the reduced density matrix (Eq. quapi_red_rho).
  brute.py   the full path sum of Eq. quapi_red_rho enumerated path by path
             with the influence functional truncated at the memory length,
             for the right-box reading and for the symmetric Trotter
             splitting (intervals centred on the points, half intervals at
             both ends).

Parity status: every function is pinned by tests/test_oracle_pins.py against
closed forms or brute force; the filter (its rule |amp| >= theta and its
place before rho) by the filtered Markov map at memory length 1 and a
hand-made set; the pre-merge of keys wider than 64 bits (premerge_rows, no
packing) by equality with the packed pre-merge wherever both apply, ties at
the group maxima included.  The masked merge together with a nonzero bath is
pinned exactly where the mathematics fixes its result: on a prefix mask
with eta vanishing from the lag where the dropped positions would first
meet a new point, both orders equal unmasked QUAPI at that shorter memory
(brute force), and the pre-merge is no longer exact one lag further while
the merge after extension is, which pins the shift of P'.  Where the merge
is an approximation (eta beyond that lag) the paper prints no value
("parity unpinned" for that combination; pinned there only by invariants:
exactness at zero coupling, trace conservation without a filter, reduction
to the unmasked result for the full mask, and convergence to it as the
mask grows).
"""
