"""GPU: masked merging where the mathematics makes it exact.

With eta_d = 0 from lag `cut` on, a merge on the prefix mask {0 .. k-1}
(plus older positions) drops only positions that meet no later new point
within the memory, so the masked run equals QUAPI with memory `cut`: k for
the pre-merge on P' (Sec. 3.1), k + 1 for the merge on P after extension
(Sec. 2.1).  The oracle's pins show both against brute-force enumeration.
Every engine (stream tile kernel with and without sub-groups, merge table,
post-merging sort engine, wide keys) is compared here with that exact
trajectory (the unmasked oracle at memory `cut`), not with the oracle's
masked run; the FP64 group and survivor counts must also equal the masked
oracle's.
"""
import numpy as np
import pytest

from oracle import iquapi
from tests.test_oracle_pins import PREFIX_CASES, prefix_case, prefix_cut

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2506_03127_gb300 import Propagator, WidePropagator, build  # noqa: E402

build.build()

TOL = {"fp64": 1e-10, "c64": 2e-6}
STEPS = {2: 14, 3: 10, 5: 6}
CASES = PREFIX_CASES + [(2, 8, 3, ()), (3, 6, 3, ())]


def stream_accepts(M, dkmax, mask):
    """The stream engine takes P' = a prefix {0 .. j} and, for M = 2, one
    more position (runs split into sub-groups)."""
    Pp = iquapi.premerge_positions(mask, dkmax)
    nextra = sum(1 for i, p in enumerate(Pp) if p != i)
    return M <= 4 and (nextra == 0 or (nextra == 1 and M == 2))


def _exact(c, M, cut, steps):
    return iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"][:cut], cut, None, 0.0, c["rho0"], steps)


def _run(p, c, steps):
    p.set_eta(c["eta"])
    p.set_mask(c["mask"])
    p.set_rho0(c["rho0"])
    p.step(steps)
    rho = p.rho(0, steps + 1)
    stats = p.stats(1, steps)
    p.close()
    return rho, stats


@pytest.mark.parametrize("precision", ["fp64", "c64"])
@pytest.mark.parametrize("engine", ["stream", "hash"])
@pytest.mark.parametrize("M,dkmax,k,extras", [c for c in CASES if c[0] <= 4])
def test_premerge_engines_exact_on_prefix_masks(M, dkmax, k, extras, engine, precision):
    cut = prefix_cut("pre", k)
    c = prefix_case(M, dkmax, k, extras, cut)
    if engine == "stream" and not stream_accepts(M, dkmax, c["mask"]):
        pytest.skip("mask outside the stream engine's form")
    steps = STEPS[M]
    p = Propagator(M, dkmax, c["dt"], c["q"], c["hs"], 0.0, precision, engine, max_paths=1 << 20)
    rho, stats = _run(p, c, steps)
    err = np.abs(rho - _exact(c, M, cut, steps).rho).max()
    assert err <= TOL[precision], err
    if precision == "fp64":
        o = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, c["mask"], 0.0, c["rho0"], steps)
        assert [(s[1], s[3]) for s in stats] == [(s.groups, s.kept) for s in o.stats]


@pytest.mark.parametrize("precision", ["fp64", "c64"])
@pytest.mark.parametrize("M,dkmax,k,extras", [c for c in CASES if c[0] <= 4])
def test_postmerge_engine_exact_on_prefix_masks(M, dkmax, k, extras, precision):
    cut = prefix_cut("post", k)
    c = prefix_case(M, dkmax, k, extras, cut)
    steps = STEPS[M]
    p = Propagator(M, dkmax, c["dt"], c["q"], c["hs"], 0.0, precision, max_paths=1 << 20, scheme="post")
    rho, _ = _run(p, c, steps)
    err = np.abs(rho - _exact(c, M, cut, steps).rho).max()
    assert err <= TOL[precision], err


@pytest.mark.parametrize("precision", ["fp64", "c64"])
@pytest.mark.parametrize("M,dkmax,k,extras", CASES)
def test_wide_keys_exact_on_prefix_masks(M, dkmax, k, extras, precision):
    cut = prefix_cut("pre", k)
    c = prefix_case(M, dkmax, k, extras, cut)
    steps = STEPS[M]
    p = WidePropagator(M, dkmax, c["dt"], c["q"], c["hs"], 0.0, precision, max_paths=1 << 20)
    rho, stats = _run(p, c, steps)
    err = np.abs(rho - _exact(c, M, cut, steps).rho).max()
    assert err <= TOL[precision], err
    if precision == "fp64":
        o = iquapi.propagate(M, c["q"], c["hs"], c["dt"], c["eta"], dkmax, c["mask"], 0.0, c["rho0"], steps)
        assert [s[3] for s in stats] == [s.kept for s in o.stats]


def test_stream_engine_takes_the_sub_group_cases():
    """At least one case runs the tile kernel with sub-groups (M = 2, one
    extra P' position) and one without."""
    forms = set()
    for M, dkmax, k, extras in CASES:
        mask = tuple(range(k)) + tuple(extras)
        if M <= 4 and stream_accepts(M, dkmax, mask):
            forms.add(len(iquapi.premerge_positions(mask, dkmax)) > k - 1)
    assert forms == {True, False}
