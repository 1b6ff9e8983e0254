"""The ordering invariant behind the stream engine (reading R10), checked on
keys alone (no GPU).

The stored set is kept in M^2 regions by newest point, each region ordered
lexicographically by its older points (position 1 first).  Then for a
prefix P' = {0 .. k-1} every pre-merge group is a run of consecutive
entries; the children of the groups, visited region by region and run by
run, are appended to the region of their own new point, and that keeps
every region ordered, whatever the filter removes.  The simulation below
runs that data flow on random filters and checks both halves at every step.
"""
import numpy as np
import pytest


def _runs(region, k):
    """Groups on positions 0 .. k-1 as (start, end) runs of equal prefixes."""
    out, start = [], 0
    for i in range(1, len(region) + 1):
        if i == len(region) or region[i][:k] != region[start][:k]:
            out.append((start, i))
            start = i
    return out


@pytest.mark.parametrize("M,L,k,seed", [(2, 8, 3, 1), (2, 10, 9, 2), (3, 6, 4, 3), (4, 5, 2, 4)])
def test_prefix_groups_are_runs_and_children_keep_the_order(M, L, k, seed):
    rng = np.random.default_rng(seed)
    codes = M * M
    # t = 0: one path per nonzero element of rho0, a window of one point
    regions = {c: [(c,)] for c in range(codes) if rng.uniform() < 0.8 or c == 0}
    for t in range(1, L + 4):                          # the window fills, then merging steps
        full = t >= L                                   # the window holds L points; groups only then
        children = {c: [] for c in range(codes)}
        seen = set()
        for r in sorted(regions):                       # regions in order of their newest point
            reg = regions[r]
            # the invariant: ordered by the older points, so prefix groups are runs
            assert reg == sorted(reg), (t, r)
            groups = _runs(reg, k) if full else [(i, i + 1) for i in range(len(reg))]
            for s, e in groups:
                pre = reg[s][:k] if full else reg[s]
                assert pre not in seen                  # a group is one run, never split
                seen.add(pre)
                rep = reg[s]                            # any member: the order depends on the prefix only
                for c in range(codes):
                    if rng.uniform() < 0.55:            # the filter keeps a random subset
                        children[c].append(((c,) + rep)[:L])
        regions = {c: v for c, v in children.items() if v}
