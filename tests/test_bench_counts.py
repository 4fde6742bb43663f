"""The benchmark's interaction counts (the numerators of its rooflines) against a
brute-force walk over every target on small hierarchies: for each leaf t at
level l with parent box F, the bottom intermediate field is the interaction
list of F (children of F's parent's 3^3 neighbours, minus F's 3^3
neighbours), and the near field the level-l positions of F's 3^3 neighbour
octs (Fig. 2)."""
import itertools
import os
import sys

import numpy as np
import pytest

from paper_2607_19489_b300 import workloads as W

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def brute(h):
    leaves = {l: set(map(tuple, h.ijk[k].tolist())) for k, l in enumerate(h.levels)}
    cells = {}
    for l in range(h.lmax, -1, -1):
        own = leaves.get(l, set())
        ref = {tuple(c >> 1 for c in x) for x in cells.get(l + 1, set())}
        cells[l] = own | ref
    refined = {l: {tuple(c >> 1 for c in x) for x in cells.get(l + 1, set())} for l in range(h.lmax + 1)}
    out = dict(m2p_pairs=0, p2p_pairs=0, nearest_pairs=0, near_m2p_pairs=0)
    rng6 = range(-2, 4)
    for l in h.levels:
        n = 1 << l
        for t in leaves[l]:
            F = tuple(c >> 1 for c in t)
            G = tuple(c >> 1 for c in F)
            for o in itertools.product(rng6, repeat=3):
                S = tuple(2 * g + d for g, d in zip(G, o))
                if min(S) < 0 or max(S) >= n // 2 or max(abs(a - b) for a, b in zip(S, F)) <= 1:
                    continue
                if S in refined[l - 1]:
                    out["m2p_pairs"] += 1
                elif S in leaves.get(l - 1, ()):
                    out["p2p_pairs"] += 1
            seen = set()
            for o in itertools.product(rng6, repeat=3):
                P = tuple(2 * f + d for f, d in zip(F, o))
                if min(P) < 0 or max(P) >= n:
                    continue
                N = tuple(c >> 1 for c in P)
                if N in leaves.get(l - 1, ()):
                    if N not in seen:
                        seen.add(N)
                        out["p2p_pairs"] += 1
                elif P in leaves[l]:
                    out["p2p_pairs"] += P != t
                elif P in refined[l]:
                    if max(abs(a - b) for a, b in zip(P, t)) <= 1:
                        out["nearest_pairs"] += 8
                    else:
                        out["near_m2p_pairs"] += 1
    return out


@pytest.mark.parametrize("h", [W.random_amr(3, 4, seed=13), W.two_level_plummer(base=3, lo=2, hi=6, seed=2),
                               W.unigrid_plummer(3)])
def test_work_counts_match_brute_force(h):
    got = bench.work_counts(h, chunk=37)   # a ragged chunk size
    want = brute(h)
    for k, v in want.items():
        assert got[k] == v, (k, got[k], v)
    assert got["targets"] == sum(h.n(l) for l in h.levels)
