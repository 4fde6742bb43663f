"""Pins of the oracle's Delta l = 2 variant (footnote of Sec. 2) on unigrids.

With Delta l = 2 the finest FMM box is the 4^3 block of cells two levels up:
the near field of a target is every cell of the 3^3 blocks around its own
(12^3 cells), the bottom intermediate field the M2P from the interaction list
of its block, and the far field the L2P of the block's parent.  The pins tie
each region to the O(N^2) direct sum:
  * on 8^3 every cell lies in the near field: the variant is the direct sum;
  * masses confined to the 12^3 neighbourhood of one target's block reach that
    target only through the near field: exact there, while Delta l = 1 (whose
    near field is the 6^3 neighbourhood) approximates part of them;
  * masses outside that neighbourhood reach it only through M2P and L2P: the
    error falls with p;
  * on whole grids the error falls monotonically with p, and, as the paper
    reports, is nearly the same as that of Delta l = 1 on 32^3.
"""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W


def rel_rms(a, b):
    num = sum(float(((a[l] - b[l]) ** 2).sum()) for l in b)
    den = sum(float((b[l] ** 2).sum()) for l in b)
    return float(np.sqrt(num / den))


def test_all_near_field_on_8cubed_is_the_direct_sum():
    h = W.unigrid_plummer(3, noise=0.3, seed=5)
    dp, da = oracle.direct(h)
    for p in (2, 6):
        ph, ac = oracle.solve_dl2(h, p)
        assert rel_rms(ac, da) < 1e-13 and rel_rms(ph, dp) < 1e-13


def _confined(level, t_ijk, inside: bool, seed=3):
    """Unigrid with random masses inside (or only outside) the 3^3 level-(l-2)
    blocks around the block of cell t_ijk."""
    h = W.unigrid_plummer(level, noise=0.0, seed=1).copy()
    ijk = h.ijk[0]
    G = np.asarray(t_ijk) >> 2
    near = np.all(np.abs((ijk >> 2) - G) <= 1, axis=1)
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.5, 1.5, ijk.shape[0])
    m[~near if inside else near] = 0.0
    h.mass[0] = m
    t = int(np.nonzero(np.all(ijk == np.asarray(t_ijk), axis=1))[0][0])
    return h, {level: np.array([t], np.int64)}


@pytest.mark.parametrize("t_ijk", [(13, 18, 9), (0, 31, 4), (16, 16, 16)])
def test_near_field_is_the_12cubed_neighbourhood(t_ijk):
    h, sel = _confined(5, t_ijk, inside=True)
    dp, da = oracle.direct(h, sel=sel)
    ph, ac = oracle.solve_dl2(h, 6, sel=sel)
    assert rel_rms(ac, da) < 1e-13 and rel_rms(ph, dp) < 1e-13
    # Delta l = 1 reaches the outer part of that block through M2P: not exact
    p1, a1 = oracle.solve(h, 6, sel=sel)
    assert rel_rms(a1, da) > 1e-8


def test_outside_the_neighbourhood_converges_with_p():
    h, sel = _confined(5, (13, 18, 9), inside=False)
    dp, da = oracle.direct(h, sel=sel)
    errs = [rel_rms(oracle.solve_dl2(h, p, sel=sel)[1], da) for p in (2, 4, 6, 8)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4, errs


def test_16cubed_converges_to_the_direct_sum():
    h = W.unigrid_plummer(4, noise=0.3, seed=5)
    dp, da = oracle.direct(h)
    errs = []
    for p in (2, 4, 6, 8):
        ph, ac = oracle.solve_dl2(h, p)
        errs.append((rel_rms(ac, da), rel_rms(ph, dp)))
    for k in range(2):
        seq = [e[k] for e in errs]
        assert all(b < 0.5 * a for a, b in zip(seq, seq[1:])), errs
    assert errs[-1][0] < 2e-5 and errs[-1][1] < 2e-6, errs


def test_32cubed_matches_delta_l_1_accuracy():
    h = W.unigrid_plummer(5, noise=0.3, seed=5)
    rng = np.random.default_rng(0)
    sel = {5: np.sort(rng.choice(h.n(5), 300, replace=False))}
    dp, da = oracle.direct(h, sel=sel)
    prev = None
    for p in (4, 6, 8):
        e2 = rel_rms(oracle.solve_dl2(h, p, sel=sel)[1], da)
        e1 = rel_rms(oracle.solve(h, p, sel=sel)[1], da)
        assert 0.5 < e2 / e1 < 2.0, (p, e2, e1)
        if prev is not None:
            assert e2 < prev
        prev = e2
    assert prev < 1e-3


def test_rejects_amr_and_small_grids():
    with pytest.raises(oracle.OracleError):
        oracle.solve_dl2(W.unigrid_plummer(2), 4)
    h = W.random_amr(3, 4, seed=1)
    assert h.lmin != h.lmax
    with pytest.raises(oracle.OracleError):
        oracle.solve_dl2(h, 4)
