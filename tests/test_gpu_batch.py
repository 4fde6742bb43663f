"""Batched solves (fmm_batch_solve), the autotuner and shared translation
tables.  A batch must give every hierarchy the result of its own solve; FP64
batches match the oracle to the FP64 bar, mixed batches match the
contexts' own solves to float rounding (the tensor-core epilogues add with
atomics, so the order of additions may differ)."""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W
from _parity import ORACLE_FP64, SELF_MIXED, check, oracle_tol

pytestmark = pytest.mark.gpu


def _np(out):
    import torch
    torch.cuda.synchronize()
    phi, acc = out
    return {l: phi[l].double().cpu().numpy() for l in phi}, {l: acc[l].double().cpu().numpy() for l in acc}


def small_batch(n=6, seed=3):
    return W.batched_blobs(count=n, seed=seed, bases=(4,))


def test_fp64_batch_matches_oracle():
    from paper_2607_19489_b300 import fmm
    hs = small_batch()
    solvers = []
    for h in hs:
        s = fmm.Solver(4, "fp64")
        s.set_hierarchy(h)
        solvers.append(s)
    outs = fmm.batch_solve(solvers)
    for s in solvers:
        s.sync()
    for h, out in zip(hs, outs):
        got_p, got_a = _np(out)
        ref_p, ref_a = oracle.solve(h, 4)
        check(got_p, got_a, ref_p, ref_a, ORACLE_FP64, "fp64 batch", h=h)


@pytest.mark.parametrize("p", [4, 6])
def test_mixed_batch_matches_own_solves(p):
    from paper_2607_19489_b300 import fmm
    hs = small_batch(8, seed=p)
    solvers, own = [], []
    for h in hs:
        s = fmm.Solver(p, "mixed")
        s.set_hierarchy(h)
        own.append(_np(s.solve()))
        solvers.append(s)
    outs = fmm.batch_solve(solvers)
    outs = fmm.batch_solve(solvers, outs=outs)  # replay of the cached graph
    for s in solvers:
        s.sync()
    for o, ref in zip(outs, own):  # same kernels; atomics may add in another order
        got_p, got_a = _np(o)
        check(got_p, got_a, ref[0], ref[1], SELF_MIXED, f"mixed batch p={p} vs own solve")


def test_batch_follows_hierarchy_changes_and_subcycles():
    from paper_2607_19489_b300 import fmm
    hs = small_batch(4, seed=9)
    other = small_batch(4, seed=10)
    solvers = []
    for h in hs:
        s = fmm.Solver(4, "fp64")
        s.set_hierarchy(h)
        solvers.append(s)
    fmm.batch_solve(solvers)
    solvers[1].set_hierarchy(other[1])   # new layout for one member: a new graph
    hs[1] = other[1]
    los = [h.lmax for h in hs]           # fine-level-only solves
    outs = fmm.batch_solve(solvers, los=los)
    for s in solvers:
        s.sync()
    for h, lo, out in zip(hs, los, outs):
        got_p, got_a = _np(out)
        ref_p, ref_a = oracle.solve(h, 4, lo=lo)
        check(got_p, got_a, ref_p, ref_a, ORACLE_FP64, f"fp64 batch lo={lo}", h=h)


def test_autotune_keeps_results():
    from paper_2607_19489_b300 import fmm
    h = W.two_level_plummer(base=5, lo=12, hi=20, seed=3)
    s = fmm.Solver(6, "mixed")
    s.set_hierarchy(h)
    before = _np(s.solve())
    t = s.autotune()
    assert t["split_m2p"] >= 0 and t["split_m2l"] >= 0 and t["near_octs_per_block"] in (4, 8, 16, 32)
    after = _np(s.solve())
    s.sync()
    # another split-K factor sums the FP32 partial products in another order
    check(after[0], after[1], before[0], before[1], SELF_MIXED, "after autotune")
    s2 = fmm.Solver(6, "mixed")
    s2.set_hierarchy(h)
    s2.set_tuning(t)
    assert s2.tuning() == t
    again = _np(s2.solve())
    s2.sync()
    check(again[0], again[1], before[0], before[1], SELF_MIXED, "tuning set on another context")


def test_shared_tables_survive_their_creator():
    import gc
    from paper_2607_19489_b300 import fmm
    h = small_batch(1, seed=4)[0]
    ref_p, ref_a = oracle.solve(h, 4)
    first = fmm.Solver(4, "fp64")
    others = [fmm.Solver(4, "fp64") for _ in range(2)]
    first.close() if hasattr(first, "close") else None
    del first
    gc.collect()
    for s in others:
        s.set_hierarchy(h)
        got_p, got_a = _np(s.solve())
        s.sync()
        check(got_p, got_a, ref_p, ref_a, ORACLE_FP64, "shared tables", h=h)
    del others
    gc.collect()
    s = fmm.Solver(4, "fp64")
    s.set_hierarchy(h)
    got_p, got_a = _np(s.solve())
    s.sync()
    check(got_p, got_a, ref_p, ref_a, ORACLE_FP64, "tables rebuilt", h=h)


def test_trailing_empty_levels():
    """lmax above the finest populated level (nothing refined there yet)."""
    from paper_2607_19489_b300 import fmm
    h = small_batch(1, seed=4)[0]
    e = W.Hierarchy(h.lmin, h.lmax + 2, [a for a in h.ijk] + [np.zeros((0, 3), np.int32)] * 2,
                    [m for m in h.mass] + [np.zeros(0)] * 2, "with empty levels")
    ref_p, ref_a = oracle.solve(h, 4)
    for precision in ("fp64", "mixed"):
        s = fmm.Solver(4, precision)
        s.set_hierarchy(e)
        phi, acc = s.solve()
        s.sync()
        assert acc[e.lmax].shape[0] == 0
        got_p, got_a = _np((phi, acc))
        check({l: got_p[l] for l in h.levels}, {l: got_a[l] for l in h.levels}, ref_p, ref_a,
              oracle_tol(precision), f"trailing empty levels {precision}", h=h)
        assert s.tree_counts()[e.lmax] == 0
        phi2, acc2 = s.solve(lo=e.lmax)  # a subcycle of an empty level: nothing to do
        s.sync()
