"""Adaptive time stepping: rebuilding only the active levels (fmm_set_levels
with lo > lmin) and solving levels lo..lmax must give what a full rebuild and
solve of the same masses gives (the far field of a box does not depend on the
target level, so stale coarse levels are exactly their last stored masses),
and the FP64 path must match the oracle's subcycle solve."""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W
from _parity import ORACLE_FP64, SELF_MIXED, check, self_tol

pytestmark = pytest.mark.gpu


def _perturb(h, lo, i):
    g = h.copy()
    for k in range(lo - h.lmin, len(h.mass)):
        g.mass[k] = h.mass[k] * (1.0 + 1e-3 * (2 * W.uniform(77, 1000 * i + k, np.arange(h.mass[k].size)) - 1))
    return g


def test_ats_schedule_equals_full_solves_mixed():
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.lognormal_amr(base=6, seed=6)
    sched = W.ats_schedule(h.lmin, h.lmax)
    s = fmm.Solver(6, "mixed", out_fp32=True)
    s.set_hierarchy(h)
    ref = fmm.Solver(6, "mixed", out_fp32=True)
    cur = h
    for i, lo in enumerate(sched):
        cur = _perturb(cur, lo, i)
        s.set_hierarchy(cur, lo=lo)
        phi, acc = s.solve(lo)
        ref.set_hierarchy(cur)
        rphi, racc = ref.solve()
        torch.cuda.synchronize()
        s.sync()
        ref.sync()
        got = {l: acc[l].double().cpu().numpy() for l in acc}
        want = {l: racc[l].double().cpu().numpy() for l in acc}
        gotp = {l: phi[l].double().cpu().numpy() for l in phi}
        wantp = {l: rphi[l].double().cpu().numpy() for l in phi}
        check(gotp, got, wantp, want, SELF_MIXED, f"ATS step {i} lo={lo}", h=cur)


def test_ats_subcycle_fp64_matches_oracle():
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.lognormal_amr(base=5, seed=6)
    s = fmm.Solver(4, "fp64")
    s.set_hierarchy(h)
    s.solve()
    cur = _perturb(h, h.lmax, 1)
    s.set_hierarchy(cur, lo=h.lmax)  # rebuild of the finest level only
    phi, acc = s.solve(h.lmax)
    torch.cuda.synchronize()
    s.sync()
    sel = {h.lmax: np.unique((W.uniform(5, 9, np.arange(300)) * h.n(h.lmax)).astype(np.int64))}
    ref_p, ref_a = oracle.solve(cur, 4, lo=h.lmax, sel=sel)
    got = {h.lmax: acc[h.lmax].cpu().numpy()[sel[h.lmax]]}
    gotp = {h.lmax: phi[h.lmax].cpu().numpy()[sel[h.lmax]]}
    check(gotp, got, ref_p, ref_a, ORACLE_FP64, "ATS subcycle fp64", h=cur, sel=sel)


def _unrefine_one(h, level, seed):
    """h with one refined cell of `level` merged into a leaf (its 8 children, leaves of
    the finest level, replaced by their total mass).  The cells of `level` keep their
    set, so this is a valid partial update from `level`."""
    k = level - h.lmin
    g = h.copy()
    child = g.ijk[k + 1]
    par = child // 2
    keys, inv = np.unique(par, axis=0, return_inverse=True)
    pick = int(W.uniform(seed, 1, 0) * keys.shape[0])
    sel = inv.reshape(-1) == pick
    g.ijk[k] = np.ascontiguousarray(np.concatenate([g.ijk[k], keys[pick][None, :].astype(np.int32)]))
    g.mass[k] = np.concatenate([g.mass[k], [g.mass[k + 1][sel].sum()]])
    g.ijk[k + 1] = np.ascontiguousarray(child[~sel])
    g.mass[k + 1] = g.mass[k + 1][~sel]
    return g


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_incremental_updates_equal_full_rebuilds(precision):
    """Partial rebuilds (set_levels from lo) followed by solves from lo, including a
    change of refinement above lo, against a fresh full build and solve."""
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.lognormal_amr(base=5, seed=6)
    assert h.lmax == h.lmin + 2
    s = fmm.Solver(6, precision)
    s.set_hierarchy(h)
    s.solve()
    ref = fmm.Solver(6, precision)
    steps = [(h.lmax, None), (h.lmin + 1, "unrefine"), (h.lmax, None), (h.lmin + 1, None), (h.lmin, None)]
    cur = h
    for i, (lo, change) in enumerate(steps):
        cur = _unrefine_one(cur, lo, seed=i) if change else _perturb(cur, lo, i)
        s.set_hierarchy(cur, lo=lo)
        phi, acc = s.solve(lo)
        ref.set_hierarchy(cur)
        rphi, racc = ref.solve()
        torch.cuda.synchronize()
        s.sync()
        ref.sync()
        got = {l: acc[l].double().cpu().numpy() for l in acc}
        want = {l: racc[l].double().cpu().numpy() for l in acc}
        gotp = {l: phi[l].double().cpu().numpy() for l in phi}
        wantp = {l: rphi[l].double().cpu().numpy() for l in phi}
        check(gotp, got, wantp, want, self_tol(precision), f"update {i} lo={lo} {precision}", h=cur)


def test_partial_update_must_keep_its_lowest_level():
    from paper_2607_19489_b300 import fmm
    h = W.lognormal_amr(base=5, seed=6)
    s = fmm.Solver(4, "fp64")
    s.set_hierarchy(h)
    bad = _unrefine_one(h, h.lmin + 1, seed=3)   # changes the cells of level lmin + 2
    with pytest.raises(fmm.FMMError) as e:
        s.set_hierarchy(bad, lo=h.lmin + 2)
    assert e.value.code == -8  # FMM_ERR_STATE
    # the rejected call already replaced its levels: a full set_levels comes next,
    # after which the same change as an update from one level coarser is accepted
    s.set_hierarchy(h)
    s.solve()
    s.set_hierarchy(bad, lo=h.lmin + 1)
    phi, acc = s.solve(h.lmin + 1)
    s.sync()
    ref_p, ref_a = oracle.solve(bad, 4, lo=h.lmin + 1)
    got = {l: acc[l].cpu().numpy() for l in acc}
    gotp = {l: phi[l].cpu().numpy() for l in phi}
    check(gotp, got, ref_p, ref_a, ORACLE_FP64, "update after a rejected one", h=bad)
