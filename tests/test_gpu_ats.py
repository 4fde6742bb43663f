"""Adaptive time stepping: rebuilding only the active levels (fmm_set_levels
with lo > lmin) and solving levels lo..lmax must give what a full rebuild and
solve of the same masses gives (the far field of a box does not depend on the
target level, so stale coarse levels are exactly their last stored masses),
and the FP64 path must match the oracle's subcycle solve."""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _rel(got, ref):
    num = sum(((got[l] - ref[l]) ** 2).sum() for l in ref)
    den = sum((ref[l] ** 2).sum() for l in ref)
    return float(np.sqrt(num / den))


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
        assert _rel(got, want) <= 1e-5


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
    assert _rel(got, ref_a) <= 1e-10
