"""CUDA-graph replay of fmm_solve against direct launches and the oracle.

A cached graph must never replay stale pointers or grid sizes: replacing the
hierarchy with one of other list lengths, or changing the output buffers,
captures a new graph, and its results match the oracle like the first."""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W
from _parity import ORACLE_FP64, check, oracle_tol, self_tol

pytestmark = pytest.mark.gpu
BITWISE = {"rms": 1e-14, "cell": 1e-13}


def _out(phi, acc):
    import torch
    torch.cuda.synchronize()
    return ({l: phi[l].double().cpu().numpy() for l in phi}, {l: acc[l].double().cpu().numpy() for l in acc})


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_follows_hierarchy_changes(precision):
    from paper_2607_19489_b300 import fmm
    s = fmm.Solver(4, precision)
    hs = [W.random_amr(3, 5, seed=13), W.two_level_plummer(base=4, lo=4, hi=12, seed=3), W.random_amr(3, 5, seed=13)]
    for h in hs:
        s.set_hierarchy(h)
        for _ in range(2):  # capture, then replay
            phi, acc = s.solve()
            s.sync()
            got_p, got_a = _out(phi, acc)
            ref_p, ref_a = oracle.solve(h, 4)
            check(got_p, got_a, ref_p, ref_a, oracle_tol(precision), f"graph replay {precision}", h=h)


def test_graph_and_direct_launches_agree():
    from paper_2607_19489_b300 import fmm
    import torch
    h = W.random_amr(3, 5, seed=19)
    s = fmm.Solver(4, "fp64")
    s.set_hierarchy(h)
    out = s.alloc_outputs()
    s.solve(out=out)
    s.sync()
    g_p, g_a = _out(*out)
    s.set_graphs(False)
    s.solve(out=out)
    s.sync()
    d_p, d_a = _out(*out)
    check(g_p, g_a, d_p, d_a, BITWISE, "graph vs direct launches")
    # replay into other output buffers
    s.set_graphs(True)
    out2 = s.alloc_outputs()
    for t in list(out2[0].values()) + list(out2[1].values()):
        t.fill_(float("nan"))
    s.solve(out=out2)
    s.sync()
    o_p, o_a = _out(*out2)
    check(o_p, o_a, d_p, d_a, BITWISE, "replay into other outputs")
    torch.cuda.synchronize()


def test_subcycle_solves_replay():
    """Alternating full and fine-level-only solves: one graph per lo."""
    from paper_2607_19489_b300 import fmm
    h = W.random_amr(3, 5, seed=13)
    s = fmm.Solver(4, "fp64")
    s.set_hierarchy(h)
    ref = {lo: oracle.solve(h, 4, lo=lo) for lo in (3, 4, 5)}
    for _ in range(2):
        for lo in (3, 5, 4, 5):
            phi, acc = s.solve(lo)
            s.sync()
            got_p, got_a = _out(phi, acc)
            check(got_p, got_a, ref[lo][0], ref[lo][1], ORACLE_FP64, f"subcycle replay lo={lo}", h=h)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_update_masses_equals_set_levels(precision):
    """Mass-only updates (no tree rebuild) of all levels and of the finest level."""
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.random_amr(3, 5, seed=13)
    s = fmm.Solver(4, precision)
    s.set_hierarchy(h)
    s.solve()
    ref = fmm.Solver(4, precision)
    cur = h.copy()
    for i, lo in enumerate([h.lmin, h.lmax, h.lmin + 1]):
        for k in range(lo - h.lmin, len(cur.mass)):
            cur.mass[k] = cur.mass[k] * (1 + 0.1 * W.uniform(3, 40 + i, np.arange(cur.mass[k].size)))
        s.update_masses([torch.as_tensor(m, device="cuda") for m in cur.mass[lo - h.lmin:]], lo=lo)
        phi, acc = s.solve()
        ref.set_hierarchy(cur)
        rphi, racc = ref.solve()
        s.sync()
        ref.sync()
        got_p, got_a = _out(phi, acc)
        want_p, want_a = _out(rphi, racc)
        check(got_p, got_a, want_p, want_a, self_tol(precision), f"mass update lo={lo} {precision}", h=cur)
