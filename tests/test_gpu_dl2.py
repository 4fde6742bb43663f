"""The Delta l = 2 variant (footnote of Sec. 2) on the GPU against the oracle.

Unigrids of 8^3 (everything in the near field), 16^3 (M2P from the level-2
interaction lists, no M2L), 32^3 and 64^3 (M2L, L2L to level l-2, M2P from
level l-2, the 12^3 near field), in FP64, split-BF16 and TF32, at several
orders (operand rows of 10 to 165 coefficients per cell: ragged K segments).
Bars as for Delta l = 1 (relative RMS and per cell, tests/_parity.py)."""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W
from _parity import check, oracle_tol

pytestmark = pytest.mark.gpu


def run(h, p, precision, sel=None, **kw):
    import torch
    from paper_2607_19489_b300 import fmm
    s = fmm.Solver(p, precision, delta_l=2, **kw)
    s.set_hierarchy(h)
    phi, acc = s.solve()
    torch.cuda.synchronize()
    s.sync()
    out_p = {l: phi[l].double().cpu().numpy() for l in phi}
    out_a = {l: acc[l].double().cpu().numpy() for l in acc}
    if sel is not None:
        out_p = {l: out_p[l][sel[l]] for l in sel}
        out_a = {l: out_a[l][sel[l]] for l in sel}
    return out_p, out_a


def _grid(level, seed):
    return W.unigrid_plummer(level, noise=0.3, seed=seed)


def _sel(h, n, seed):
    rng = np.random.default_rng(seed)
    l = h.lmin
    return {l: np.sort(rng.choice(h.n(l), min(n, h.n(l)), replace=False))}


@pytest.mark.parametrize("precision", ["fp64", "mixed", "tf32"])
@pytest.mark.parametrize("level,p", [(3, 4), (4, 4), (4, 6), (5, 6)])
def test_matches_oracle(level, p, precision):
    h = _grid(level, 7 + level)
    sel = _sel(h, 3000, 1) if level >= 5 else None
    rp, ra = oracle.solve_dl2(h, p, sel=sel)
    gp, ga = run(h, p, precision, sel=sel)
    check(gp, ga, rp, ra, oracle_tol(precision), f"delta_l=2 {precision} {2**level}^3 p={p}", h=h, sel=sel)


@pytest.mark.parametrize("p", [2, 3, 8])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_other_orders_match_oracle(p, precision):
    h = _grid(4, 21)
    rp, ra = oracle.solve_dl2(h, p)
    gp, ga = run(h, p, precision)
    check(gp, ga, rp, ra, oracle_tol(precision), f"delta_l=2 {precision} 16^3 p={p}", h=h)


def test_multipole_order_matches_oracle():
    h = _grid(5, 3)
    sel = _sel(h, 2000, 2)
    rp, ra = oracle.solve_dl2(h, 3, sel=sel, p_m=2)
    gp, ga = run(h, 3, "mixed", sel=sel, p_m=2)
    check(gp, ga, rp, ra, oracle_tol("mixed"), "delta_l=2 (p_m, p) = (2, 3)", h=h, sel=sel)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_unigrid64_p6_sampled(precision):
    h = _grid(6, 4)
    sel = _sel(h, 600, 3)
    rp, ra = oracle.solve_dl2(h, 6, sel=sel)
    gp, ga = run(h, 6, precision, sel=sel)
    check(gp, ga, rp, ra, oracle_tol(precision), f"delta_l=2 {precision} 64^3 p=6", h=h, sel=sel)


def test_repeated_solves_and_mass_updates():
    """A second solve after new masses (the accumulators are zero between solves)."""
    import torch
    from paper_2607_19489_b300 import fmm
    h = _grid(5, 5)
    h2 = h.copy()
    h2.mass[0] = h2.mass[0][::-1].copy()
    sel = _sel(h, 1500, 4)
    s = fmm.Solver(6, "mixed", delta_l=2)
    s.set_hierarchy(h)
    s.solve()
    s.update_masses([torch.as_tensor(h2.mass[0], device="cuda")])
    phi, acc = s.solve()
    torch.cuda.synchronize()
    s.sync()
    l = h.lmin
    gp = {l: phi[l].double().cpu().numpy()[sel[l]]}
    ga = {l: acc[l].double().cpu().numpy()[sel[l]]}
    rp, ra = oracle.solve_dl2(h2, 6, sel=sel)
    check(gp, ga, rp, ra, oracle_tol("mixed"), "delta_l=2 after update_masses", h=h2, sel=sel)


def test_rejections():
    from paper_2607_19489_b300 import fmm
    with pytest.raises(fmm.FMMError):
        fmm.Solver(4, "mixed", delta_l=3)
    with pytest.raises(fmm.FMMError):
        fmm.Solver(4, "mixed", delta_l=2, bottom="m2l")
    s = fmm.Solver(4, "mixed", delta_l=2)
    with pytest.raises(fmm.FMMError) as e:
        s.set_hierarchy(W.random_amr(3, 5, seed=13))
    assert e.value.name == "FMM_ERR_ARG"
    with pytest.raises(fmm.FMMError):
        s.set_hierarchy(W.unigrid_plummer(2))
    # the context stays usable
    h = _grid(3, 1)
    s.set_hierarchy(h)
    phi, acc = s.solve()
    rp, ra = oracle.solve_dl2(h, 4)
    gp = {3: phi[3].double().cpu().numpy()}
    ga = {3: acc[3].double().cpu().numpy()}
    check(gp, ga, rp, ra, oracle_tol("mixed"), "delta_l=2 after rejections", h=h)
