"""Periodic boundaries on the GPU against the oracle's periodic FMM.

Unigrids of 8^3 to 32^3 (level-1 M2L and the lattice term carry most of the
far field at 8^3), random graded AMR (also moved by half the box, so that its
refined regions cross the box edge) and a two-level workload whose refined
block sits inside the box, in FP64, split-BF16 and TF32; a subcycle (lo >
lmin); a mass update; the rejections.  FP64 has the plain relative bars; the
reduced precisions measure errors against the field scale G M_total / L when
the periodic field is smaller than it (tests/_parity.py says why)."""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W
from _parity import ORACLE_TF32_PERIODIC, PERIODIC_PHI_FLOOR, check as _check, oracle_tol as _oracle_tol

pytestmark = pytest.mark.gpu


def oracle_tol(precision):
    return ORACLE_TF32_PERIODIC if precision == "tf32" else _oracle_tol(precision)


def check(gp, ga, rp, ra, tol, what, h=None, sel=None):
    """The parity check; reduced precisions against max(RMS, G M_total)."""
    scale = 0.0 if tol is _oracle_tol("fp64") else float(h.total_mass())
    return _check(gp, ga, rp, ra, tol, what, h=h, sel=sel, floors={"phi": PERIODIC_PHI_FLOOR},
                  scales={"phi": scale, "accel": scale})


def run(h, p, precision, sel=None, lo=None, **kw):
    import torch
    from paper_2607_19489_b300 import fmm
    s = fmm.Solver(p, precision, periodic=True, **kw)
    s.set_hierarchy(h)
    phi, acc = s.solve(lo)
    torch.cuda.synchronize()
    s.sync()
    out_p = {l: phi[l].double().cpu().numpy() for l in phi}
    out_a = {l: acc[l].double().cpu().numpy() for l in acc}
    if sel is not None:
        out_p = {l: out_p[l][sel[l]] for l in sel}
        out_a = {l: out_a[l][sel[l]] for l in sel}
    return out_p, out_a


def _sel(h, n, seed):
    rng = np.random.default_rng(seed)
    return {l: np.sort(rng.choice(h.n(l), min(n, h.n(l)), replace=False)) for l in h.levels if h.n(l)}


def _across_edge():
    """random_amr(3, 5, 13) moved by half the box: its refined regions cross the box edge."""
    h = W.random_amr(3, 5, seed=13).copy()
    for k, l in enumerate(h.levels):
        s = 4 << (l - h.lmin)
        h.ijk[k] = np.ascontiguousarray(((h.ijk[k].astype(np.int64) + s) % (1 << l)).astype(np.int32))
    return h


CASES = {
    "unigrid8": (lambda: W.unigrid_plummer(3, noise=0.3, seed=2), None),
    "unigrid16": (lambda: W.unigrid_plummer(4, noise=0.3, seed=3), None),
    "unigrid32": (lambda: W.unigrid_plummer(5, noise=0.3, seed=4), 2500),
    "amr_3_5": (lambda: W.random_amr(3, 5, seed=13), None),
    "twolevel16": (lambda: W.two_level_plummer(base=4, lo=4, hi=12, seed=3), None),
    "amr_across_edge": (_across_edge, None),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed", "tf32"])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("p", [4, 6])
def test_matches_oracle(name, p, precision):
    make, nsel = CASES[name]
    h = make()
    sel = _sel(h, nsel, 1) if nsel else None
    rp, ra = oracle.solve_periodic(h, p, sel=sel)
    gp, ga = run(h, p, precision, sel=sel)
    check(gp, ga, rp, ra, oracle_tol(precision), f"periodic {precision} {name} p={p}", h=h, sel=sel)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_other_orders_and_pm(precision):
    h = W.random_amr(3, 5, seed=19)
    for p, pm in ((2, 0), (3, 2), (8, 0)):
        rp, ra = oracle.solve_periodic(h, p, p_m=pm or None)
        gp, ga = run(h, p, precision, p_m=pm or None)
        check(gp, ga, rp, ra, oracle_tol(precision), f"periodic {precision} p={p} p_m={pm}", h=h)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_subcycle_and_mass_update(precision):
    """A solve of the finest level only (lo > lmin) after new masses on it."""
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.random_amr(3, 5, seed=13)
    s = fmm.Solver(6, precision, periodic=True)
    s.set_hierarchy(h)
    s.solve()
    h2 = h.copy()
    h2.mass[-1] = h2.mass[-1][::-1].copy()
    s.update_masses([torch.as_tensor(h2.mass[-1], device="cuda")], lo=h.lmax)
    phi, acc = s.solve(h.lmax)
    torch.cuda.synchronize()
    s.sync()
    gp = {h.lmax: phi[h.lmax].double().cpu().numpy()}
    ga = {h.lmax: acc[h.lmax].double().cpu().numpy()}
    rp, ra = oracle.solve_periodic(h2, 6, lo=h.lmax)
    check(gp, ga, rp, ra, oracle_tol(precision), f"periodic {precision} subcycle", h=h2)


def test_rejections():
    import torch
    from paper_2607_19489_b300 import fmm
    with pytest.raises(fmm.FMMError):
        fmm.Solver(4, "mixed", periodic=True, bottom="m2l")
    with pytest.raises(fmm.FMMError):
        fmm.Solver(4, "mixed", periodic=True, delta_l=2)
    s = fmm.Solver(4, "fp64", periodic=True)
    with pytest.raises(fmm.FMMError) as e:
        s.set_hierarchy(W.unigrid_plummer(2))
    assert e.value.name == "FMM_ERR_ARG"
    refined = W.nested_boxes(3, [(0, 4), (0, 4)])  # graded inside the box, not across its edge
    leaves = W.leaves_from_refined(3, 5, refined)
    hc = W.Hierarchy(3, 5, [np.ascontiguousarray(c, dtype=np.int32) for c in leaves],
                     [np.ones(c.shape[0]) for c in leaves])
    with pytest.raises(fmm.FMMError) as e:
        s.set_hierarchy(hc)
    assert e.value.name == "FMM_ERR_NOT_GRADED"
    h = W.unigrid_plummer(3, noise=0.3, seed=2)
    s.set_hierarchy(h)
    with pytest.raises(fmm.FMMError):
        s.direct_sum(3, torch.arange(4, device="cuda"))
    with pytest.raises(fmm.FMMError):
        s.solve_adjoint({3: torch.ones(h.n(3), dtype=torch.float64, device="cuda")},
                        {3: torch.zeros(h.n(3), 3, dtype=torch.float64, device="cuda")})
    # the context stays usable
    phi, acc = s.solve()
    rp, ra = oracle.solve_periodic(h, 4)
    check({3: phi[3].double().cpu().numpy()}, {3: acc[3].double().cpu().numpy()}, rp, ra,
          oracle_tol("fp64"), "periodic after rejections", h=h)
