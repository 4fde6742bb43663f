"""Adjoint solve (fmm_solve_adjoint) and its torch.autograd wrapper.

The solve is a linear map m -> (phi, accel); its adjoint must be the exact
transpose.  Checked three ways:
  * against the oracle's transpose on small graded hierarchies: column j of
    the oracle's map is its solve with a unit mass at cell j, so
    (A^T g)_j = <g, A e_j> (FP64 bar 1e-10, relative RMS);
  * the dot-product identity <g, A m> = <A^T g, m> on larger hierarchies,
    with A m the GPU forward solve;
  * central finite differences (h = 1e-6, FP64) of loss = sum_cells w . accel
    on 100 seeded cells of the nested two-Plummer hierarchy (32^3 base, two
    nested refined levels)."""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W
from _parity import ORACLE_FP64, check_arrays

pytestmark = pytest.mark.gpu


def nested(lmin, boxes, seed):
    refined = W.nested_boxes(lmin, boxes)
    lmax = lmin + len(boxes)
    leaves = W.leaves_from_refined(lmin, lmax, refined)
    h = W.Hierarchy(lmin, lmax, name=f"nested {boxes}")
    for k, c in enumerate(leaves):
        h.ijk.append(np.ascontiguousarray(c, dtype=np.int32))
        h.mass.append(W.uniform(seed, 50 + k, np.arange(c.shape[0])) + 0.1)
    return h


def cotangents(h, lo, seed):
    gp = {l: W.normal(seed, 100 + l, np.arange(h.n(l))) for l in range(lo, h.lmax + 1)}
    ga = {l: W.normal(seed, 200 + l, np.arange(3 * h.n(l))).reshape(-1, 3) for l in range(lo, h.lmax + 1)}
    return gp, ga


def oracle_transpose(h, p, gp, ga, lo):
    """(A^T g)_j = <g, A e_j>, one oracle solve per leaf."""
    out = {}
    for k, l in enumerate(h.levels):
        col = np.zeros(h.n(l))
        for j in range(h.n(l)):
            hj = W.Hierarchy(h.lmin, h.lmax, name="unit")
            hj.ijk = h.ijk
            hj.mass = [np.zeros_like(m) for m in h.mass]
            hj.mass[k][j] = 1.0
            phi, acc = oracle.solve(hj, p, lo=lo, threads=1)
            col[j] = sum(float(gp[t] @ phi[t]) + float((ga[t] * acc[t]).sum()) for t in gp)
        out[l] = col
    return out


def gpu_adjoint(h, p, gp, ga, lo):
    import torch
    from paper_2607_19489_b300 import fmm
    s = fmm.Solver(p, "fp64")
    s.set_hierarchy(h)
    g = s.solve_adjoint({l: torch.as_tensor(v, device="cuda") for l, v in gp.items()},
                        {l: torch.as_tensor(v, device="cuda").contiguous() for l, v in ga.items()}, lo=lo)
    s.sync()
    return {l: g[l].cpu().numpy() for l in g}, s


def rel_rms(got, ref):
    num = sum(((got[l] - ref[l]) ** 2).sum() for l in ref)
    den = sum((ref[l] ** 2).sum() for l in ref)
    return float(np.sqrt(num / den))


@pytest.mark.parametrize("boxes,lo_off", [([(0, 3), (2, 4)], 0), ([(1, 4), (4, 6)], 1)])
def test_adjoint_is_the_oracle_transpose(boxes, lo_off):
    h = nested(2, boxes, seed=7)
    lo = h.lmin + lo_off
    gp, ga = cotangents(h, lo, seed=11)
    ref = oracle_transpose(h, 4, gp, ga, lo)
    got, _ = gpu_adjoint(h, 4, gp, ga, lo)
    check_arrays(got, ref, ORACLE_FP64, "adjoint vs the oracle's transpose")


@pytest.mark.parametrize("name", ["random_amr", "two_level16", "nested_p6"])
def test_dot_product_identity(name):
    import torch
    from paper_2607_19489_b300 import fmm
    h, p = {"random_amr": (W.random_amr(3, 5, seed=13), 4),
            "two_level16": (W.two_level_plummer(base=4, lo=4, hi=12, seed=3), 4),
            "nested_p6": (nested(2, [(1, 4), (4, 6)], seed=5), 6)}[name]
    for lo in (h.lmin, h.lmax):
        gp, ga = cotangents(h, lo, seed=21)
        gm, s = gpu_adjoint(h, p, gp, ga, lo)
        phi, acc = s.solve(lo)
        s.sync()
        lhs = sum(float(gp[l] @ phi[l].cpu().numpy()) + float((ga[l] * acc[l].cpu().numpy()).sum()) for l in gp)
        rhs = sum(float(gm[l] @ h.mass[k]) for k, l in enumerate(h.levels))
        scale = sum(float(np.abs(gm[l]) @ np.abs(h.mass[k])) for k, l in enumerate(h.levels))
        assert abs(lhs - rhs) <= 1e-12 * scale
        torch.cuda.synchronize()


def test_finite_differences_nested_two_plummer():
    """loss = sum over cells of w . accel, seeded Gaussian w; central differences
    with h = 1e-6 (FP64) on 100 seeded cells."""
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.nested_two_plummer(base=5, boxes=((6, 26), (19, 45)))
    s = fmm.Solver(6, "fp64")
    ijk = [torch.as_tensor(a, device="cuda").contiguous() for a in h.ijk]
    mass = [torch.as_tensor(m, device="cuda").contiguous() for m in h.mass]
    w = {l: torch.as_tensor(W.normal(31, 300 + l, np.arange(3 * h.n(l))).reshape(-1, 3), device="cuda")
         for l in h.levels}
    s.set_levels(h.lmin, h.lmax, ijk, mass)
    out = s.alloc_outputs()
    gm = s.solve_adjoint({l: torch.zeros(h.n(l), dtype=torch.float64, device="cuda") for l in h.levels}, w)
    s.sync()

    def loss(ms):
        s.set_levels(h.lmin, h.lmax, ijk, ms)
        s.solve(out=out)
        s.sync()
        return sum(float((w[l] * out[1][l]).sum()) for l in h.levels)

    n_all = sum(h.n(l) for l in h.levels)
    picks = np.unique((W.uniform(41, 1, np.arange(100)) * n_all).astype(np.int64))
    offs = np.cumsum([0] + [h.n(l) for l in h.levels])
    eps = 1e-6
    errs = []
    for g in picks:
        k = int(np.searchsorted(offs, g, side="right") - 1)
        j = int(g - offs[k])
        mp = [m.clone() for m in mass]
        mp[k][j] += eps
        lp = loss(mp)
        mp[k][j] -= 2 * eps
        lm = loss(mp)
        fd = (lp - lm) / (2 * eps)
        ad = float(gm[h.lmin + k][j])
        errs.append(abs(fd - ad) / max(abs(ad), 1e-30))
    assert len(picks) >= 95
    assert max(errs) <= 1e-5, max(errs)


def test_autograd_matches_adjoint_and_gradcheck():
    import torch
    from paper_2607_19489_b300 import fmm
    from paper_2607_19489_b300.autograd import potential
    h = nested(2, [(0, 3), (2, 4)], seed=9)
    s = fmm.Solver(4, "fp64")
    ijk = [torch.as_tensor(a, device="cuda").contiguous() for a in h.ijk]
    masses = [torch.as_tensor(m, device="cuda").clone().requires_grad_(True) for m in h.mass]
    w = {l: torch.as_tensor(W.normal(3, 400 + l, np.arange(3 * h.n(l))).reshape(-1, 3), device="cuda")
         for l in h.levels}
    phi, acc = potential(s, h.lmin, h.lmax, ijk, masses)
    loss = sum((w[l] * acc[l]).sum() + 0.5 * phi[l].sum() for l in h.levels)
    grads = torch.autograd.grad(loss, masses)
    gm = s.solve_adjoint({l: torch.full((h.n(l),), 0.5, dtype=torch.float64, device="cuda") for l in h.levels}, w)
    s.sync()
    for k, l in enumerate(h.levels):
        assert torch.allclose(grads[k], gm[l], rtol=1e-12, atol=0)

    def f(*ms):
        phi, acc = potential(s, h.lmin, h.lmax, ijk, list(ms))
        return tuple(acc[l] for l in h.levels) + tuple(phi[l] for l in h.levels)

    # the transposed near field sums onto each source with atomics, so repeated
    # backward passes differ in the last bits: nondet_tol allows rounding only
    assert torch.autograd.gradcheck(f, tuple(masses), eps=1e-6, atol=1e-8, rtol=1e-6, fast_mode=True,
                                    nondet_tol=1e-10)


def test_adjoint_needs_fp64_context():
    import torch
    from paper_2607_19489_b300 import fmm
    h = nested(2, [(0, 3), (2, 4)], seed=9)
    s = fmm.Solver(4, "mixed")
    s.set_hierarchy(h)
    g = {l: torch.zeros(h.n(l), dtype=torch.float64, device="cuda") for l in h.levels}
    ga = {l: torch.zeros(h.n(l), 3, dtype=torch.float64, device="cuda") for l in h.levels}
    with pytest.raises(fmm.FMMError) as e:
        s.solve_adjoint(g, ga)
    assert e.value.code == -1


def test_finite_differences_full_size_nested_two_plummer():
    """The 128^3-base nested two-Plummer hierarchy itself (13.6 M cells, three
    levels): central differences on 8 seeded cells (each costs two FP64 solves
    of the whole hierarchy; the 100-cell check runs on the 32^3-base version)."""
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.nested_two_plummer()
    s = fmm.Solver(6, "fp64")
    ijk = [torch.as_tensor(a, device="cuda").contiguous() for a in h.ijk]
    mass = [torch.as_tensor(m, device="cuda").contiguous() for m in h.mass]
    w = {l: torch.as_tensor(W.normal(31, 300 + l, np.arange(3 * h.n(l))).reshape(-1, 3), device="cuda")
         for l in h.levels}
    s.set_levels(h.lmin, h.lmax, ijk, mass)
    out = s.alloc_outputs()
    gm = s.solve_adjoint({l: torch.zeros(h.n(l), dtype=torch.float64, device="cuda") for l in h.levels}, w)
    s.sync()
    n_all = sum(h.n(l) for l in h.levels)
    offs = np.cumsum([0] + [h.n(l) for l in h.levels])
    picks = np.unique((W.uniform(43, 1, np.arange(8)) * n_all).astype(np.int64))
    eps = 1e-6
    for g in picks:
        k = int(np.searchsorted(offs, g, side="right") - 1)
        j = int(g - offs[k])
        vals = []
        for sgn in (1, -1):
            mp = [m.clone() for m in mass]
            mp[k][j] += sgn * eps
            s.set_levels(h.lmin, h.lmax, ijk, mp)
            s.solve(out=out)
            s.sync()
            vals.append(sum(float((w[l] * out[1][l]).sum()) for l in h.levels))
        fd = (vals[0] - vals[1]) / (2 * eps)
        ad = float(gm[h.lmin + k][j])
        assert abs(fd - ad) <= 1e-5 * abs(ad), (g, fd, ad)
