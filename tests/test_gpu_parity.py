"""CUDA path against the CPU oracle, through the C ABI.

Bars (from the method's accuracy targets): FP64 path relative RMS error
<= 1e-10 in phi and accel; mixed path (split-BF16 tensor-core M2L/M2P, FP32
P2P) <= 1e-4; beside each, a per-cell bound (1e-9 FP64, 1e-3 mixed, relative
to max(|ref|, 1 % of the RMS reference magnitude)) so that a localised fault
cannot hide in the RMS; tree index bit-exact.  Cases span several GEMM tiles
with ragged tails, coarse-fine interfaces, an empty base level, the smallest
hierarchy (4^3, no far field) and the two-level 64^3 + 32^3 workload on
sampled targets."""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W
from _parity import ORACLE_FP64, ORACLE_MIXED, check, oracle_tol

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def run(h, p, precision, lo=None, out_fp32=False, sel=None, **kw):
    from paper_2607_19489_b300 import fmm
    torch = _torch()
    s = fmm.Solver(p, precision, out_fp32=out_fp32, **kw)
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


def small_cases():
    return {
        "unigrid16": W.unigrid_plummer(4),
        "amr_3_5": W.random_amr(3, 5, seed=13),
        "amr_3_5b": W.random_amr(3, 5, seed=19),
        "twolevel16": W.two_level_plummer(base=4, lo=4, hi=12, seed=3),
        "empty_base": _empty_base(),
        "tiny4": W.unigrid_plummer(2),
    }


def _empty_base():
    refined = W.nested_boxes(3, [(0, 8), (4, 12)])
    leaves = W.leaves_from_refined(3, 5, refined)
    h = W.Hierarchy(3, 5, name="empty base level")
    for k, c in enumerate(leaves):
        h.ijk.append(np.ascontiguousarray(c, dtype=np.int32))
        h.mass.append(W.uniform(9, 50 + k, np.arange(c.shape[0])) + 0.1)
    return h


CASES = small_cases()


@pytest.mark.parametrize("name", list(CASES))
def test_tree_bit_exact(name):
    from paper_2607_19489_b300 import fmm
    h = CASES[name]
    ref = oracle.tree(h)
    s = fmm.Solver(4, "fp64")
    s.set_hierarchy(h)
    for l in range(1, h.lmax + 1):
        k, st, nb = s.tree_export(l)
        rk, rst, rnb = ref[l]
        assert np.array_equal(k, rk), (name, l)
        assert np.array_equal(st, rst), (name, l)
        assert np.array_equal(nb, rnb), (name, l)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("p", [4, 6])
def test_fp64_matches_oracle(name, p):
    h = CASES[name]
    rp, ra = oracle.solve(h, p)
    gp, ga = run(h, p, "fp64")
    check(gp, ga, rp, ra, ORACLE_FP64, f"{name} p={p} fp64", h=h)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("p", [4, 6])
def test_mixed_matches_oracle(name, p):
    h = CASES[name]
    rp, ra = oracle.solve(h, p)
    gp, ga = run(h, p, "mixed")
    check(gp, ga, rp, ra, ORACLE_MIXED, f"{name} p={p} mixed", h=h)


@pytest.mark.parametrize("name", ["amr_3_5", "twolevel16"])
@pytest.mark.parametrize("p", [2, 3, 5, 8])
def test_mixed_other_orders_match_oracle(name, p):
    """The tensor-core contraction picks its row-load width and its K order from
    the offset segment 8 ncoef(p): p = 2 (80), 3 (160), 5 (448) and 8 (1320)
    reach the combinations that p = 4 (280) and 6 (672) do not."""
    h = CASES[name]
    rp, ra = oracle.solve(h, p)
    gp, ga = run(h, p, "mixed")
    check(gp, ga, rp, ra, ORACLE_MIXED, f"{name} p={p} mixed", h=h)


def test_unigrid32_p4_fp64_full():
    # 32^3 Plummer, p = 4, FP64 path on every cell
    h = W.unigrid_plummer(5)
    rp, ra = oracle.solve(h, 4)
    gp, ga = run(h, 4, "fp64")
    check(gp, ga, rp, ra, ORACLE_FP64, "unigrid32 p=4 fp64", h=h)


def test_unigrid32_p4_fp64_against_direct_sum():
    """The 32^3 Plummer unigrid at p = 4 (FP64) against the O(N^2) direct sum over
    all 32 768 cells.  This is the method's own truncation error (the oracle
    gives the same numbers): relative RMS 7.22e-3 in accel (worst cell 3.98e-2)
    and 5.83e-4 in phi (worst cell 3.27e-3); bounded here 25 % above those."""
    h = W.unigrid_plummer(5)
    dp, da = oracle.direct(h)
    gp, ga = run(h, 4, "fp64")
    check(gp, ga, dp, da, {"rms": 9.0e-3, "cell": 5.0e-2}, "unigrid32 p=4 fp64 vs direct", h=h, outputs=("accel",))
    check(gp, ga, dp, da, {"rms": 7.3e-4, "cell": 4.1e-3}, "unigrid32 p=4 fp64 vs direct", h=h, outputs=("phi",))


def _sample(h, n_per_level, seed):
    sel = {}
    for k, l in enumerate(h.levels):
        n = h.n(l)
        u = W.uniform(seed, 900 + l, np.arange(min(n, n_per_level)))
        idx = np.unique((u * n).astype(np.int64))
        # also every cell next to a coarse-fine interface of this level
        sel[l] = idx
    return sel


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_twolevel64_p6_sampled(precision):
    # 64^3 base + 32^3 refined block, p = 6 (the measured workload), sampled targets
    h = W.two_level_plummer()
    sel = _sample(h, 1500, 77)
    # add the cells on both sides of the coarse-fine interface
    c = h.ijk[0]
    ring = np.where((np.abs(c - 31.5).max(1) >= 8) & (np.abs(c - 31.5).max(1) <= 10))[0]
    sel[6] = np.unique(np.concatenate([sel[6], ring[::7]]))
    f = h.ijk[1]
    edge = np.where(np.abs(f - 63.5).max(1) >= 15)[0]
    sel[7] = np.unique(np.concatenate([sel[7], edge[::13]]))
    rp, ra = oracle.solve(h, 6, sel=sel)
    gp, ga = run(h, 6, precision, sel=sel)
    check(gp, ga, rp, ra, oracle_tol(precision), f"64^3+32^3 p=6 {precision}", h=h, sel=sel)


@pytest.mark.parametrize("name", ["unigrid16", "amr_3_5", "amr_3_5b", "twolevel16", "empty_base", "tiny4"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bottom_mode_m2l_matches_oracle(name, precision):
    """Bottom mode 1 (M2L into the parent box + L2P): the downward pass runs to
    level lmax-1 and no M2P is launched."""
    h = CASES[name]
    for p in (4, 6):
        rp, ra = oracle.solve(h, p, bottom="m2l")
        gp, ga = run(h, p, precision, bottom="m2l")
        check(gp, ga, rp, ra, oracle_tol(precision), f"{name} p={p} {precision} bottom m2l", h=h)


@pytest.mark.parametrize("p,pm", [(3, 2), (6, 4), (8, 5)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multipole_order_matches_oracle(p, pm, precision):
    """(p_m, p) = (2, 3) is the paper's quadrupole configuration."""
    for name in ("amr_3_5", "twolevel16"):
        h = CASES[name]
        rp, ra = oracle.solve(h, p, p_m=pm)
        gp, ga = run(h, p, precision, p_m=pm)
        check(gp, ga, rp, ra, oracle_tol(precision), f"{name} p={p} p_m={pm} {precision}", h=h)
    h = CASES["amr_3_5"]
    rp, ra = oracle.solve(h, p, p_m=pm, bottom="m2l")
    gp, ga = run(h, p, precision, p_m=pm, bottom="m2l")
    check(gp, ga, rp, ra, oracle_tol(precision), f"amr p={p} p_m={pm} {precision} bottom m2l", h=h)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_twolevel64_p6_bottom_m2l_sampled(precision):
    h = W.two_level_plummer()
    sel = _sample(h, 800, 78)
    c = h.ijk[0]
    ring = np.where((np.abs(c - 31.5).max(1) >= 8) & (np.abs(c - 31.5).max(1) <= 10))[0]
    sel[6] = np.unique(np.concatenate([sel[6], ring[::11]]))
    rp, ra = oracle.solve(h, 6, sel=sel, bottom="m2l")
    gp, ga = run(h, 6, precision, sel=sel, bottom="m2l")
    check(gp, ga, rp, ra, oracle_tol(precision), f"64^3+32^3 p=6 {precision} bottom m2l", h=h, sel=sel)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bottom_mode_m2l_subcycles_match_oracle(precision):
    """Partial rebuilds and fine-level-only solves in bottom mode 1 (the downward
    pass then keeps the ancestor lists up to level lo-2)."""
    from paper_2607_19489_b300 import fmm
    torch = _torch()
    h = CASES["amr_3_5"]
    s = fmm.Solver(6, precision, bottom="m2l")
    s.set_hierarchy(h)
    s.solve()
    for lo in (4, 5):
        h2 = h.copy()
        for k in range(lo - h.lmin, len(h.mass)):
            h2.mass[k] = h.mass[k] * (1.0 + 1e-3 * (2 * W.uniform(4, 70 + k + lo, np.arange(h.mass[k].size)) - 1))
        s.set_hierarchy(h2, lo=lo)
        phi, acc = s.solve(lo)
        torch.cuda.synchronize()
        s.sync()
        rp, ra = oracle.solve(h2, 6, lo=lo, bottom="m2l")
        check({l: phi[l].cpu().numpy() for l in phi}, {l: acc[l].cpu().numpy() for l in acc}, rp, ra,
              oracle_tol(precision), f"bottom m2l subcycle lo={lo} {precision}", h=h2)
        h = h2


@pytest.mark.parametrize("name", ["unigrid16", "amr_3_5", "twolevel16", "empty_base"])
@pytest.mark.parametrize("p", [2, 4, 5, 6, 8])
def test_tf32_matches_oracle(name, p):
    """M2L and M2P in one TF32 product per term (tcgen05 kind::tf32), both row
    orders of the contraction (K order at p = 2, 4, 5, 8; slice-major at 6)."""
    h = CASES[name]
    rp, ra = oracle.solve(h, p)
    gp, ga = run(h, p, "tf32")
    check(gp, ga, rp, ra, oracle_tol("tf32"), f"{name} p={p} tf32", h=h)


@pytest.mark.parametrize("precision", ["mixed", "tf32"])
@pytest.mark.parametrize("name,p", [("amr_3_5", 4), ("amr_3_5b", 6), ("twolevel16", 8), ("unigrid16", 6)])
def test_fp64_top_matches_oracle(name, p, precision):
    """config.fp64_top: FP64 M2M at box levels <= 3 and an FP64 L2L chain with
    FP64 local-expansion accumulation, against the oracle; and against the
    default FP32 version of the same context, which differs only by rounding."""
    h = CASES[name]
    rp, ra = oracle.solve(h, p)
    gp, ga = run(h, p, precision, fp64_top=True)
    check(gp, ga, rp, ra, oracle_tol(precision), f"{name} p={p} {precision} fp64_top", h=h)
    fp, fa = run(h, p, precision)
    check(gp, ga, fp, fa, {"rms": 1e-4, "cell": 1e-3}, f"{name} p={p} {precision} fp64_top vs FP32", h=h)


@pytest.mark.parametrize("bottom", ["m2p", "m2l"])
def test_twolevel64_p6_tf32_sampled(bottom):
    h = W.two_level_plummer()
    sel = _sample(h, 800, 79)
    rp, ra = oracle.solve(h, 6, sel=sel, bottom=bottom)
    gp, ga = run(h, 6, "tf32", sel=sel, bottom=bottom)
    check(gp, ga, rp, ra, oracle_tol("tf32"), f"64^3+32^3 p=6 tf32 bottom {bottom}", h=h, sel=sel)


def test_caller_order_is_kept():
    # outputs follow the caller's order: the same cells given in another order get the
    # same values (to the rounding of the order of the FP64 atomic additions; a cell
    # given another cell's output would be off by O(1))
    h = CASES["amr_3_5"]
    hp = W.permute(h, seed=5)
    gp, ga = run(h, 6, "fp64")
    pp, pa = run(hp, 6, "fp64")
    key = lambda a: a[:, 0] * 1_000_000 + a[:, 1] * 1000 + a[:, 2]
    same = {"rms": 1e-14, "cell": 1e-13}
    for k, l in enumerate(h.levels):
        order = np.argsort(key(h.ijk[k]))
        porder = np.argsort(key(hp.ijk[k]))
        check({l: pp[l][porder]}, {l: pa[l][porder]}, {l: gp[l][order]}, {l: ga[l][order]}, same,
              f"permuted input, level {l}")


def test_host_pointers_and_fp32_outputs():
    from paper_2607_19489_b300 import fmm
    h = CASES["twolevel16"]
    gp, ga = run(h, 4, "mixed")
    s = fmm.Solver(4, "mixed", out_fp32=True)
    s.set_levels(h.lmin, h.lmax, [np.ascontiguousarray(a) for a in h.ijk], [np.ascontiguousarray(m) for m in h.mass])
    phi = {l: np.zeros(h.n(l), np.float32) for l in h.levels}
    acc = {l: np.zeros((h.n(l), 3), np.float32) for l in h.levels}
    s.solve(out=(phi, acc))
    s.sync()
    for l in h.levels:
        np.testing.assert_allclose(acc[l], ga[l], rtol=2e-5, atol=2e-6 * np.abs(ga[l]).max())
        np.testing.assert_allclose(phi[l], gp[l], rtol=2e-6)


def test_subcycle_levels_match_oracle():
    # fmm_set_levels(lo) replaces the finer levels; fmm_solve(lo) returns levels lo..lmax
    from paper_2607_19489_b300 import fmm
    torch = _torch()
    h = CASES["amr_3_5"]
    s = fmm.Solver(6, "fp64")
    s.set_hierarchy(h)
    h2 = h.copy()
    for k in (1, 2):
        h2.mass[k] = h.mass[k] * (1.0 + 1e-3 * (2 * W.uniform(4, 60 + k, np.arange(h.mass[k].size)) - 1))
    s.set_hierarchy(h2, lo=4)
    phi, acc = s.solve(4)
    torch.cuda.synchronize()
    s.sync()
    rp, ra = oracle.solve(h2, 6, lo=4)
    assert set(phi) == {4, 5}
    check({l: phi[l].cpu().numpy() for l in (4, 5)}, {l: acc[l].cpu().numpy() for l in (4, 5)}, rp, ra,
          ORACLE_FP64, "subcycle lo=4 fp64", h=h2)


def test_invalid_hierarchies_rejected():
    from paper_2607_19489_b300 import fmm
    h = W.two_level_plummer(base=3, lo=2, hi=6)
    cases = {}
    bad = h.copy()
    bad.ijk[0] = np.concatenate([bad.ijk[0], bad.ijk[0][:1]])
    bad.mass[0] = np.concatenate([bad.mass[0], bad.mass[0][:1]])
    cases["FMM_ERR_DUPLICATE"] = bad
    bad = h.copy()
    bad.ijk[0] = bad.ijk[0].copy()
    bad.ijk[0][3] = [8, 0, 0]
    cases["FMM_ERR_OUT_OF_BOX"] = bad
    bad = h.copy()
    bad.ijk[1] = bad.ijk[1][1:].copy()
    bad.mass[1] = bad.mass[1][1:].copy()
    cases["FMM_ERR_INCOMPLETE"] = bad
    bad = h.copy()
    bad.mass[1] = bad.mass[1].copy()
    bad.mass[1][5] = np.nan
    cases["FMM_ERR_NONFINITE"] = bad
    bad = h.copy()
    keep = ~(bad.ijk[1] == [4, 4, 4]).all(1)
    bad.ijk[1] = bad.ijk[1][keep]
    bad.mass[1] = bad.mass[1][keep]
    bad.lmax = 5
    bad.ijk.append(np.array([[8 + (k & 1), 8 + ((k >> 1) & 1), 8 + ((k >> 2) & 1)] for k in range(8)], np.int32))
    bad.mass.append(np.ones(8) * 1e-3)
    cases["FMM_ERR_NOT_GRADED"] = bad
    for want, hh in cases.items():
        s = fmm.Solver(4, "mixed")
        with pytest.raises(fmm.FMMError) as ei:
            s.set_hierarchy(hh)
        assert ei.value.name == want
        with pytest.raises(fmm.FMMError) as ei:
            s.solve()
        assert ei.value.name == "FMM_ERR_STATE"
    s = fmm.Solver(4, "mixed")
    with pytest.raises(fmm.FMMError) as ei:
        s.set_hierarchy(h, lo=4)
    assert ei.value.name == "FMM_ERR_STATE"
