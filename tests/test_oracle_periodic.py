"""Pins of the oracle's periodic boundaries.

The periodic problem (images of the box everywhere, a uniform neutralising
background) has no plain O(N^2) sum, so the oracle carries Ewald's sum as its
ground truth and pins it first:
  * the rock-salt lattice (alternating +1/-1 masses on a 2^3 or 4^3 grid) gives
    the textbook Madelung constant at every site, with zero force;
  * Ewald's splitting parameter drops out (a wrong background constant or a
    lost reciprocal term would not), for a system with net mass;
  * the force is minus the gradient of the potential (central differences).
The lattice tensor of the root (the far images and the background) is pinned
by closed forms: the Laplacian of the background in its second moments
(T_200 = T_020 = T_002 = -4 pi / 3), harmonic traces at higher orders, zero odd
moments, cubic symmetry, independence of the splitting parameter.  The
periodic FMM then converges to the Ewald sum as p grows (unigrids and AMR,
also with the refined regions moved across the box edge, where the Ewald sum
itself is translation invariant and force-free in total), and the graded rule
wraps around the box.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W

MADELUNG_NACL = 1.747564594633182  # rock salt, in units of the nearest-neighbour distance


def rel_rms(a, b):
    num = sum(float(((a[l] - b[l]) ** 2).sum()) for l in b)
    den = sum(float((b[l] ** 2).sum()) for l in b)
    return float(np.sqrt(num / den))


def _grid(level, mass):
    n = 1 << level
    ijk = np.array([(i, j, k) for k in range(n) for j in range(n) for i in range(n)], np.int32)
    return W.Hierarchy(level, level, [ijk], [mass(ijk)])


@pytest.mark.parametrize("level", [1, 2])
def test_ewald_rock_salt_madelung(level):
    h = _grid(level, lambda ijk: np.where(ijk.sum(1) % 2 == 0, 1.0, -1.0))
    for alpha in (6.0, 9.0):
        phi, acc = oracle.ewald(h, alpha=alpha)
        q = h.mass[0]
        # phi = sum_j q_j g(r), g = -1/r: a site of charge q sees q M / d, d = 2^-level
        np.testing.assert_allclose(phi[level], q * MADELUNG_NACL * (1 << level), rtol=1e-11)
        assert np.abs(acc[level]).max() < 1e-11


def test_ewald_independent_of_the_splitting():
    h = W.unigrid_plummer(3, noise=0.3, seed=5)  # net mass 1: the background matters
    p1, a1 = oracle.ewald(h, alpha=6.0)
    p2, a2 = oracle.ewald(h, alpha=9.0)
    assert rel_rms(a1, a2) < 1e-12 and rel_rms(p1, p2) < 1e-12


def test_ewald_force_is_minus_the_gradient():
    level = 5
    n = 1 << level
    h = _grid(level, lambda ijk: np.where((ijk == [5, 9, 20]).all(1), 1.0,
                                          np.where((ijk == [25, 3, 11]).all(1), 0.5, 0.0)))
    ijk = h.ijk[0]
    sel = []
    for x in range(12, 20):
        for d in (-2, -1, 0, 1, 2):
            c = np.array([x + d, 16, 3])
            sel.append(int(np.nonzero((ijk == c).all(1))[0][0]))
    phi, acc = oracle.ewald(h, alpha=7.0, sel={level: np.array(sel, np.int64)})
    ph = phi[level].reshape(-1, 5)
    ax = acc[level].reshape(-1, 5, 3)[:, 2, 0]
    # fourth-order central difference of phi along x
    fd = -(-ph[:, 4] + 8 * ph[:, 3] - 8 * ph[:, 1] + ph[:, 0]) * n / 12.0
    np.testing.assert_allclose(ax, fd, rtol=1e-3, atol=1e-3 * np.abs(ax).max())


def _T(q, alpha=2.0):
    T = oracle.lattice_tensor(q, alpha)
    mi = oracle.multi_index(q)
    return T, {tuple(int(v) for v in m): k for k, m in enumerate(mi)}


def test_lattice_tensor_closed_forms():
    q = 8
    T, I = _T(q)
    for g, k in I.items():
        if sum(g) % 2:
            assert abs(T[k]) < 1e-12, g
    for g in [(2, 0, 0), (0, 2, 0), (0, 0, 2)]:
        assert abs(T[I[g]] + 4 * np.pi / 3) < 1e-12
    for g, k in I.items():  # harmonic beyond the background's quadratic
        if 1 <= sum(g) <= q - 2:
            tr = sum(T[I[tuple(g[j] + 2 * (j == i) for j in range(3))]] for i in range(3))
            assert abs(tr) < 1e-9 * max(1.0, np.abs(T).max()), g
    for g, k in I.items():  # cubic symmetry
        for perm in itertools.permutations(range(3)):
            assert abs(T[I[tuple(g[perm[j]] for j in range(3))]] - T[k]) < 1e-10 * max(1.0, abs(T[k]))


def test_lattice_tensor_independent_of_the_splitting():
    T1, _ = _T(8, 2.0)
    T2, _ = _T(8, 1.5)
    assert np.max(np.abs(T1 - T2) / np.maximum(np.abs(T1), 1.0)) < 1e-10


def test_periodic_fmm_converges_to_ewald_on_8cubed():
    h = W.unigrid_plummer(3, noise=0.3, seed=5)
    ep, ea = oracle.ewald(h, alpha=8.0)
    errs = [rel_rms(oracle.solve_periodic(h, p)[1], ea) for p in (2, 4, 6, 8, 10)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 3e-4, errs


def test_periodic_fmm_converges_to_ewald_on_16cubed_and_amr():
    for h, lo_bar in ((W.unigrid_plummer(4, noise=0.3, seed=5), 2e-3), (W.random_amr(3, 5, seed=13), 4e-3)):
        sel = {l: np.arange(0, h.n(l), max(1, h.n(l) // 300)) for l in h.levels}
        ep, ea = oracle.ewald(h, alpha=8.0, sel=sel)
        errs = [rel_rms(oracle.solve_periodic(h, p, sel=sel)[1], ea) for p in (2, 4, 6, 8)]
        assert all(b < a for a, b in zip(errs, errs[1:])), errs
        assert errs[-1] < lo_bar, errs


def test_periodic_graded_rule_wraps():
    # refined corner blocks touching the box edge at levels 3 and 4: the level-4
    # block's fathers have level-3 neighbours across the edge, not refined
    refined = W.nested_boxes(3, [(0, 4), (0, 4)])
    leaves = W.leaves_from_refined(3, 5, refined)
    h = W.Hierarchy(3, 5, [np.ascontiguousarray(c, dtype=np.int32) for c in leaves],
                    [np.ones(c.shape[0]) for c in leaves])
    oracle.solve(h, 2)  # graded inside the box
    with pytest.raises(oracle.OracleError) as e:
        oracle.solve_periodic(h, 2)  # not across it: the far side's cells are not refined
    assert e.value.code == -2
    with pytest.raises(oracle.OracleError):
        oracle.solve_periodic(W.unigrid_plummer(2), 4)  # lmin >= 3


def _shifted(h, shift):
    """The same masses moved by `shift` cells of each level (periodic wrap), and
    for each level the index map old -> new."""
    g = h.copy()
    maps = {}
    for k, l in enumerate(h.levels):
        n = 1 << l
        s = np.asarray(shift, np.int64) * (1 << (l - h.lmin))
        new = (h.ijk[k].astype(np.int64) + s) % n
        g.ijk[k] = np.ascontiguousarray(new.astype(np.int32))
        maps[l] = np.arange(h.n(l))
    return g, maps


def test_ewald_is_translation_invariant_and_force_free():
    h = W.unigrid_plummer(3, noise=0.3, seed=7)
    p0, a0 = oracle.ewald(h, alpha=7.0)
    g, _ = _shifted(h, (3, 5, 1))  # any whole-cell shift of the torus
    p1, a1 = oracle.ewald(g, alpha=7.0)
    assert rel_rms(p1, p0) < 1e-12 and rel_rms(a1, a0) < 1e-12
    m = h.mass[0]
    tot = (m[:, None] * a0[3]).sum(0)  # Newton's third law; the background pulls every cell alike
    assert np.abs(tot).max() < 1e-12 * (np.abs(m[:, None] * a0[3]).sum(0)).max()


def test_periodic_fmm_across_the_box_edge():
    """Moving every mass by half the box carries the refined regions across the
    box edge (the lists and the graded rule then wrap through them).  The Ewald
    sum moves with the masses exactly; the FMM's root expansion does not (the
    root box does not map onto itself), so the shifted FMM is checked against
    the shifted Ewald sum: of the same size as before the shift (masses near
    the root's corners converge more slowly in its expansion) and falling
    with p."""
    h = W.random_amr(3, 5, seed=13)
    sel = {l: np.arange(0, h.n(l), max(1, h.n(l) // 300)) for l in h.levels}
    ep, ea = oracle.ewald(h, alpha=8.0, sel=sel)
    e0 = rel_rms(oracle.solve_periodic(h, 6, sel=sel)[1], ea)
    for shift in ((4, 0, 0), (0, 4, 4), (4, 4, 4)):
        g, _ = _shifted(h, shift)
        gp, ga = oracle.ewald(g, alpha=8.0, sel=sel)
        assert rel_rms(ga, ea) < 1e-12 and rel_rms(gp, ep) < 1e-12, shift
        errs = [rel_rms(oracle.solve_periodic(g, p, sel=sel)[1], ga) for p in (4, 6, 8)]
        assert errs[1] < 3 * e0, (shift, e0, errs)
        assert errs[2] < errs[1] < errs[0], (shift, errs)
