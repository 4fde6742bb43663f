"""The library's translation tables (host code, box units) against the
oracle's operators in physical coordinates (independent code paths).

Box units: a box of size h stores Mt_alpha = M_alpha / h^|alpha| and
Lt_beta = L_beta h^(|beta|+1).  The geometry of each table is set up here
with the source box of size 1 (so box units and physical units coincide for
the source) and compared operator by operator."""
import math

import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import fmm

NBR26 = [q for q in range(27) if q != 13]


def bits(c):
    return np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], dtype=np.float64)


def dq_of(q27):
    return np.array([q27 % 3 - 1, (q27 // 3) % 3 - 1, q27 // 9 - 1], dtype=np.float64)


def degrees(p):
    return oracle.multi_index(p).sum(1)


@pytest.fixture(scope="module", params=[3, 6])
def p(request):
    return request.param


def test_m2p_table(p):
    nc = oracle.ncoef(p)
    T = fmm.host_table(p, "m2p")
    rng = np.random.default_rng(p)
    checked = 0
    for f in (0, 5, 7):
        for t in (0, 3, 6):
            for qi in (0, 7, 12, 13, 25):
                for s in (0, 2, 7):
                    q27 = NBR26[qi]
                    cF = bits(f) + 0.5
                    cS = 2 * dq_of(q27) + bits(s) + 0.5
                    x = cF + (bits(t) - 0.5) / 2
                    cols = slice((qi * 8 + s) * nc, (qi * 8 + s + 1) * nc)
                    block = T[(f * 8 + t) * 4:(f * 8 + t) * 4 + 4, cols]
                    if np.abs(bits(f) - 2 * dq_of(q27) - bits(s)).max() <= 1:
                        assert np.all(block == 0)
                        continue
                    M = rng.normal(size=nc)
                    ref = oracle.m2p(p, M, cS, x)
                    got = block @ M
                    np.testing.assert_allclose(got[0], ref[0], rtol=1e-12, atol=1e-13)
                    np.testing.assert_allclose(got[1:], -ref[1:], rtol=1e-11, atol=1e-13)
                    checked += 1
    assert checked > 20


def test_m2l_table(p):
    nc = oracle.ncoef(p)
    T = fmm.host_table(p, "m2l")
    rng = np.random.default_rng(10 + p)
    for b in (0, 3, 7):
        for qi in (0, 4, 13, 20, 25):
            for s in (1, 6):
                q27 = NBR26[qi]
                cB = bits(b) + 0.5
                cS = 2 * dq_of(q27) + bits(s) + 0.5
                block = T[b * nc:(b + 1) * nc, (qi * 8 + s) * nc:(qi * 8 + s + 1) * nc]
                if np.abs(cB - cS).max() <= 1:
                    assert np.all(block == 0)
                    continue
                M = rng.normal(size=nc)
                np.testing.assert_allclose(block @ M, oracle.m2l(p, M, cS, cB), rtol=1e-11, atol=1e-13)


def test_near_table(p):
    nc = oracle.ncoef(p)
    T = fmm.host_table(p, "near")
    rng = np.random.default_rng(20 + p)
    for R in ([2, 0, 0], [-3, 1, -2], [0, -2, 3], [3, 3, 3], [-2, -2, -1]):
        idx = ((R[2] + 3) * 7 + (R[1] + 3)) * 7 + (R[0] + 3)
        M = rng.normal(size=nc)
        ref = oracle.m2p(p, M, [0.0, 0.0, 0.0], np.array(R, dtype=np.float64))
        got = T[idx].T @ M
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(got[1:], -ref[1:], rtol=1e-11, atol=1e-14)


def test_l2p_table(p):
    nc = oracle.ncoef(p)
    T = fmm.host_table(p, "l2p")
    rng = np.random.default_rng(30 + p)
    for f in range(8):
        for t in (0, 5):
            L = rng.normal(size=nc)
            x = (bits(f) - 0.5) / 2 + (bits(t) - 0.5) / 4
            ref = oracle.l2p(p, L, [0.0, 0.0, 0.0], x)
            got = T[f * 8 + t].T @ L
            np.testing.assert_allclose(got[0], ref[0], rtol=1e-12, atol=1e-14)
            np.testing.assert_allclose(got[1:], -ref[1:], rtol=1e-12, atol=1e-14)


def test_m2m_table(p):
    # child box size 1/2 at (+-1/4) of a unit parent box centred at 0
    nc = oracle.ncoef(p)
    T = fmm.host_table(p, "m2m")
    d = degrees(p)
    rng = np.random.default_rng(40 + p)
    for c in range(8):
        Mc_box = rng.normal(size=nc)
        Mc_phys = Mc_box * 0.5 ** d
        cc = (bits(c) - 0.5) / 2
        ref = oracle.m2m(p, Mc_phys, cc, [0.0, 0.0, 0.0])
        np.testing.assert_allclose(T[c] @ Mc_box, ref, rtol=1e-12, atol=1e-14)


def test_l2l_table(p):
    nc = oracle.ncoef(p)
    T = fmm.host_table(p, "l2l")
    d = degrees(p)
    rng = np.random.default_rng(50 + p)
    for c in range(8):
        Lp = rng.normal(size=nc)  # unit parent box: box units == physical
        cc = (bits(c) - 0.5) / 2
        ref = oracle.l2l(p, Lp, [0.0, 0.0, 0.0], cc) * 0.5 ** (d + 1)
        np.testing.assert_allclose(T[c] @ Lp, ref, rtol=1e-12, atol=1e-14)


def test_m2p_delta_l2_table(p):
    """Delta l = 2: M2P from a level l-2 source box (size 1 here) to the 512
    level-l cells under a row oct, returned in level l-1 units (phi / 2, accel / 4)."""
    nc = oracle.ncoef(p)
    T = fmm.host_table(p, "m2p_dl2")
    rng = np.random.default_rng(30 + p)
    checked = 0
    for g in (0, 6):
        for f in (1, 7):
            for t in (0, 5):
                for qi in (0, 9, 13, 25):
                    for s in (0, 7):
                        q27 = NBR26[qi]
                        cS = 2 * dq_of(q27) + bits(s) + 0.5
                        x = bits(g) + (2 * bits(f) + bits(t) + 0.5) / 4
                        n0 = ((g * 8 + f) * 8 + t) * 4
                        block = T[n0:n0 + 4, (qi * 8 + s) * nc:(qi * 8 + s + 1) * nc]
                        if np.abs(bits(g) - 2 * dq_of(q27) - bits(s)).max() <= 1:
                            assert np.all(block == 0)
                            continue
                        M = rng.normal(size=nc)
                        ref = oracle.m2p(p, M, cS, x)
                        got = block @ M
                        np.testing.assert_allclose(got[0], 0.5 * ref[0], rtol=1e-12, atol=1e-13)
                        np.testing.assert_allclose(got[1:], -0.25 * ref[1:], rtol=1e-11, atol=1e-13)
                        checked += 1
    assert checked > 20


def test_p2p_ring_delta_l2_table():
    """Delta l = 2: the near-field ring as point-mass sources (the 8 children of
    each level l-1 source cell), level l-1 units, zero where the source cell
    touches the target's parent F (Delta l = 1's near field)."""
    T = fmm.host_table(4, "p2p_ring_dl2")
    checked = 0
    for f in (0, 5):
        for t in (1, 6):
            for qi in (0, 9, 13, 25):
                for s in (0, 3, 7):
                    q27 = NBR26[qi]
                    n0 = (f * 8 + t) * 4
                    block = T[n0:n0 + 4, (qi * 8 + s) * 8:(qi * 8 + s + 1) * 8]
                    if np.abs(bits(f) - 2 * dq_of(q27) - bits(s)).max() <= 1:
                        assert np.all(block == 0)
                        continue
                    x = bits(f) + (bits(t) + 0.5) / 2  # target centre, level l-1 cells
                    m = np.random.default_rng(checked).uniform(0.5, 1.5, 8)
                    phi, acc = 0.0, np.zeros(3)
                    for kc in range(8):
                        y = 2 * dq_of(q27) + bits(s) + (bits(kc) + 0.5) / 2
                        r = x - y
                        d = np.sqrt(r @ r)
                        phi -= m[kc] / d
                        acc -= m[kc] * r / d ** 3
                    got = block @ m
                    np.testing.assert_allclose(got[0], phi, rtol=1e-13)
                    np.testing.assert_allclose(got[1:], acc, rtol=1e-12, atol=1e-14)
                    checked += 1
    assert checked > 10


def test_lattice_tables(p):
    """Periodic boundaries: the library's lattice tensor (Taylor-mode Ewald) against
    the oracle's (radial recursion), and the level-1 operator against the oracle's
    M2M, Eq. 3 with that tensor and L2L, plus the oracle's M2L from the 26 images of
    the level-1 oct around it, in level-1 box units."""
    T_lib = fmm.host_table(p, "lattice_tensor")
    T = oracle.lattice_tensor(p)
    assert np.max(np.abs(T_lib - T) / np.maximum(np.abs(T), 1.0)) < 1e-9
    nc = oracle.ncoef(p)
    mi = oracle.multi_index(p)
    idx = {tuple(int(v) for v in m): k for k, m in enumerate(mi)}
    deg = mi.sum(1)
    fact = np.array([np.prod([math.factorial(int(v)) for v in m]) for m in mi], dtype=np.float64)
    A = fmm.host_table(p, "lattice")
    h1, c0 = 0.5, np.full(3, 0.5)
    rng = np.random.default_rng(p)
    for cs in (0, 5):
        Mt = rng.normal(size=nc)
        M0 = oracle.m2m(p, Mt * h1 ** deg, (bits(cs) + 0.5) * h1, c0)
        L0 = np.zeros(nc)
        for b, B in enumerate(mi):
            for a, Al in enumerate(mi):
                if deg[a] + deg[b] <= p:
                    L0[b] += (-1.0) ** deg[a] / fact[a] * T[idx[tuple(int(v) for v in Al + B)]] * M0[a]
        for ct in (0, 3, 7):
            cT = (bits(ct) + 0.5) * h1
            Lp = oracle.l2l(p, L0, c0, cT)
            for q27 in NBR26:
                cS = (2 * dq_of(q27) + bits(cs) + 0.5) * h1
                if np.abs(bits(ct) - 2 * dq_of(q27) - bits(cs)).max() > 1:
                    Lp = Lp + oracle.m2l(p, Mt * h1 ** deg, cS, cT)
            ref = Lp * h1 ** (deg + 1)
            got = A[ct * nc:(ct + 1) * nc, cs * nc:(cs + 1) * nc] @ Mt
            np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("order", [1, 2, 3])
def test_variant_tables_at_low_orders(order):
    """The periodic and Delta l = 2 tables at the lowest orders (series of degree
    1 have no |x|^2 term): finite, and the lattice tensor equal to the oracle's."""
    for w in ("lattice", "m2p_dl2", "p2p_ring_dl2"):
        assert np.isfinite(fmm.host_table(order, w)).all(), w
    T = oracle.lattice_tensor(order)
    assert np.max(np.abs(fmm.host_table(order, "lattice_tensor") - T) / np.maximum(np.abs(T), 1.0)) < 1e-12
