"""The library's translation tables (host code, box units) against the
oracle's operators in physical coordinates (independent code paths).

Box units: a box of size h stores Mt_alpha = M_alpha / h^|alpha| and
Lt_beta = L_beta h^(|beta|+1).  The geometry of each table is set up here
with the source box of size 1 (so box units and physical units coincide for
the source) and compared operator by operator."""
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
