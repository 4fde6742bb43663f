"""Host-side checks of the C ABI: the library loads, exports every declared
symbol, validates arguments before touching the GPU, and builds its
translation tables from the same integer numerators as the oracle (reached
by a different recurrence)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2607_19489_b300 import fmm
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = fmm.lib()
    names = declared_symbols()
    assert "fmm_solve" in names and "fmm_set_levels" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(fmm.EXPORTED)


def test_create_rejects_bad_arguments_without_gpu():
    L = fmm.lib()
    h = ctypes.c_void_p()
    none = fmm.ALLOC_FN()
    # (p, precision, bottom mode, p_m, mass_fp32, fp64_top)
    for p, prec, bottom, pm, m32, t64 in [(0, 0, 0, 0, 0, 0), (9, 0, 0, 0, 0, 0), (4, 7, 0, 0, 0, 0),
                                          (4, 0, 2, 0, 0, 0), (4, 0, 0, 5, 0, 0), (4, 0, 0, -1, 0, 0),
                                          (4, 1, 0, 0, 2, 0), (4, 1, 0, 0, 0, 3)]:
        cfg = fmm._Config(p, prec, 1.0, 0, 0, bottom, pm, m32, t64)
        assert L.fmm_create(ctypes.byref(cfg), none, None, ctypes.byref(h)) == -1, (p, prec, bottom, pm, m32, t64)
    # (delta_l, periodic, bottom mode): out of range, or a combination the variants exclude
    for dl, per, bottom in [(3, 0, 0), (-1, 0, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (2, 1, 0)]:
        cfg = fmm._Config(4, 1, 1.0, 0, 0, bottom, 0, 0, 0, dl, per)
        assert L.fmm_create(ctypes.byref(cfg), none, None, ctypes.byref(h)) == -1, (dl, per, bottom)
    assert L.fmm_create(None, none, None, ctypes.byref(h)) == -1
    assert L.fmm_set_wait_limit(None, 1.0) == -1
    assert L.fmm_set_levels(None, 2, 3, 2, None, None, None, None) == -1
    assert L.fmm_solve(None, 2, None, None, None) == -1
    assert L.fmm_last_error(None) == b"null context"


@pytest.mark.parametrize("u", [[1, 2, 3], [3, -1, 2], [13, -9, 5], [0, 0, 7], [-4, 4, 1]])
def test_host_numerators_match_oracle(u):
    q = 9
    lib_n = fmm.host_numerators(q, u)
    orc_n = oracle.numerators(q, u)
    # both sides use the graded order (degree, a desc, b desc)
    assert np.array_equal(oracle.multi_index(q)[:, 0] + oracle.multi_index(q)[:, 1] + oracle.multi_index(q)[:, 2],
                          np.repeat(np.arange(q + 1), [(n + 1) * (n + 2) // 2 for n in range(q + 1)]))
    assert np.array_equal(lib_n, orc_n)


def test_host_numerators_golden():
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "inv_r_numerators.txt"))
            if l.strip() and not l.startswith("#")]
    mi = oracle.multi_index(4)
    idx = {tuple(int(v) for v in m): k for k, m in enumerate(mi)}
    for r in rows:
        g = tuple(int(v) for v in r[0:3])
        u = [int(v) for v in r[3:6]]
        assert fmm.host_numerators(4, u)[idx[g]] == int(r[6])
