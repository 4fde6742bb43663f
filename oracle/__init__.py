"""Oracle for the adaptive FMM (TEST INFRASTRUCTURE ONLY).

Python access to the plain FP64 C++ implementation in fmm_oracle.cpp.  Only
the tests, the smoke check and the benchmark's CPU-baseline leg use this
package; the CUDA library never imports, links or calls it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboracle.so")
SRC_PATH = os.path.join(_HERE, "fmm_oracle.cpp")

ERRORS = {0: "ok", -1: "arg", -2: "not_graded", -3: "duplicate", -4: "out_of_box",
          -10: "incomplete"}


def build(force: bool = False) -> str:
    """Compile fmm_oracle.cpp into liboracle.so (g++, OpenMP)."""
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC_PATH)):
        return LIB_PATH
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", SRC_PATH,
           "-o", LIB_PATH + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(LIB_PATH + ".tmp", LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.oracle_fmm_solve.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, P, P,
                                       P, ctypes.c_int]
        L.oracle_fmm_solve_dl2.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                           P, P, P, P, ctypes.c_int]
        L.oracle_fmm_solve_periodic.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, P, P, ctypes.c_int]
        L.oracle_ewald_sum.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, P, P, P, P, ctypes.c_int]
        L.oracle_lattice_tensor.argtypes = [ctypes.c_int, ctypes.c_double, P]
        L.oracle_direct_sum.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_double,
                                        ctypes.c_int, P, P, P, P, ctypes.c_int]
        L.oracle_tree.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P]
        L.oracle_ncoef.argtypes = [ctypes.c_int]
        L.oracle_multi_index.argtypes = [ctypes.c_int, P]
        L.oracle_inv_r_derivs.argtypes = [ctypes.c_int, P, P]
        L.oracle_numerators.argtypes = [ctypes.c_int, P, P]
        L.oracle_p2m.argtypes = [ctypes.c_int, ctypes.c_double, P, P, P]
        L.oracle_m2m.argtypes = [ctypes.c_int, P, P, P, P]
        L.oracle_m2l.argtypes = [ctypes.c_int, P, P, P, P]
        L.oracle_l2l.argtypes = [ctypes.c_int, P, P, P, P]
        L.oracle_l2p.argtypes = [ctypes.c_int, P, P, P, P]
        L.oracle_m2p.argtypes = [ctypes.c_int, P, P, P, P]
        L.oracle_max_threads.restype = ctypes.c_int
        del i64
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ptr_array(arrs):
    t = (ctypes.c_void_p * len(arrs))()
    for i, a in enumerate(arrs):
        t[i] = a.ctypes.data if a.size else 0
    return t


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code} ({ERRORS.get(code, '?')})")
        self.code = code


def _inputs(h):
    ijk = [np.ascontiguousarray(a, dtype=np.int32) for a in h.ijk]
    mass = [np.ascontiguousarray(m, dtype=np.float64) for m in h.mass]
    n = np.array([a.shape[0] for a in ijk], dtype=np.int64)
    return n, ijk, mass


def _call(fn, h, lo, sel, extra_front, threads):
    n, ijk, mass = _inputs(h)
    lo = h.lmin if lo is None else lo
    nl = h.lmax - h.lmin + 1
    if sel is None:
        counts = n.copy()
        sels = None
    else:
        sels = [np.ascontiguousarray(sel.get(l, np.zeros(0, np.int64)), dtype=np.int64)
                for l in h.levels]
        counts = np.array([s.shape[0] for s in sels], dtype=np.int64)
    phi = [np.zeros(int(counts[k]), np.float64) for k in range(nl)]
    acc = [np.zeros((int(counts[k]), 3), np.float64) for k in range(nl)]
    t_ijk, t_mass = _ptr_array(ijk), _ptr_array(mass)
    t_phi, t_acc = _ptr_array(phi), _ptr_array(acc)
    if sels is None:
        nsel_p, sel_p = None, None
    else:
        nsel_p, sel_p = _ptr(counts), _ptr_array(sels)
    threads = threads or lib().oracle_max_threads()
    rc = fn(h.lmin, h.lmax, _ptr(n), t_ijk, t_mass, *extra_front, lo, nsel_p, sel_p,
            t_phi, t_acc, threads)
    if rc != 0:
        raise OracleError(rc)
    return ({l: phi[l - h.lmin] for l in h.levels if l >= lo},
            {l: acc[l - h.lmin] for l in h.levels if l >= lo})


def solve(h, p: int, G: float = 1.0, lo: int | None = None, sel: dict | None = None,
          threads: int | None = None, p_m: int | None = None, bottom: str = "m2p",
          vel: list | None = None, dt: list | None = None):
    """FMM potential and acceleration of the leaf cells of levels lo..lmax.

    sel maps level -> indices into that level's leaf list (None: all leaves).
    p_m: multipole order of M2L / M2P (None: p); bottom: "m2p" (the paper's bottom
    intermediate field) or "m2l" (M2L into the parent box, then L2P).
    vel[k] ([n, 3] velocities of level lmin+k) and dt[k] (time since level lmin+k was
    set): drift the multipoles of the stale trees below lo.
    Returns (phi, acc) dicts keyed by level."""
    mode = {"m2p": 0, "m2l": 1}[bottom]
    keep = None
    if vel is not None and dt is not None:
        keep = [np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3) for v in vel]
        t_vel = _ptr_array(keep)
        t_dt = np.ascontiguousarray(dt, dtype=np.float64)
        extra = (p, G, 0 if p_m is None else p_m, mode, t_vel, _ptr(t_dt))
    else:
        extra = (p, G, 0 if p_m is None else p_m, mode, None, None)
    out = _call(lib().oracle_fmm_solve, h, lo, sel, extra, threads)
    del keep
    return out


def solve_dl2(h, p: int, G: float = 1.0, sel: dict | None = None, threads: int | None = None,
              p_m: int | None = None):
    """The Delta l = 2 variant (finest FMM box = 4^3 cells, near field = the
    cells of the 3^3 neighbour boxes) on a single complete level h.lmin ==
    h.lmax >= 3.  Returns (phi, acc) dicts keyed by level."""
    if h.lmin != h.lmax:
        raise OracleError(-1)

    def fn(lmin, lmax, n, ijk, mass, p_, G_, pm_, lo, nsel, sel_, phi, acc, threads_):
        return lib().oracle_fmm_solve_dl2(lmin, n, ijk, mass, p_, G_, pm_, nsel, sel_, phi, acc, threads_)

    return _call(fn, h, None, sel, (p, G, 0 if p_m is None else p_m), threads)


def solve_periodic(h, p: int, G: float = 1.0, lo: int | None = None, sel: dict | None = None,
                   threads: int | None = None, p_m: int | None = None):
    """FMM with periodic boundaries (images everywhere, neutralising background;
    see fmm_oracle.cpp), bottom M2P, lmin >= 3.  Returns (phi, acc) dicts."""
    return _call(lib().oracle_fmm_solve_periodic, h, lo, sel, (p, G, 0 if p_m is None else p_m), threads)


def ewald(h, G: float = 1.0, alpha: float = 8.0, lo: int | None = None, sel: dict | None = None,
          threads: int | None = None):
    """The periodic potential and acceleration by Ewald's sum over all pairs
    (splitting parameter alpha >= 6; the result does not depend on it)."""
    return _call(lib().oracle_ewald_sum, h, lo, sel, (G, float(alpha)), threads)


def lattice_tensor(q: int, alpha: float = 2.0) -> np.ndarray:
    """T_gamma = d^gamma psi_far(0), |gamma| <= q, in multi-index order."""
    out = np.zeros(ncoef(q))
    lib().oracle_lattice_tensor(q, float(alpha), _ptr(out))
    return out


def direct(h, G: float = 1.0, lo: int | None = None, sel: dict | None = None,
           threads: int | None = None):
    """O(N^2) direct sum over all leaves (self term excluded)."""
    return _call(lib().oracle_direct_sum, h, lo, sel, (G,), threads)


def tree(h):
    """Canonical tree index: per level l >= 1, (oct_key, status, nbr)."""
    n, ijk, mass = _inputs(h)
    L = lib()
    n_oct = np.zeros(h.lmax + 1, np.int64)
    rc = L.oracle_tree(h.lmin, h.lmax, _ptr(n), _ptr_array(ijk), _ptr_array(mass),
                       _ptr(n_oct), None, None, None)
    if rc != 0:
        raise OracleError(rc)
    keys = [np.zeros(int(n_oct[l]), np.uint64) for l in range(h.lmax + 1)]
    status = [np.zeros(8 * int(n_oct[l]), np.int64) for l in range(h.lmax + 1)]
    nbr = [np.zeros(27 * int(n_oct[l]), np.int64) for l in range(h.lmax + 1)]
    rc = L.oracle_tree(h.lmin, h.lmax, _ptr(n), _ptr_array(ijk), _ptr_array(mass),
                       _ptr(n_oct), _ptr_array(keys), _ptr_array(status), _ptr_array(nbr))
    if rc != 0:
        raise OracleError(rc)
    return {l: (keys[l], status[l], nbr[l].reshape(-1, 27)) for l in range(1, h.lmax + 1)}


def validate(h) -> int:
    """0 if the hierarchy is a valid graded octree, else the oracle's error code."""
    n, ijk, mass = _inputs(h)
    n_oct = np.zeros(h.lmax + 1, np.int64)
    return lib().oracle_tree(h.lmin, h.lmax, _ptr(n), _ptr_array(ijk), _ptr_array(mass),
                             _ptr(n_oct), None, None, None)


# ---- unit operators (physical coordinates) --------------------------------

def ncoef(p: int) -> int:
    return lib().oracle_ncoef(p)


def multi_index(p: int) -> np.ndarray:
    out = np.zeros((ncoef(p), 3), np.int32)
    lib().oracle_multi_index(p, _ptr(out))
    return out


def inv_r_derivs(q: int, R) -> np.ndarray:
    R = np.ascontiguousarray(R, dtype=np.float64)
    out = np.zeros(ncoef(q), np.float64)
    lib().oracle_inv_r_derivs(q, _ptr(R), _ptr(out))
    return out


def numerators(q: int, u) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.int64)
    out = np.zeros(ncoef(q), np.int64)
    lib().oracle_numerators(q, _ptr(u), _ptr(out))
    return out


def p2m(p, m, x, c, M=None):
    M = np.zeros(ncoef(p)) if M is None else np.ascontiguousarray(M, dtype=np.float64).copy()
    lib().oracle_p2m(p, float(m), _ptr(np.asarray(x, np.float64)), _ptr(np.asarray(c, np.float64)), _ptr(M))
    return M


def m2m(p, Mc, cc, cp, Mp=None):
    Mp = np.zeros(ncoef(p)) if Mp is None else np.ascontiguousarray(Mp, dtype=np.float64).copy()
    Mc = np.ascontiguousarray(Mc, dtype=np.float64)
    lib().oracle_m2m(p, _ptr(Mc), _ptr(np.asarray(cc, np.float64)), _ptr(np.asarray(cp, np.float64)), _ptr(Mp))
    return Mp


def m2l(p, M, cs, ct, L=None):
    L = np.zeros(ncoef(p)) if L is None else np.ascontiguousarray(L, dtype=np.float64).copy()
    M = np.ascontiguousarray(M, dtype=np.float64)
    lib().oracle_m2l(p, _ptr(M), _ptr(np.asarray(cs, np.float64)), _ptr(np.asarray(ct, np.float64)), _ptr(L))
    return L


def l2l(p, Lp, cp, cc, Lc=None):
    Lc = np.zeros(ncoef(p)) if Lc is None else np.ascontiguousarray(Lc, dtype=np.float64).copy()
    Lp = np.ascontiguousarray(Lp, dtype=np.float64)
    lib().oracle_l2l(p, _ptr(Lp), _ptr(np.asarray(cp, np.float64)), _ptr(np.asarray(cc, np.float64)), _ptr(Lc))
    return Lc


def l2p(p, L, c, x):
    """Returns [phi, dphi/dx, dphi/dy, dphi/dz] of the local expansion at x."""
    out = np.zeros(4)
    L = np.ascontiguousarray(L, dtype=np.float64)
    lib().oracle_l2p(p, _ptr(L), _ptr(np.asarray(c, np.float64)), _ptr(np.asarray(x, np.float64)), _ptr(out))
    return out


def m2p(p, M, cs, x):
    """Returns [phi, dphi/dx, dphi/dy, dphi/dz] of the multipole at x (g = -1/r)."""
    out = np.zeros(4)
    M = np.ascontiguousarray(M, dtype=np.float64)
    lib().oracle_m2p(p, _ptr(M), _ptr(np.asarray(cs, np.float64)), _ptr(np.asarray(x, np.float64)), _ptr(out))
    return out
