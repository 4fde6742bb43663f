"""Comparison of solver outputs with reference outputs, used by every GPU test.

Two numbers are checked for each output (phi, then accel):
  * the relative RMS error over all compared cells (the accuracy metric of the
    method: sqrt(sum |x - x_ref|^2 / sum |x_ref|^2));
  * a per-cell bound, max_i |x_i - x_ref,i| / max(|x_ref,i|, floor), with
    floor = FLOOR x the RMS magnitude of the reference over the compared cells
    (accelerations vanish at centres of symmetry, where a plain relative error
    would be meaningless).
A relative RMS alone hides a localised fault: one interface cell 0.3 % wrong
among a few thousand moves it by ~5e-5 only.  The per-cell bound catches it.
With periodic boundaries the field is the small remainder of large partial
sums: the images of every mass and the uniform background cancel to a
potential of zero mean (it crosses zero on a surface through every
hierarchy) and to accelerations far below those of the isolated problem.
The partial sums are of the size of the field scale G M_total / L (L = 1),
and a fixed-precision path rounds them at that size, so the reduced-precision
tests of that mode measure errors against max(RMS of the reference, G
M_total) (`scales`), the per-cell floor for phi is 10 % of that
(PERIODIC_PHI_FLOOR: it still flags a typical cell 0.3 % wrong), and TF32,
whose 10-bit operands round the image terms by up to ~1e-3 of their size with
a systematic part, has the bar ORACLE_TF32_PERIODIC.  The FP64 path keeps the
plain relative bars (and pins the zero-mean convention).
On failure the message names the worst cell: its level, its index in the
compared set and, when the hierarchy is given, its (i, j, k).
"""
from __future__ import annotations

import numpy as np

FLOOR = 1e-2
PERIODIC_PHI_FLOOR = 1e-1

# against the FP64 oracle
ORACLE_FP64 = {"rms": 1e-10, "cell": 1e-9}
ORACLE_MIXED = {"rms": 1e-4, "cell": 1e-3}
# TF32: one product per term with 10-bit mantissas, each operand rounded by up to
# 2^-11 (4.9e-4 relative), so a product carries up to ~1e-3 and, with
# independent rounding over the terms, an RMS of ~3e-4 of the far-field part.
# The relative RMS bar is that (measured 0.6-1.4e-4 on random AMR, under 1e-4 on
# the two-level workload); a cell whose acceleration is a few times smaller than
# the far-field terms summed into it (a partial cancellation, bounded below by
# the 1 % floor) sees the per-term error amplified: the per-cell bar is 1e-2.
ORACLE_TF32 = {"rms": 3e-4, "cell": 1e-2}
ORACLE_TF32_PERIODIC = {"rms": 1e-3, "cell": 1e-2}
# the same kernels run twice (another launch shape, another order of the FP32
# atomic additions, graph vs direct launches)
SELF_FP64 = {"rms": 1e-12, "cell": 1e-11}
SELF_MIXED = {"rms": 1e-5, "cell": 1e-4}


def oracle_tol(precision: str) -> dict:
    return {"fp64": ORACLE_FP64, "tf32": ORACLE_TF32}.get(precision, ORACLE_MIXED)


def self_tol(precision: str) -> dict:
    return SELF_FP64 if precision == "fp64" else SELF_MIXED


def _rows(a) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    return a.reshape(a.shape[0], -1) if a.ndim else a.reshape(1, 1)


def errors(got: dict, ref: dict, floor_frac: float = FLOOR, scale: float = 0.0):
    """(relative RMS, worst per-cell relative error, (level, index) of that cell).
    Errors are relative to max(RMS of the reference, scale)."""
    levels = [l for l in ref if np.asarray(ref[l]).size]
    if not levels:
        return 0.0, 0.0, None
    num = den = 0.0
    mags = {}
    for l in levels:
        r = _rows(ref[l])
        g = _rows(got[l])
        assert g.shape == r.shape, (l, g.shape, r.shape)
        num += float(((g - r) ** 2).sum())
        den += float((r ** 2).sum())
        mags[l] = np.sqrt((r ** 2).sum(1))
    n = sum(m.size for m in mags.values())
    norm = max(np.sqrt(den / max(n, 1)), scale)
    floor = floor_frac * norm
    worst, where = 0.0, None
    for l in levels:
        d = np.sqrt(((_rows(got[l]) - _rows(ref[l])) ** 2).sum(1))
        rel = d / np.maximum(mags[l], floor)
        if not np.all(np.isfinite(rel)):
            i = int(np.where(~np.isfinite(rel))[0][0])
            return float("inf"), float("inf"), (l, i)
        i = int(np.argmax(rel))
        if rel[i] > worst:
            worst, where = float(rel[i]), (l, i)
    if scale > 0:
        return float(np.sqrt(num / max(n, 1)) / norm), worst, where
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num)), worst, where


def check(got_phi: dict, got_acc: dict, ref_phi: dict, ref_acc: dict, tol: dict, what: str = "",
          h=None, sel: dict | None = None, outputs=("accel", "phi"), floors: dict | None = None,
          scales: dict | None = None) -> dict:
    """Assert both bounds for accel and phi; returns the measured errors.  floors:
    per output, the per-cell floor as a fraction of the RMS (default FLOOR);
    scales: per output, a field scale the errors are measured against when it
    exceeds the reference's RMS."""
    out = {}
    pairs = {"accel": (got_acc, ref_acc), "phi": (got_phi, ref_phi)}
    for name in outputs:
        got, ref = pairs[name]
        rms, cell, where = errors(got, ref, (floors or {}).get(name, FLOOR), (scales or {}).get(name, 0.0))
        out[name] = (rms, cell)
        if rms <= tol["rms"] and cell <= tol["cell"]:
            continue
        loc = ""
        if where is not None:
            l, i = where
            loc = f" at level {l}, compared cell {i}"
            if h is not None:
                idx = int(sel[l][i]) if sel is not None else i
                loc += f" (input index {idx}, ijk {tuple(int(x) for x in h.ijk[l - h.lmin][idx])})"
        raise AssertionError(f"{what} {name}: rel-RMS {rms:.3e} (bar {tol['rms']:.0e}), worst cell "
                             f"{cell:.3e} (bar {tol['cell']:.0e}){loc}")
    return out


def check_arrays(got: dict, ref: dict, tol: dict, what: str = "") -> tuple:
    """Both bounds for one output family (dict level -> array)."""
    rms, cell, where = errors(got, ref)
    assert rms <= tol["rms"] and cell <= tol["cell"], (
        f"{what}: rel-RMS {rms:.3e} (bar {tol['rms']:.0e}), worst cell {cell:.3e} (bar {tol['cell']:.0e}) at {where}")
    return rms, cell
