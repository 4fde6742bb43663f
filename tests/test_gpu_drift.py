"""Multipole drifting of stale trees (fmm_set_velocities, fmm_set_drift) against
the oracle's drifting, and its bookkeeping: a zero time step changes nothing,
drifting without velocities is refused, and a later solve without drifting
recomputes the undrifted multipoles."""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W
from _parity import check, oracle_tol, self_tol

pytestmark = pytest.mark.gpu


def _np(phi, acc):
    import torch
    torch.cuda.synchronize()
    return {l: phi[l].double().cpu().numpy() for l in phi}, {l: acc[l].double().cpu().numpy() for l in acc}


def _case(seed=13):
    h = W.lognormal_amr(base=5, seed=6) if seed is None else W.random_amr(3, 5, seed=seed)
    vel = [0.3 * W.normal(5, 10 + k, np.arange(3 * h.n(l))).reshape(-1, 3) for k, l in enumerate(h.levels)]
    return h, vel


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("seed", [13, None])
def test_drift_matches_oracle(precision, seed):
    from paper_2607_19489_b300 import fmm
    h, vel = _case(seed)
    nl = h.lmax - h.lmin + 1
    s = fmm.Solver(6, precision)
    s.set_hierarchy(h)
    s.set_velocities(vel)
    for lo in range(h.lmin + 1, h.lmax + 1):
        dt = [0.02 * (1 + k) if h.lmin + k < lo else 0.0 for k in range(nl)]
        s.set_drift(dt)
        phi, acc = s.solve(lo)
        s.sync()
        got = _np(phi, acc)
        ref = oracle.solve(h, 6, lo=lo, vel=vel, dt=dt)
        check(*got, *ref, oracle_tol(precision), f"drift lo={lo} {precision}", h=h)
        undrifted = oracle.solve(h, 6, lo=lo)
        moved = max(float(np.abs(ref[1][l] - undrifted[1][l]).max() / np.abs(undrifted[1][l]).max())
                    for l in ref[1] if ref[1][l].size)
        if lo > h.lmin + 1 or seed is not None:
            assert moved > 1e-5, (lo, moved)   # the case really drifts something


def test_zero_step_and_off_change_nothing_and_velocities_are_required():
    from paper_2607_19489_b300 import fmm
    h, vel = _case(13)
    nl = h.lmax - h.lmin + 1
    lo = h.lmax
    s = fmm.Solver(6, "fp64")
    s.set_hierarchy(h)
    base = _np(*s.solve(lo))
    s.set_drift([0.1] * nl)
    with pytest.raises(fmm.FMMError) as e:   # drifting stale levels needs their velocities
        s.solve(lo)
    assert e.value.name == "FMM_ERR_STATE"
    s.set_velocities(vel)
    s.set_drift([0.0] * nl)
    zero = _np(*s.solve(lo))
    s.sync()
    check(*zero, *base, self_tol("fp64"), "dt = 0")
    s.set_drift([0.05] * nl)
    moved = _np(*s.solve(lo))
    s.set_drift(None)   # off again: the next solve rebuilds the undrifted multipoles
    again = _np(*s.solve(lo))
    s.sync()
    check(*again, *base, self_tol("fp64"), "drift off after a drifted solve")
    assert max(float(np.abs(moved[1][l] - base[1][l]).max()) for l in base[1] if base[1][l].size) > 0
    # a new hierarchy invalidates the velocities of the levels it replaces
    s.set_drift([0.05] * nl)
    s.set_hierarchy(h, lo=h.lmax)
    s.solve(h.lmax)   # only levels < lmax are stale: their velocities are still valid
    s.set_hierarchy(h)
    with pytest.raises(fmm.FMMError):
        s.solve(h.lmax)
