"""torch.autograd support: gradients of losses on phi / accel with respect to
the cell masses, through the library's adjoint solve (fmm_solve_adjoint).

The tree structure (cell indices) is fixed; the masses are the differentiable
inputs.  Forward runs fmm_set_levels + fmm_solve, backward fmm_solve_adjoint;
both are FP64 (the adjoint needs an FP64 solver)."""
from __future__ import annotations

import torch

from . import fmm


class _Potential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, lmin, lmax, lo, ijk, *masses):
        solver.set_levels(lmin, lmax, list(ijk), [m.detach().contiguous() for m in masses])
        phi, acc = solver.solve(lo)
        ctx.solver, ctx.lo, ctx.lmin, ctx.lmax = solver, lo, lmin, lmax
        levels = range(lo, lmax + 1)
        return tuple(phi[l] for l in levels) + tuple(acc[l] for l in levels)

    @staticmethod
    def backward(ctx, *grads):
        s, lo, lmax = ctx.solver, ctx.lo, ctx.lmax
        levels = list(range(lo, lmax + 1))
        k = len(levels)
        g_phi, g_acc = {}, {}
        for i, l in enumerate(levels):
            gp, ga = grads[i], grads[k + i]
            g_phi[l] = (gp if gp is not None else torch.zeros(s.n[l], dtype=torch.float64, device="cuda")).contiguous()
            g_acc[l] = (ga if ga is not None else torch.zeros(s.n[l], 3, dtype=torch.float64, device="cuda")).contiguous()
        gm = s.solve_adjoint(g_phi, g_acc, lo=lo)
        return (None, None, None, None, None) + tuple(gm[l] for l in range(ctx.lmin, lmax + 1))


def potential(solver: "fmm.Solver", lmin: int, lmax: int, ijk, masses, lo: int | None = None):
    """phi, accel of the leaves of levels lo..lmax as differentiable functions of
    `masses` (list of float64 device tensors, levels lmin..lmax; `ijk` the matching
    int32 [n,3] device tensors).  Returns (phi, acc): dicts level -> tensor."""
    if solver.precision != "fp64":
        raise ValueError("gradients need an FP64 solver (fmm.Solver(p, 'fp64'))")
    lo = lmin if lo is None else lo
    out = _Potential.apply(solver, lmin, lmax, lo, tuple(ijk), *masses)
    levels = list(range(lo, lmax + 1))
    k = len(levels)
    return {l: out[i] for i, l in enumerate(levels)}, {l: out[k + i] for i, l in enumerate(levels)}
