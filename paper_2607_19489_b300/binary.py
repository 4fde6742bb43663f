"""The binary orbit test of the paper (Sec. 4, Figs. 5-6): two equal point masses
on a circular orbit, evolved with the solver in the paper's particle-mesh form.

Each step:
  * the AMR grid follows the particles: the level-lmax cells of each particle's
    cloud-in-cell (CIC) stencil are refined into, their parent cells and
    `nexpand` layers around them are refined at level lmax-1, and every coarser
    level refines the parents of the finer refined cells and the layers the
    graded rule (Sec. 3.2) and `nexpand` require; level lmin covers the box;
  * the particle masses are deposited onto the level-lmax cells by CIC (the
    paper's mass deposition, Sec. 1);
  * the solver gives every cell's acceleration; each particle's is the CIC
    interpolation from the same eight cells (the same weights as the deposit,
    so pair forces stay equal and opposite where the field is);
  * kick-drift-kick leapfrog with a fixed step (no subcycling), as in the paper.

The grid building, deposit and interpolation of two particles are host
bookkeeping; every field evaluation is the library's solve.  Diagnostics follow
Fig. 6: relative change of the total energy (kinetic plus the two-body
potential energy -G m1 m2 / r) and of the angular momentum about the centre of
mass, centre-of-mass drift, relative change of the separation, phase drift and
the mean distance from the analytic circular orbit.
"""
from __future__ import annotations

import numpy as np

from . import fmm


def _dilate(mask: np.ndarray, k: int) -> np.ndarray:
    """k layers of the 3x3x3 neighbourhood (separable: one axis after the other)."""
    out = mask.copy()
    for _ in range(k):
        for axis in range(3):
            src = np.moveaxis(out.copy(), axis, 0)
            dst = np.moveaxis(out, axis, 0)
            dst[1:] |= src[:-1]
            dst[:-1] |= src[1:]
    return out


def _cic(pos: np.ndarray, level: int):
    """Lower cell index and weights of the CIC stencils (8 cells of `level` whose
    centres surround each particle)."""
    n = 1 << level
    u = pos * n - 0.5
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    cells, w = [], []
    for c in range(8):
        b = np.array([(c >> a) & 1 for a in range(3)])
        cells.append(i0 + b)
        w.append(np.prod(np.where(b, f, 1.0 - f), axis=1))
    return np.stack(cells, 1), np.stack(w, 1)  # [np, 8, 3], [np, 8]


def build_grid(pos: np.ndarray, lmin: int, lmax: int, nexpand: int = 2):
    """Leaf cells per level (lmin..lmax) of the graded hierarchy around the particles;
    returns the list of int32 [n, 3] arrays."""
    refined = {}
    cells, _ = _cic(pos, lmax)
    if lmax > lmin:
        n = 1 << (lmax - 1)
        m = np.zeros((n,) * 3, bool)
        par = cells.reshape(-1, 3) >> 1
        m[par[:, 0], par[:, 1], par[:, 2]] = True
        refined[lmax - 1] = _dilate(m, nexpand)
        for l in range(lmax - 2, lmin - 1, -1):
            fine = refined[l + 1]
            m = fine.reshape(1 << l, 2, 1 << l, 2, 1 << l, 2).any(axis=(1, 3, 5))
            refined[l] = _dilate(m, max(1, nexpand))  # graded rule: the parent's 3^3 neighbours
        for l in range(lmin + 1, lmax):  # a refined cell needs a refined parent
            up = np.repeat(np.repeat(np.repeat(refined[l - 1], 2, 0), 2, 1), 2, 2)
            refined[l] &= up
    out = []
    for l in range(lmin, lmax + 1):
        n = 1 << l
        exists = np.ones((n,) * 3, bool) if l == lmin else np.repeat(
            np.repeat(np.repeat(refined[l - 1], 2, 0), 2, 1), 2, 2)
        leaf = exists & ~refined.get(l, np.zeros((n,) * 3, bool))
        out.append(np.ascontiguousarray(np.argwhere(leaf).astype(np.int32)))
    return out


class Binary:
    """Two masses m (G = 1) at separation r0 about the box centre, circular orbit in
    the xy plane."""

    def __init__(self, lmin: int = 6, lmax: int = 6, p: int = 6, precision: str = "mixed", gm: float = 0.01,
                 r0: float = 0.15, nexpand: int = 2):
        self.lmin, self.lmax, self.nexpand = lmin, lmax, nexpand
        self.m = np.array([gm, gm])
        self.r0 = r0
        self.omega = np.sqrt(2 * gm / r0 ** 3)
        c = np.array([0.5, 0.5, 0.5])
        self.c = c
        self.x = np.array([c + [r0 / 2, 0, 0], c - [r0 / 2, 0, 0]])
        v = self.omega * r0 / 2
        self.v = np.array([[0, v, 0], [0, -v, 0]], float)
        self.t = 0.0
        self.solver = fmm.Solver(p, precision)
        self.solves = 0

    def accel(self) -> np.ndarray:
        import torch
        lev = build_grid(self.x, self.lmin, self.lmax, self.nexpand)
        cells, w = _cic(self.x, self.lmax)
        k = self.lmax - self.lmin
        fine = lev[k]
        n = 1 << self.lmax
        key = fine[:, 0].astype(np.int64) * n * n + fine[:, 1] * n + fine[:, 2]
        order = np.argsort(key)
        q = cells[..., 0] * n * n + cells[..., 1] * n + cells[..., 2]
        idx = order[np.searchsorted(key[order], q)]
        assert np.array_equal(key[idx], q), "a CIC stencil cell is not a leaf of the finest level"
        mass = [np.zeros(len(a)) for a in lev]
        np.add.at(mass[k], idx.reshape(-1), (w * self.m[:, None]).reshape(-1))
        self.solver.set_levels(self.lmin, self.lmax, [torch.as_tensor(a, device="cuda") for a in lev],
                               [torch.as_tensor(m, device="cuda") for m in mass])
        _, acc = self.solver.solve()
        self.solves += 1
        a = acc[self.lmax][torch.as_tensor(idx.reshape(-1), device="cuda")].double().cpu().numpy().reshape(2, 8, 3)
        if not np.isfinite(a).all():
            bad = {l: int((~torch.isfinite(acc[l])).any(1).sum()) for l in acc}
            raise FloatingPointError(f"non-finite acceleration at t = {self.t:.6f} (solve {self.solves}): stencil "
                                     f"cells {np.argwhere(~np.isfinite(a).all(2)).tolist()}, non-finite cells per "
                                     f"level {bad}, leaves per level {[len(q) for q in lev]}, x = {self.x.tolist()}")
        return (w[..., None] * a).sum(1)

    def run(self, t_end: float, dt: float) -> dict:
        a = self.accel()
        e0, l0, com0 = self.energy(), self.ang_mom(), self.com()
        steps = int(round(t_end / dt))
        for _ in range(steps):
            self.v += 0.5 * dt * a
            self.x += dt * self.v
            a = self.accel()
            self.v += 0.5 * dt * a
            self.t += dt
        return self.diagnostics(e0, l0, com0)

    def energy(self) -> float:
        r = np.linalg.norm(self.x[0] - self.x[1])
        return 0.5 * float((self.m * (self.v ** 2).sum(1)).sum()) - self.m[0] * self.m[1] / r

    def com(self) -> np.ndarray:
        return (self.m[:, None] * self.x).sum(0) / self.m.sum()

    def ang_mom(self) -> float:
        d = self.x - self.com()
        return float((self.m * np.cross(d, self.v)[:, 2]).sum())

    def diagnostics(self, e0, l0, com0) -> dict:
        sep = self.x[0] - self.x[1]
        r = float(np.linalg.norm(sep))
        phase = float(np.arctan2(sep[1], sep[0]))
        ana = self.omega * self.t
        dphi = float((phase - ana + np.pi) % (2 * np.pi) - np.pi)
        u = np.array([np.cos(ana), np.sin(ana), 0.0]) * self.r0 / 2
        x_ana = np.array([self.c + u, self.c - u])
        return {"t": self.t, "dE_over_E0": (self.energy() - e0) / abs(e0), "dL_over_L0": (self.ang_mom() - l0) / abs(l0),
                "com_drift": float(np.linalg.norm(self.com() - com0)), "dr_over_r0": (r - self.r0) / self.r0,
                "phase_drift": dphi, "mean_deviation": float(np.linalg.norm(self.x - x_ana, axis=1).mean()),
                "solves": self.solves}
