"""Seeded synthetic AMR hierarchies (inputs only; none of the solver's arithmetic).

A hierarchy is a graded octree over the unit box (Sec. 3.2 of the paper): per
AMR level l in [lmin, lmax] a list of leaf cells (integer ijk in [0, 2^l)) with
masses.  Refined cells are implied (they are the parents of finer cells).
Every generator is deterministic: random numbers come from a counter-based
SplitMix64 stream keyed by (seed, stream, counter), so the same inputs are
produced on any machine.

The density recipes follow the workloads the method is measured on:
Plummer spheres sampled at cell centres with uniform or lognormal noise,
nested refined boxes, Gaussian blobs (Sec. 4 uses NFW halos and uniform
spheres built from particle deposits; those need the paper's initial
conditions, which stand in here as analytic profiles).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLD = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)
_STREAM = np.uint64(0xD1B54A32D192ED03)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) on uint64 arrays (wrapping)."""
    with np.errstate(over="ignore"):
        z = z + _GOLD
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, stream: int, counter: np.ndarray | int) -> np.ndarray:
    """U[0,1) doubles from (seed, stream, counter) with 53 random bits."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) * _GOLD + np.uint64(stream) * _STREAM + c
    z = _splitmix64(_splitmix64(z))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, counter: np.ndarray | int) -> np.ndarray:
    """Standard normal by Box-Muller from two independent uniform streams."""
    u1 = uniform(seed, 2 * stream + 1, counter)
    u2 = uniform(seed, 2 * stream + 2, counter)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class Hierarchy:
    """Leaf cells per AMR level; ijk[k], mass[k] belong to level lmin + k."""

    lmin: int
    lmax: int
    ijk: list = field(default_factory=list)    # int32 [n, 3] per level
    mass: list = field(default_factory=list)   # float64 [n] per level
    name: str = ""

    @property
    def levels(self):
        return list(range(self.lmin, self.lmax + 1))

    def n(self, level: int) -> int:
        return int(self.ijk[level - self.lmin].shape[0])

    @property
    def n_cells(self) -> int:
        return int(sum(a.shape[0] for a in self.ijk))

    def total_mass(self) -> float:
        return float(sum(m.sum() for m in self.mass))

    def centres(self, level: int) -> np.ndarray:
        return (self.ijk[level - self.lmin].astype(np.float64) + 0.5) * 2.0 ** (-level)

    def copy(self) -> "Hierarchy":
        return Hierarchy(self.lmin, self.lmax, [a.copy() for a in self.ijk],
                         [m.copy() for m in self.mass], self.name)


# ---------------------------------------------------------------------------
# Geometry: which cells are refined at each level.

def _grid(n: int) -> np.ndarray:
    ax = np.arange(n, dtype=np.int32)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    return g


def leaves_from_refined(lmin: int, lmax: int, refined: dict) -> list:
    """Leaf cells per level, given boolean refined masks per level.

    refined[l] is a dense bool array of shape (2^l,)*3 for l in [lmin, lmax-1];
    a level l+1 cell exists iff its parent is refined.  Returns a list of int32
    [n,3] leaf arrays for levels lmin..lmax (lexicographic order).
    """
    out = []
    exists = np.ones((2 ** lmin,) * 3, dtype=bool)
    for l in range(lmin, lmax + 1):
        ref = refined.get(l)
        if ref is None or l == lmax:
            ref = np.zeros_like(exists)
        leaf = exists & ~ref
        out.append(np.argwhere(leaf).astype(np.int32))
        if l < lmax:
            exists = np.repeat(np.repeat(np.repeat(exists & ref, 2, 0), 2, 1), 2, 2)
    return out


def graded_filter(refined_coarse: np.ndarray, cand_fine: np.ndarray) -> np.ndarray:
    """Keep candidate refinements at level l+1 allowed by the graded rule.

    A level-(l+1) cell may be refined only if the 3^3 neighbours of its father
    (level l) are all refined (Sec. 3.2).  refined_coarse: bool (2^l)^3;
    cand_fine: bool (2^(l+1))^3.
    """
    n = refined_coarse.shape[0]
    pad = np.pad(refined_coarse, 1, constant_values=True)  # outside the box: no constraint
    ok = np.ones_like(refined_coarse)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                ok &= pad[1 + dx:1 + dx + n, 1 + dy:1 + dy + n, 1 + dz:1 + dz + n]
    ok &= refined_coarse
    ok_f = np.repeat(np.repeat(np.repeat(ok, 2, 0), 2, 1), 2, 2)
    return cand_fine & ok_f


def nested_boxes(lmin: int, boxes: list) -> dict:
    """Refined masks for nested boxes: boxes[k] = (lo, hi) in level (lmin+k) cells,
    half-open, the cells of level lmin+k that are refined."""
    refined = {}
    for k, (lo, hi) in enumerate(boxes):
        l = lmin + k
        m = np.zeros((2 ** l,) * 3, dtype=bool)
        lo3 = np.broadcast_to(np.asarray(lo), (3,))
        hi3 = np.broadcast_to(np.asarray(hi), (3,))
        m[lo3[0]:hi3[0], lo3[1]:hi3[1], lo3[2]:hi3[2]] = True
        refined[l] = m
    return refined


# ---------------------------------------------------------------------------
# Densities (mass = rho(centre) * h^3, renormalised to total mass 1).

def plummer_rho(x: np.ndarray, centre, a: float, M: float = 1.0) -> np.ndarray:
    r2 = ((x - np.asarray(centre)) ** 2).sum(-1)
    return 3.0 * M / (4.0 * np.pi * a ** 3) * (1.0 + r2 / a ** 2) ** (-2.5)


def _assemble(lmin, lmax, leaves, rho_fn, name):
    h = Hierarchy(lmin, lmax, name=name)
    for k, c in enumerate(leaves):
        l = lmin + k
        x = (c.astype(np.float64) + 0.5) * 2.0 ** (-l)
        h.ijk.append(np.ascontiguousarray(c, dtype=np.int32))
        h.mass.append(rho_fn(x) * 8.0 ** (-l))
    return h


def _normalise(h: Hierarchy, total: float = 1.0) -> Hierarchy:
    s = h.total_mass()
    h.mass = [m * (total / s) for m in h.mass]
    return h


def _uniform_noise(h: Hierarchy, seed: int, amp: float) -> Hierarchy:
    for k, m in enumerate(h.mass):
        u = uniform(seed, 100 + h.lmin + k, np.arange(m.size))
        h.mass[k] = m * (1.0 + amp * (2.0 * u - 1.0))
    return h


def _lognormal_noise(h: Hierarchy, seed: int, sigma: float) -> Hierarchy:
    for k, m in enumerate(h.mass):
        xi = normal(seed, 200 + h.lmin + k, np.arange(m.size))
        h.mass[k] = m * np.exp(sigma * xi - 0.5 * sigma ** 2)
    return h


# ---------------------------------------------------------------------------
# The measured workloads.

def unigrid_plummer(level: int = 5, a: float = 0.1, noise: float = 0.01, seed: int = 1) -> Hierarchy:
    """Unigrid 2^level cubed, Plummer sphere (scale a, centred, M=1) at cell
    centres plus seeded uniform noise of relative amplitude `noise`."""
    leaves = leaves_from_refined(level, level, {})
    h = _assemble(level, level, leaves, lambda x: plummer_rho(x, (0.5, 0.5, 0.5), a),
                  f"unigrid {2**level}^3 plummer")
    return _normalise(_uniform_noise(_normalise(h), seed, noise))


def two_level_plummer(base: int = 6, lo: int = 24, hi: int = 40, a: float = 0.05,
                      sigma: float = 0.3, seed: int = 2) -> Hierarchy:
    """Base 2^base cubed plus one refined level over coarse cells [lo,hi)^3;
    Plummer density (scale a) with seeded lognormal noise (sigma)."""
    refined = nested_boxes(base, [(lo, hi)])
    leaves = leaves_from_refined(base, base + 1, refined)
    h = _assemble(base, base + 1, leaves, lambda x: plummer_rho(x, (0.5, 0.5, 0.5), a),
                  f"two-level {2**base}^3 + {2*(hi-lo)}^3 plummer")
    return _normalise(_lognormal_noise(_normalise(h), seed, sigma))


def nested_two_plummer(base: int = 7, boxes=((24, 104), (76, 180)), seed: int = 4) -> Hierarchy:
    """Base 2^base cubed with nested refined boxes (one per extra level), two
    Plummer spheres (a = 0.03 and 0.05, masses 1/2 each, centres 0.5 -+ 0.08 in x)."""
    refined = nested_boxes(base, list(boxes))
    lmax = base + len(boxes)
    leaves = leaves_from_refined(base, lmax, refined)

    def rho(x):
        return (plummer_rho(x, (0.42, 0.5, 0.5), 0.03, 0.5) +
                plummer_rho(x, (0.58, 0.5, 0.5), 0.05, 0.5))

    h = _assemble(base, lmax, leaves, rho, f"nested two-plummer {2**base}^3 + {len(boxes)} levels")
    return _normalise(h)


def random_amr(lmin: int, lmax: int, seed: int, frac: float = 0.3, blobs: int = 3) -> Hierarchy:
    """Small random graded hierarchy for tests: at each level a union of seeded
    spherical regions is proposed for refinement and filtered by the graded
    rule; masses are seeded lognormal."""
    refined = {}
    prev = None
    counter = 0
    for l in range(lmin, lmax):
        n = 2 ** l
        x = (_grid(n).astype(np.float64) + 0.5) / n
        cand = np.zeros(n ** 3, dtype=bool)
        for b in range(blobs):
            c = uniform(seed, 10 + l, np.arange(counter, counter + 3)) * 0.6 + 0.2
            counter += 3
            rad = frac * (0.5 + 0.5 * uniform(seed, 20 + l, counter))
            counter += 1
            cand |= ((x - c) ** 2).sum(-1) < rad ** 2
        cand = cand.reshape(n, n, n)
        if prev is not None:
            exists = np.repeat(np.repeat(np.repeat(prev, 2, 0), 2, 1), 2, 2)
            cand &= exists
            cand = graded_filter(prev, cand)
        refined[l] = cand
        prev = cand
        if not cand.any():
            break
    leaves = leaves_from_refined(lmin, lmax, refined)
    h = Hierarchy(lmin, lmax, name=f"random amr {lmin}-{lmax} seed {seed}")
    for k, c in enumerate(leaves):
        l = lmin + k
        h.ijk.append(np.ascontiguousarray(c, dtype=np.int32))
        xi = normal(seed, 300 + l, np.arange(c.shape[0]))
        h.mass.append(np.exp(0.5 * xi) * 8.0 ** (-l))
    return _normalise(h)


def permute(h: Hierarchy, seed: int) -> Hierarchy:
    """Same hierarchy with each level's leaf list in a seeded random order."""
    out = h.copy()
    for k in range(len(out.ijk)):
        n = out.ijk[k].shape[0]
        order = np.argsort(uniform(seed, 400 + k, np.arange(n)), kind="stable")
        out.ijk[k] = np.ascontiguousarray(out.ijk[k][order])
        out.mass[k] = np.ascontiguousarray(out.mass[k][order])
    return out


CONFIGS = {
    "unigrid32_p4": dict(make=lambda: unigrid_plummer(5), p=4),
    "twolevel64_p6": dict(make=lambda: two_level_plummer(), p=6),
    "nested128_p6": dict(make=lambda: nested_two_plummer(), p=6),
}


def _box_cells(lo, hi) -> np.ndarray:
    """All cells of the half-open box [lo, hi)^3 (per-axis bounds), int32 [n, 3]."""
    ax = [np.arange(lo[i], hi[i], dtype=np.int32) for i in range(3)]
    g = np.stack(np.meshgrid(*ax, indexing="ij"), -1)
    return g.reshape(-1, 3)


def _outside(cells: np.ndarray, lo, hi) -> np.ndarray:
    inside = np.all((cells >= np.asarray(lo)) & (cells < np.asarray(hi)), axis=1)
    return cells[~inside]


def blob_hierarchy(base: int, widths: list, seed: int, stream: int) -> Hierarchy:
    """Base grid 2^base cubed with up to len(widths) nested refined regions.

    Region k (cells of level base+k) is a box whose width is a fraction
    widths[k] of the width of the region it refines (the whole grid for k = 0,
    else the cells under the previous region), rounded to an even number of
    cells, with even corners (whole octs below it) and at least 2 parent cells
    (4 cells of its own level) inside that region, which keeps the graded rule.
    Nesting stops early when no such box fits.  Density: 1-8 Gaussian blobs
    (widths U(0.02, 0.1), centres U(0.2, 0.8)^3, amplitudes U(0.5, 2)) plus a
    small floor; total mass 1.  Built box by box, without dense masks."""
    ctr = [0]

    def u(n=1):
        v = uniform(seed, stream, np.arange(ctr[0], ctr[0] + n))
        ctr[0] += n
        return v

    margin = 4
    elo, ehi = np.zeros(3, np.int64), np.full(3, 2 ** base, np.int64)  # cells of the current level
    leaves = []
    for k, f in enumerate(widths + [None]):
        span = ehi - elo - 2 * margin
        w = None if f is None else 2 * np.maximum(1, np.round(f * (ehi - elo) / 2.0)).astype(np.int64)
        if f is None or np.any(span < w):
            leaves.append(_box_cells(elo, ehi))
            break
        lo = elo + margin + 2 * np.floor(u(3) * ((span - w) // 2 + 1)).astype(np.int64)
        hi = lo + w
        leaves.append(_outside(_box_cells(elo, ehi), lo, hi))
        elo, ehi = 2 * lo, 2 * hi
    nb = 1 + min(int(u()[0] * 8), 7)
    cen = 0.2 + 0.6 * u(3 * nb).reshape(nb, 3)
    sig = 0.02 + 0.08 * u(nb)
    amp = 0.5 + 1.5 * u(nb)
    peak = float((amp / sig ** 3).max())

    def rho(x):
        r = np.full(x.shape[0], 1e-6 * peak)
        for j in range(nb):
            r += amp[j] * np.exp(-((x - cen[j]) ** 2).sum(-1) / (2 * sig[j] ** 2)) / sig[j] ** 3
        return r

    lmax = base + len(leaves) - 1
    h = _assemble(base, lmax, leaves, rho, f"blobs {2**base}^3 + {lmax - base} levels")
    return _normalise(h)


def batched_blobs(count: int = 64, seed: int = 5, bases=(5, 6, 7)) -> list:
    """`count` independent isolated hierarchies for one batched solve: base grid
    2^b cubed with b drawn from `bases`, 1-3 nested refinement levels, each
    refined region a seeded 1/4-1/2 of its parent's width, Gaussian-blob
    densities (1-8 blobs, widths 0.02-0.1 box)."""
    out = []
    for i in range(count):
        v = uniform(seed, 900, np.arange(5 * i, 5 * i + 5))
        base = bases[min(int(v[0] * len(bases)), len(bases) - 1)]
        nlev = 1 + min(int(v[1] * 3), 2)
        widths = [0.25 + 0.25 * float(x) for x in v[2:2 + nlev]]
        out.append(blob_hierarchy(base, widths, seed, 1000 + i))
    return out


def gaussian_field(n: int, slope: float, seed: int, stream: int = 0) -> np.ndarray:
    """Periodic Gaussian random field on an n^3 grid with power spectrum
    P(k) ~ k^slope (k in grid units, the k = 0 mode removed), normalised to
    zero mean and unit variance; white noise from the counter-based generator."""
    white = normal(seed, stream, np.arange(n ** 3)).reshape(n, n, n)
    f = np.fft.rfftn(white)
    kx = np.fft.fftfreq(n) * n
    kz = np.fft.rfftfreq(n) * n
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    amp[k2 > 0] = k2[k2 > 0] ** (slope / 4.0)  # sqrt(P(k)) = k^(slope/2)
    g = np.fft.irfftn(f * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    return g / g.std()


def _keys(idx: np.ndarray, level: int) -> np.ndarray:
    n = np.int64(2 ** level)
    return (idx[:, 0].astype(np.int64) * n + idx[:, 1]) * n + idx[:, 2]


_OFF27 = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)], np.int64)
_OFF8 = np.array([(c & 1, (c >> 1) & 1, (c >> 2) & 1) for c in range(8)], np.int64)


def _neighbour_keys(idx: np.ndarray, level: int):
    """Keys of the 27 neighbours of each cell (K x 27) and their in-box mask."""
    nb = idx[:, None, :] + _OFF27[None, :, :]
    ok = np.all((nb >= 0) & (nb < 2 ** level), axis=2)
    return _keys(np.clip(nb, 0, 2 ** level - 1).reshape(-1, 3), level).reshape(-1, 27), ok


def lognormal_amr(base: int = 8, sigma: float = 1.0, slope: float = -2.0, threshold: float = 8.0,
                  max_levels: int = 4, sigma_sub: float = 0.5, seed: int = 6,
                  max_leaves: int = 64_000_000) -> Hierarchy:
    """Lognormal density on a 2^base cubed base grid with mass refinement.

    Base cells: rho = exp(sigma g - sigma^2/2), g a Gaussian field with
    P(k) ~ k^slope (mean density 1).  A cell is flagged when its mass exceeds
    `threshold` times the mean base-cell mass (a fixed mass, the
    quasi-Lagrangian criterion, at every level); flags are dilated by one cell
    (within the existing cells) and, above the base, kept only where the graded
    rule allows; flagged cells are refined, up to `max_levels` levels.  A
    refined cell's mass is shared by its 8 children with seeded lognormal
    weights (sigma_sub), normalised per oct, so mass is conserved.  If fewer
    than `max_levels` levels appear, sigma_sub is raised once by half (the
    name records the value used).  Refinement also stops before the leaves
    would exceed `max_leaves`.  Sparse throughout (sorted cell keys)."""
    n = 2 ** base
    g = gaussian_field(n, slope, seed)
    m_thr = threshold / n ** 3

    def build(ssub):
        idx = np.argwhere(np.ones((n,) * 3, dtype=bool)).astype(np.int64)
        mass = np.exp(sigma * g[idx[:, 0], idx[:, 1], idx[:, 2]] - 0.5 * sigma ** 2) / n ** 3
        ref_keys_prev = None
        leaves, lmass = [], []
        total = 0
        for k in range(max_levels + 1):
            l = base + k
            keys = _keys(idx, l)
            order = np.argsort(keys)
            keys, idx, mass = keys[order], idx[order], mass[order]
            cand = np.zeros(keys.size, dtype=bool)
            if k < max_levels:
                fl = idx[mass > m_thr]
                if fl.size:
                    nk, ok = _neighbour_keys(fl, l)
                    dil = np.unique(nk[ok])
                    cand = np.isin(keys, dil)
                if k > 0 and cand.any():  # graded: the father's 27 neighbours must be refined
                    fk, fok = _neighbour_keys(idx[cand] // 2, l - 1)
                    good = np.all(np.isin(fk, ref_keys_prev) | ~fok, axis=1)
                    sel = np.flatnonzero(cand)
                    cand[sel[~good]] = False
                if total + int((~cand).sum()) + 8 * int(cand.sum()) > max_leaves:
                    cand[:] = False
            leaves.append(idx[~cand].astype(np.int32))
            lmass.append(mass[~cand])
            total += int((~cand).sum())
            if not cand.any():
                break
            ref_keys_prev = keys[cand]
            par, pm = idx[cand], mass[cand]
            w = np.exp(ssub * normal(seed, 500 + l, np.arange(8 * par.shape[0])).reshape(-1, 8) - 0.5 * ssub ** 2)
            w /= w.sum(1, keepdims=True)
            idx = (2 * par[:, None, :] + _OFF8[None, :, :]).reshape(-1, 3)
            mass = (pm[:, None] * w).reshape(-1)
        return leaves, lmass

    ssub = sigma_sub
    leaves, lmass = build(ssub)
    if len(leaves) - 1 < max_levels:
        ssub = 1.5 * sigma_sub
        leaves, lmass = build(ssub)
    lmax = base + len(leaves) - 1
    h = Hierarchy(base, lmax, name=f"lognormal {n}^3 sigma={sigma} P(k)~k^{slope:g}, sigma_sub={ssub:g}, "
                                   f"{lmax - base} refined levels")
    for c, m in zip(leaves, lmass):
        h.ijk.append(np.ascontiguousarray(c, dtype=np.int32))
        h.mass.append(np.ascontiguousarray(m, dtype=np.float64))
    return _normalise(h)


def ats_schedule(lmin: int, lmax: int) -> list:
    """The solves of one coarse step with adaptive time stepping (Alg. 1 inside
    the amr_step recursion): level l is rebuilt and solved (levels l..lmax) when
    l = lmin or on its second substep.  Returns the list of lo values in order;
    lo = k occurs 2^(k-lmin-1) times for k > lmin."""
    out = []

    def step(l, icount):
        if l == lmin or icount > 1:
            out.append(l)
        if l < lmax:
            step(l + 1, 1)
            step(l + 1, 2)

    step(lmin, 1)
    return out
