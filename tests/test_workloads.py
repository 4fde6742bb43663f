"""Seeded synthetic workloads: valid graded hierarchies, reproducible."""
import numpy as np

import oracle
from paper_2607_19489_b300 import workloads as W


def test_batched_blobs_are_valid_and_seeded():
    a = W.batched_blobs(count=8, seed=4, bases=(4, 5))
    b = W.batched_blobs(count=8, seed=4, bases=(4, 5))
    assert len(a) == 8
    assert any(h.lmax > h.lmin for h in a)
    for h, g in zip(a, b):
        assert 0 <= h.lmax - h.lmin <= 3
        assert h.lmin in (4, 5)
        oracle.validate(h)  # graded, complete octs, base level covers the box
        assert abs(h.total_mass() - 1.0) < 1e-12
        for x, y in zip(h.ijk, g.ijk):
            assert np.array_equal(x, y)
        for x, y in zip(h.mass, g.mass):
            assert np.array_equal(x, y)
    c = W.batched_blobs(count=8, seed=5, bases=(4, 5))
    assert any(h.n_cells != g.n_cells or h.lmin != g.lmin for h, g in zip(a, c))


def test_blob_boxes_span_a_quarter_to_a_half():
    h = W.blob_hierarchy(5, [0.25, 0.5], seed=1, stream=7)
    # refined region of level 5 = the parents of the level-6 cells
    par = np.unique(h.ijk[1] // 2, axis=0)
    ext = par.max(0) - par.min(0) + 1
    assert np.all(ext == 8)                      # 0.25 of 32 cells
    par6 = np.unique(h.ijk[2] // 2, axis=0)
    ext6 = par6.max(0) - par6.min(0) + 1
    assert np.all(ext6 == 8)                     # 0.5 of the 16-cell level-6 region


def test_ats_schedule_counts_and_order():
    assert W.ats_schedule(2, 4) == [2, 4, 3, 4]
    s = W.ats_schedule(8, 12)
    for k in range(8, 13):
        assert s.count(k) == (1 if k == 8 else 2 ** (k - 9))
    assert W.ats_schedule(5, 5) == [5]


def test_gaussian_field_spectrum():
    g = W.gaussian_field(32, -2.0, seed=3)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    f = np.abs(np.fft.fftn(g)) ** 2
    k = np.sqrt(sum(a ** 2 for a in np.meshgrid(*[np.fft.fftfreq(32) * 32] * 3, indexing="ij")))
    shells = [(4, 6), (8, 12)]
    p = [f[(k >= a) & (k < b)].mean() for a, b in shells]
    slope = np.log(p[1] / p[0]) / np.log(10.0 / 5.0)
    assert -2.6 < slope < -1.4


def test_lognormal_amr_threshold_and_validity():
    h = W.lognormal_amr(base=5, seed=6)
    oracle.validate(h)
    assert h.lmax > h.lmin
    assert abs(h.total_mass() - 1.0) < 1e-12
    # base-level leaves were not flagged: their mass is at most 8x the mean base-cell
    # mass, i.e. their density rho = exp(g - 1/2) is at most 8
    g = W.gaussian_field(32, -2.0, seed=6)
    c = h.ijk[0]
    assert np.exp(g[c[:, 0], c[:, 1], c[:, 2]] - 0.5).max() <= 8.0
    # and every flagged cell was refined
    flagged = np.argwhere(np.exp(g - 0.5) > 8.0)
    leaf = set(map(tuple, c.tolist()))
    assert not any(tuple(x) in leaf for x in flagged.tolist())
