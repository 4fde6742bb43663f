"""Seeded synthetic workloads: valid graded hierarchies, reproducible."""
import numpy as np

import oracle
from paper_2607_19489_b300 import workloads as W


def test_batched_blobs_are_valid_and_seeded():
    a = W.batched_blobs(count=8, seed=3, bases=(3, 4))
    b = W.batched_blobs(count=8, seed=3, bases=(3, 4))
    assert len(a) == 8
    for h, g in zip(a, b):
        assert 1 <= h.lmax - h.lmin <= 3
        assert h.lmin in (3, 4)
        oracle.validate(h)  # graded, complete octs, base level covers the box
        assert abs(h.total_mass() - 1.0) < 1e-12
        for x, y in zip(h.ijk, g.ijk):
            assert np.array_equal(x, y)
        for x, y in zip(h.mass, g.mass):
            assert np.array_equal(x, y)
    c = W.batched_blobs(count=8, seed=4, bases=(3, 4))
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
