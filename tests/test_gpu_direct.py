"""fmm_direct_sum, the exact sum the FMM approximates, against the oracle's
O(N^2) direct sum (FP64, summed in another order: 1e-12 per cell)."""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W
from _parity import check

pytestmark = pytest.mark.gpu
TIGHT = {"rms": 1e-13, "cell": 1e-12}


@pytest.mark.parametrize("name", ["amr", "twolevel", "unigrid32"])
def test_direct_sum_matches_oracle(name):
    import torch
    from paper_2607_19489_b300 import fmm
    h = {"amr": W.random_amr(3, 5, seed=13), "twolevel": W.two_level_plummer(base=4, lo=4, hi=12, seed=3),
         "unigrid32": W.unigrid_plummer(5)}[name]
    s = fmm.Solver(4, "mixed")
    s.set_hierarchy(h)
    sel = {l: np.unique((W.uniform(8, l, np.arange(700)) * h.n(l)).astype(np.int64)) for l in h.levels}
    ref_p, ref_a = oracle.direct(h, sel=sel)
    got_p, got_a = {}, {}
    for l in h.levels:
        p, a = s.direct_sum(l, torch.as_tensor(sel[l], device="cuda"))
        torch.cuda.synchronize()
        got_p[l], got_a[l] = p.cpu().numpy(), a.cpu().numpy()
    check(got_p, got_a, ref_p, ref_a, TIGHT, f"direct sum {name}", h=h, sel=sel)


def test_direct_sum_bad_index_gives_nan():
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.unigrid_plummer(3)
    s = fmm.Solver(4, "fp64")
    s.set_hierarchy(h)
    p, a = s.direct_sum(3, torch.tensor([0, 512, -1, 5], device="cuda"))
    torch.cuda.synchronize()
    p = p.cpu().numpy()
    assert np.isfinite(p[[0, 3]]).all() and np.isnan(p[[1, 2]]).all()
    with pytest.raises(fmm.FMMError):
        s.direct_sum(9, torch.tensor([0], device="cuda"))
