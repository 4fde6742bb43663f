"""The allocation-free unigrid solve against the regular entry points.

fmm_solve_unigrid_static serves callers that cannot call cudaMalloc while
they run (their device memory is owned by another allocator, or they must
not allocate after initialisation): its scratch is a static array inside the
library.  Its results must match fmm_set_levels + fmm_solve on the same grid,
within the parity tolerances of the other GPU tests, on consecutive calls
(the static array keeps the previous call's contents)."""
import numpy as np
import pytest

from paper_2607_19489_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-4}


def rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("level", [3, 4])
def test_static_unigrid_matches_solve(precision, level):
    import torch
    from paper_2607_19489_b300 import fmm
    s = fmm.Solver(4 if level == 3 else 6, precision)
    h = W.permute(W.unigrid_plummer(level, seed=level), seed=7)   # arbitrary input order
    s.set_hierarchy(h)
    phi_ref, acc_ref = s.solve()
    torch.cuda.synchronize()
    s.sync()
    ijk = torch.as_tensor(h.ijk[0], device="cuda")
    mass = torch.as_tensor(h.mass[0], device="cuda")
    for call in range(2):   # two calls in a row share the static scratch
        phi = torch.full((h.n(level),), float("nan"), dtype=torch.float64, device="cuda")
        acc = torch.full((h.n(level), 3), float("nan"), dtype=torch.float64, device="cuda")
        s.solve_unigrid_static(level, ijk, mass, phi, acc)
        torch.cuda.synchronize()
        s.sync()
        assert rel_rms(acc.cpu().numpy(), acc_ref[level].cpu().numpy()) <= TOL[precision], call
        assert rel_rms(phi.cpu().numpy(), phi_ref[level].cpu().numpy()) <= TOL[precision], call
    # the context's own hierarchy is untouched
    phi2, acc2 = s.solve()
    torch.cuda.synchronize()
    assert rel_rms(acc2[level].cpu().numpy(), acc_ref[level].cpu().numpy()) <= TOL[precision]


def test_static_unigrid_rejects_sizes_beyond_the_maximum():
    import torch
    from paper_2607_19489_b300 import fmm
    s = fmm.Solver(4, "fp64")
    h = W.unigrid_plummer(5)
    ijk = torch.as_tensor(h.ijk[0], device="cuda")
    mass = torch.as_tensor(h.mass[0], device="cuda")
    phi = torch.empty(h.n(5), dtype=torch.float64, device="cuda")
    acc = torch.empty(h.n(5), 3, dtype=torch.float64, device="cuda")
    with pytest.raises(fmm.FMMError) as ei:
        s.solve_unigrid_static(5, ijk, mass, phi, acc)
    assert ei.value.name == "FMM_ERR_ARG" and "level must be 2..4" in str(ei.value)
    with pytest.raises(fmm.FMMError) as ei:
        s.solve_unigrid_static(4, ijk[:100], mass[:100], phi, acc)
    assert ei.value.name == "FMM_ERR_ARG"
    s8 = fmm.Solver(8, "fp64")
    h4 = W.unigrid_plummer(4)
    with pytest.raises(fmm.FMMError) as ei:
        s8.solve_unigrid_static(4, torch.as_tensor(h4.ijk[0], device="cuda"),
                                torch.as_tensor(h4.mass[0], device="cuda"), phi[:4096], acc[:4096])
    assert ei.value.name == "FMM_ERR_ARG"
