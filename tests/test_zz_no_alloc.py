"""The allocation-free unigrid solve against the regular entry points.

fmm_solve_unigrid_static serves callers that cannot call cudaMalloc while
they run (their device memory is owned by another allocator, or they must
not allocate after initialisation): its scratch is a static array inside the
library.  Its results must match fmm_set_levels + fmm_solve on the same grid
to near rounding (the same kernels run on the same data; only the order of
the FP32 atomic additions of the mixed path may differ) and the oracle within
the parity bars, on consecutive calls (the static array keeps the previous
call's contents)."""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W
from _parity import check, oracle_tol

pytestmark = pytest.mark.gpu

# same kernels, same data: rounding of the order of atomic additions only
SAME = {"fp64": {"rms": 1e-13, "cell": 1e-12}, "mixed": {"rms": 1e-6, "cell": 1e-5}}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("level", [3, 4])
def test_static_unigrid_matches_solve(precision, level):
    import torch
    from paper_2607_19489_b300 import fmm
    p = 4 if level == 3 else 6
    s = fmm.Solver(p, precision)
    h = W.permute(W.unigrid_plummer(level, seed=level), seed=7)   # arbitrary input order
    s.set_hierarchy(h)
    phi_ref, acc_ref = s.solve()
    torch.cuda.synchronize()
    s.sync()
    reg = ({level: phi_ref[level].cpu().numpy()}, {level: acc_ref[level].cpu().numpy()})
    orc = oracle.solve(h, p)
    ijk = torch.as_tensor(h.ijk[0], device="cuda")
    mass = torch.as_tensor(h.mass[0], device="cuda")
    for call in range(2):   # two calls in a row share the static scratch
        phi = torch.full((h.n(level),), float("nan"), dtype=torch.float64, device="cuda")
        acc = torch.full((h.n(level), 3), float("nan"), dtype=torch.float64, device="cuda")
        s.solve_unigrid_static(level, ijk, mass, phi, acc)
        torch.cuda.synchronize()
        s.sync()
        got = ({level: phi.cpu().numpy()}, {level: acc.cpu().numpy()})
        check(*got, *reg, SAME[precision], f"static call {call} vs fmm_solve", h=h)
        check(*got, *orc, oracle_tol(precision), f"static call {call} vs oracle", h=h)
    # the context's own hierarchy is untouched
    phi2, acc2 = s.solve()
    torch.cuda.synchronize()
    check({level: phi2[level].cpu().numpy()}, {level: acc2[level].cpu().numpy()}, *reg, SAME[precision],
          "fmm_solve after the static calls")


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
        s.solve_unigrid_static(4, ijk[:100], mass[:100], phi[:100], acc[:100])
    assert ei.value.name == "FMM_ERR_ARG"
    s8 = fmm.Solver(8, "fp64")
    h4 = W.unigrid_plummer(4)
    with pytest.raises(fmm.FMMError) as ei:
        s8.solve_unigrid_static(4, torch.as_tensor(h4.ijk[0], device="cuda"),
                                torch.as_tensor(h4.mass[0], device="cuda"), phi[:4096], acc[:4096])
    assert ei.value.name == "FMM_ERR_ARG"


def test_static_unigrid_rejects_host_and_mistyped_arguments():
    """Host arrays, wrong dtypes and short outputs are refused before any launch, by
    the binding and (for host memory) by the library itself."""
    import ctypes
    import torch
    from paper_2607_19489_b300 import fmm
    s = fmm.Solver(4, "fp64")
    h = W.unigrid_plummer(3)
    n = h.n(3)
    ijk = torch.as_tensor(h.ijk[0], device="cuda")
    mass = torch.as_tensor(h.mass[0], device="cuda")
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    acc = torch.empty(n, 3, dtype=torch.float64, device="cuda")
    bad = [(h.ijk[0], mass, phi, acc), (ijk, h.mass[0], phi, acc), (ijk, mass.float(), phi, acc),
           (ijk.long(), mass, phi, acc), (ijk, mass, phi[:-1], acc), (ijk, mass, phi.float(), acc)]
    for args in bad:
        with pytest.raises(fmm.FMMError) as ei:
            s.solve_unigrid_static(3, *args)
        assert ei.value.name == "FMM_ERR_ARG"
    # the C entry point itself refuses host memory
    host_ijk = np.ascontiguousarray(h.ijk[0])
    rc = fmm.lib().fmm_solve_unigrid_static(s._h, 3, n, host_ijk.ctypes.data, mass.data_ptr(), phi.data_ptr(),
                                            acc.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == -1 and b"device pointers" in fmm.lib().fmm_last_error(s._h)
    del ctypes
