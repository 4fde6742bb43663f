"""The C ABI's resource and failure paths on the GPU.

* A memory budget too small for the hierarchy makes fmm_set_levels return
  FMM_ERR_OOM (a budget that fits works, and the context stays usable).
* The caller's allocator (PyTorch's caching allocator in the binding) supplies
  the library's device memory: torch's count of allocated bytes grows by the
  library's workspace and falls back when the context is destroyed.
* Masses given as float32 are widened exactly: the outputs equal those of the
  same values given as float64 (to the rounding of the order of additions).
* A bounded device-side wait that runs out: with the limit set to zero every
  tensor-core CTA gives up at its first pipeline wait that is not already
  complete, latches FMM_ERR_TIMEOUT (returned by fmm_sync), waits for its own
  copies and MMAs in flight and frees its tensor memory.  The context stays
  usable: with the limit restored the next solve matches the oracle.  No GPU
  fault is involved: the wait simply stops early.
"""
import numpy as np
import pytest

import oracle
from paper_2607_19489_b300 import workloads as W
from _parity import ORACLE_MIXED, check

pytestmark = pytest.mark.gpu


def _np(phi, acc):
    import torch
    torch.cuda.synchronize()
    return {l: phi[l].double().cpu().numpy() for l in phi}, {l: acc[l].double().cpu().numpy() for l in acc}


def test_memory_budget_gives_oom_and_a_fitting_budget_works():
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.two_level_plummer(base=5, lo=12, hi=20, seed=3)
    # 1 MiB: less than the workspace (and than the tables, if this context builds them)
    with pytest.raises(fmm.FMMError) as e:
        s = fmm.Solver(4, "fp64", mem_budget=1 << 20)
        s.set_hierarchy(h)
    assert e.value.name == "FMM_ERR_OOM"
    # 64 MiB holds the p = 4 FP64 tables (~31 MB) and this hierarchy's workspace
    s = fmm.Solver(4, "fp64", mem_budget=64 << 20)
    s.set_hierarchy(h)
    phi, acc = s.solve()
    s.sync()
    ref_p, ref_a = oracle.solve(h, 4)
    got_p, got_a = _np(phi, acc)
    check(got_p, got_a, ref_p, ref_a, {"rms": 1e-10, "cell": 1e-9}, "within the budget", h=h)
    big = W.unigrid_plummer(7)   # 128^3: its workspace exceeds 64 MiB
    with pytest.raises(fmm.FMMError) as e:
        s.set_hierarchy(big)
    assert e.value.name == "FMM_ERR_OOM"
    s.set_hierarchy(h)          # the failed call released its workspace: the first hierarchy fits again
    phi, acc = s.solve()
    s.sync()
    got_p, got_a = _np(phi, acc)
    check(got_p, got_a, ref_p, ref_a, {"rms": 1e-10, "cell": 1e-9}, "after an OOM", h=h)
    torch.cuda.synchronize()


def test_torch_caching_allocator_supplies_the_workspace():
    import gc
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.two_level_plummer(base=5, lo=12, hi=20, seed=3)
    torch.cuda.synchronize()
    gc.collect()
    base = torch.cuda.memory_allocated()
    s = fmm.Solver(6, "mixed", allocator="torch")
    s.set_hierarchy(h)
    phi, acc = s.solve()
    s.sync()
    with_ctx = torch.cuda.memory_allocated()
    # the outputs (phi, acc) are torch tensors too; the library's workspace is far larger
    out_bytes = sum(t.numel() * t.element_size() for t in list(phi.values()) + list(acc.values()))
    assert with_ctx - base > out_bytes + (4 << 20)
    got_p, got_a = _np(phi, acc)
    ref_p, ref_a = oracle.solve(h, 6)
    check(got_p, got_a, ref_p, ref_a, ORACLE_MIXED, "torch allocator", h=h)
    del phi, acc
    s.close()
    del s
    gc.collect()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() <= base + (1 << 20)
    # cudaMalloc contexts leave torch's count alone
    c = fmm.Solver(6, "mixed", allocator="cuda")
    c.set_hierarchy(h)
    c.sync()
    assert torch.cuda.memory_allocated() <= base + (1 << 20) + sum(
        np.asarray(m).nbytes + np.asarray(i).nbytes for m, i in zip(h.mass, h.ijk))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_float32_masses_equal_their_float64_values(precision):
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.random_amr(3, 5, seed=13)
    h32 = h.copy()
    h32.mass = [m.astype(np.float32) for m in h.mass]
    h64 = h.copy()
    h64.mass = [m.astype(np.float32).astype(np.float64) for m in h.mass]
    a = fmm.Solver(4, precision, mass_fp32=True)
    a.set_hierarchy(h32)
    pa, aa = _np(*a.solve())
    b = fmm.Solver(4, precision)
    b.set_hierarchy(h64)
    pb, ab = _np(*b.solve())
    a.sync()
    b.sync()
    # same inputs: rounding of the order of additions only (the tensor-core
    # epilogues of the mixed path add with atomics)
    same = {"rms": 1e-14, "cell": 1e-13} if precision == "fp64" else {"rms": 1e-6, "cell": 1e-5}
    check(pa, aa, pb, ab, same, "fp32 masses")
    # mass-only updates in float32 too
    new = [(m * 1.5).astype(np.float32) for m in h.mass]
    a.update_masses([torch.as_tensor(m, device="cuda") for m in new])
    pa2, aa2 = _np(*a.solve())
    a.sync()
    h64.mass = [m.astype(np.float64) for m in new]
    b.set_hierarchy(h64)
    pb2, ab2 = _np(*b.solve())
    b.sync()
    check(pa2, aa2, pb2, ab2, {"rms": 1e-6, "cell": 1e-5}, "fp32 mass update")


def test_bounded_wait_runs_out_and_the_context_recovers():
    import torch
    from paper_2607_19489_b300 import fmm
    h = W.two_level_plummer(base=4, lo=4, hi=12, seed=3)
    s = fmm.Solver(6, "mixed")
    s.set_hierarchy(h)
    s.set_wait_limit(0.0)
    s.solve()
    with pytest.raises(fmm.FMMError) as e:
        s.sync()
    assert e.value.name == "FMM_ERR_TIMEOUT"
    s.set_wait_limit(2.0)
    phi, acc = s.solve()
    s.sync()
    torch.cuda.synchronize()
    got_p, got_a = _np(phi, acc)
    ref_p, ref_a = oracle.solve(h, 6)
    check(got_p, got_a, ref_p, ref_a, ORACLE_MIXED, "after a timeout", h=h)
    with pytest.raises(fmm.FMMError):
        s.set_wait_limit(-1.0)


def test_recycled_memory_from_the_caching_allocator():
    """Memory handed back by PyTorch's caching allocator is not cleared: fill its
    cache with NaN blocks before each growth of the hierarchy; every buffer the
    library reads before writing (the accumulators that are zero between solves)
    must be cleared by the library itself, also when a grown buffer comes back at
    its old address."""
    import torch
    from paper_2607_19489_b300 import fmm
    hs = [W.two_level_plummer(base=3, lo=2, hi=6, seed=2), W.random_amr(3, 5, seed=13),
          W.two_level_plummer(base=4, lo=4, hi=12, seed=3), W.two_level_plummer(base=5, lo=12, hi=20, seed=3)]
    for precision in ("mixed", "fp64"):
        s = fmm.Solver(6, precision)
        for k, h in enumerate(hs):
            junk = [torch.full((n,), float("nan"), device="cuda") for n in (1 << 12, 1 << 15, 1 << 18, 1 << 21, 1 << 23)]
            del junk
            s.set_hierarchy(h)
            for rep in range(2):
                got = _np(*s.solve())
                s.sync()
            ref_p, ref_a = oracle.solve(h, 6)
            tol = {"rms": 1e-10, "cell": 1e-9} if precision == "fp64" else ORACLE_MIXED
            check(*got, ref_p, ref_a, tol, f"recycled memory {precision} hierarchy {k}", h=h)
