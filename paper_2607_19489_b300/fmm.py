"""Python binding of libfmm (include/fmm.h): argument marshalling only.

Every step of the solve runs in the CUDA library; this module only passes
pointers, sizes and streams.  PyTorch provides device memory and streams.
If the compiled library is missing the import of `lib()` raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfmm.so")

STATUS = {0: "FMM_OK", -1: "FMM_ERR_ARG", -2: "FMM_ERR_NOT_GRADED", -3: "FMM_ERR_DUPLICATE",
          -4: "FMM_ERR_OUT_OF_BOX", -5: "FMM_ERR_OOM", -6: "FMM_ERR_CUDA", -7: "FMM_ERR_NONFINITE",
          -8: "FMM_ERR_STATE", -9: "FMM_ERR_TIMEOUT", -10: "FMM_ERR_INCOMPLETE"}
PRECISION = {"fp64": 0, "mixed": 1, "bf16x3": 1, "tf32": 2}
BOTTOM = {"m2p": 0, "m2l": 1}

EXPORTED = ["fmm_create", "fmm_set_levels", "fmm_solve", "fmm_sync", "fmm_last_error", "fmm_destroy",
            "fmm_tree_counts", "fmm_tree_export", "fmm_host_numerators", "fmm_host_table",
            "fmm_set_timing", "fmm_set_graphs", "fmm_stage_times", "fmm_stats", "fmm_solve_unigrid_static",
            "fmm_solve_adjoint", "fmm_batch_solve", "fmm_autotune", "fmm_get_tuning",
            "fmm_set_tuning", "fmm_update_masses", "fmm_set_wait_limit", "fmm_direct_sum",
            "fmm_set_velocities", "fmm_set_drift"]


class FMMError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class _Config(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("precision", ctypes.c_int), ("G", ctypes.c_double),
                ("out_fp32", ctypes.c_int), ("mem_budget", ctypes.c_size_t), ("bottom_mode", ctypes.c_int),
                ("p_m", ctypes.c_int), ("mass_fp32", ctypes.c_int), ("fp64_top", ctypes.c_int),
                ("delta_l", ctypes.c_int), ("periodic", ctypes.c_int)]


# fmm_alloc_fn: (user, ptr, bytes, stream) -> ptr
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_shutting_down = False


def _torch_alloc(user, ptr, nbytes, stream):
    """The library's device memory from PyTorch's caching allocator, on the stream of
    the library call that needs it.  Frees after interpreter shutdown has begun are
    skipped (the process is exiting; torch may already be torn down)."""
    try:
        import torch
        if ptr:
            if not _shutting_down:
                torch.cuda.caching_allocator_delete(ptr)
            return None
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
    except Exception:  # out of memory (or no CUDA): the library reports FMM_ERR_OOM
        return None


TORCH_ALLOC = ALLOC_FN(_torch_alloc)   # kept alive for as long as the module is


def _at_exit():
    global _shutting_down
    _shutting_down = True


import atexit  # noqa: E402
atexit.register(_at_exit)

_lib = None


def lib() -> ctypes.CDLL:
    """Load libfmm.so (built by paper_2607_19489_b300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2607_19489_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    L.fmm_create.argtypes = [ctypes.POINTER(_Config), ALLOC_FN, P, ctypes.POINTER(P)]
    L.fmm_set_levels.argtypes = [P, I, I, I, P, P, P, P]
    L.fmm_solve.argtypes = [P, I, P, P, P]
    L.fmm_sync.argtypes = [P]
    L.fmm_last_error.argtypes = [P]
    L.fmm_last_error.restype = ctypes.c_char_p
    L.fmm_destroy.argtypes = [P]
    L.fmm_destroy.restype = None
    L.fmm_tree_counts.argtypes = [P, P]
    L.fmm_tree_export.argtypes = [P, I, P, P, P]
    L.fmm_host_numerators.argtypes = [I, P, P]
    L.fmm_host_table.argtypes = [I, I, P, I64]
    L.fmm_stats.argtypes = [P, P]
    L.fmm_solve_unigrid_static.argtypes = [P, I, I64, P, P, P, P, P]
    L.fmm_set_timing.argtypes = [P, I]
    L.fmm_set_graphs.argtypes = [P, I]
    L.fmm_solve_adjoint.argtypes = [P, I, P, P, P, P]
    L.fmm_batch_solve.argtypes = [P, I, P, P, P, P]
    L.fmm_autotune.argtypes = [P, I, P]
    L.fmm_get_tuning.argtypes = [P, P]
    L.fmm_set_tuning.argtypes = [P, P]
    L.fmm_update_masses.argtypes = [P, I, P, P]
    L.fmm_stage_times.argtypes = [P, P]
    L.fmm_set_wait_limit.argtypes = [P, ctypes.c_double]
    L.fmm_direct_sum.argtypes = [P, I, I64, P, P, P, P]
    L.fmm_set_velocities.argtypes = [P, I, P, P]
    L.fmm_set_drift.argtypes = [P, P, I]
    for name in EXPORTED:
        fn = getattr(L, name)
        if name not in ("fmm_last_error", "fmm_destroy"):
            fn.restype = ctypes.c_int
    _lib = L
    return L


def _ptrs(values):
    arr = (ctypes.c_void_p * max(1, len(values)))()
    for i, v in enumerate(values):
        arr[i] = v
    return arr


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def host_numerators(q: int, u) -> np.ndarray:
    """Integer numerators of d^gamma(1/r) at integer u, |gamma| <= q (host only)."""
    u = np.ascontiguousarray(u, dtype=np.int64)
    n = (q + 1) * (q + 2) * (q + 3) // 6
    out = np.zeros(n, np.int64)
    rc = lib().fmm_host_numerators(q, u.ctypes.data, out.ctypes.data)
    if rc:
        raise FMMError(rc, "fmm_host_numerators")
    return out


_TABLE_SHAPES = {
    0: lambda nc: (256, 26 * 8 * nc), 1: lambda nc: (8 * nc, 26 * 8 * nc), 2: lambda nc: (343, nc, 4),
    3: lambda nc: (64, nc, 4), 4: lambda nc: (8, nc, nc), 5: lambda nc: (8, nc, nc), 6: lambda nc: (nc,),
    7: lambda nc: (8 * nc, 8 * nc), 8: lambda nc: (2048, 26 * 8 * nc), 9: lambda nc: (256, 26 * 64)}
TABLES = {"m2p": 0, "m2l": 1, "near": 2, "l2p": 3, "m2m": 4, "l2l": 5, "lattice_tensor": 6, "lattice": 7,
          "m2p_dl2": 8, "p2p_ring_dl2": 9}


def host_table(p: int, which: str) -> np.ndarray:
    """FP64 translation operator built by the library's host code (no GPU)."""
    nc = (p + 1) * (p + 2) * (p + 3) // 6
    shape = _TABLE_SHAPES[TABLES[which]](nc)
    out = np.zeros(int(np.prod(shape)), np.float64)
    rc = lib().fmm_host_table(p, TABLES[which], out.ctypes.data, out.size)
    if rc:
        raise FMMError(rc, "fmm_host_table")
    return out.reshape(shape)


class Solver:
    """One FMM context (fmm_ctx) on the current CUDA device.

    precision: "fp64", "mixed" (split-BF16 tensor-core translations) or "tf32";
    bottom: "m2p" (the paper's bottom intermediate field) or "m2l" (M2L into the
    parent box + L2P); p_m: multipole order of the translations (None: p);
    mass_fp32: masses are given as float32; fp64_top: mixed precisions keep FP64
    for the top-of-tree M2M and the L2L chain / local-expansion accumulation;
    delta_l: levels between the cells and the finest FMM box, 1 (the paper's) or 2
    (the variant of the footnote of Sec. 2: a 12^3-cell near field; one complete
    level only); periodic: periodic boundaries (Ewald's potential with a
    neutralising background, lmin >= 3); allocator: "torch" (PyTorch's caching allocator supplies the library's device
    memory) or "cuda" (cudaMalloc)."""

    def __init__(self, p: int = 6, precision: str = "mixed", G: float = 1.0, out_fp32: bool = False,
                 mem_budget: int = 0, bottom: str = "m2p", p_m: int | None = None, mass_fp32: bool = False,
                 allocator: str = "torch", fp64_top: bool = False, delta_l: int = 1, periodic: bool = False):
        self.p = p
        self.precision = precision
        self.out_fp32 = out_fp32
        self.mass_fp32 = mass_fp32
        self.bottom = bottom
        self.p_m = p if p_m is None else p_m
        self.delta_l = delta_l
        self.periodic = bool(periodic)
        cfg = _Config(p, PRECISION[precision], float(G), int(out_fp32), int(mem_budget), BOTTOM[bottom],
                      0 if p_m is None else int(p_m), int(mass_fp32), int(fp64_top), int(delta_l), int(periodic))
        if allocator not in ("torch", "cuda"):
            raise ValueError("allocator must be 'torch' or 'cuda'")
        h = ctypes.c_void_p()
        fn = TORCH_ALLOC if allocator == "torch" else ALLOC_FN()
        rc = lib().fmm_create(ctypes.byref(cfg), fn, None, ctypes.byref(h))
        if rc:
            raise FMMError(rc, "fmm_create")
        self._h = h
        self.lmin = self.lmax = None
        self.n = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.fmm_destroy(h)
            self._h = None

    def close(self):
        self.__del__()

    def _check(self, rc, what):
        if rc:
            msg = lib().fmm_last_error(self._h)
            raise FMMError(rc, f"{what}: {msg.decode() if msg else ''}")

    def set_levels(self, lmin: int, lmax: int, ijk, mass, lo: int | None = None, stream=None):
        """ijk[k] int32 [n,3] and mass[k] float64 [n] (float32 when mass_fp32) for levels
        lo..lmax (torch tensors on the device, or numpy arrays on the host)."""
        lo = lmin if lo is None else lo
        n = np.array([int(a.shape[0]) for a in ijk], dtype=np.int64)
        keep = list(ijk) + list(mass)
        pi = _ptrs([_data_ptr(a) for a in ijk])
        pm = _ptrs([_data_ptr(m) for m in mass])
        rc = lib().fmm_set_levels(self._h, lmin, lmax, lo, n.ctypes.data, pi, pm, _stream_ptr(stream))
        del keep
        if rc:
            self.lmin = self.lmax = None
        self._check(rc, "fmm_set_levels")
        self.lmin, self.lmax = lmin, lmax
        for k, l in enumerate(range(lo, lmax + 1)):
            self.n[l] = int(n[k])

    def update_masses(self, mass, lo: int | None = None, stream=None) -> None:
        """New masses for levels lo..lmax (same cells, same order as set_levels)."""
        lo = self.lmin if lo is None else lo
        keep = list(mass)
        pm = _ptrs([_data_ptr(m) for m in mass])
        rc = lib().fmm_update_masses(self._h, lo, pm, _stream_ptr(stream))
        del keep
        self._check(rc, "fmm_update_masses")

    def set_hierarchy(self, h, device="cuda", lo: int | None = None, stream=None):
        import torch
        lo = h.lmin if lo is None else lo
        ks = range(lo - h.lmin, h.lmax - h.lmin + 1)
        mdt = torch.float32 if self.mass_fp32 else torch.float64
        ijk = [torch.as_tensor(h.ijk[k], dtype=torch.int32, device=device).contiguous() for k in ks]
        mass = [torch.as_tensor(h.mass[k], dtype=mdt, device=device).contiguous() for k in ks]
        self.set_levels(h.lmin, h.lmax, ijk, mass, lo=lo, stream=stream)

    def alloc_outputs(self, lo: int | None = None, device="cuda"):
        import torch
        lo = self.lmin if lo is None else lo
        dt = torch.float32 if self.out_fp32 else torch.float64
        phi = {l: torch.empty(self.n[l], dtype=dt, device=device) for l in range(lo, self.lmax + 1)}
        acc = {l: torch.empty(self.n[l], 3, dtype=dt, device=device) for l in range(lo, self.lmax + 1)}
        return phi, acc

    def solve(self, lo: int | None = None, out=None, stream=None):
        """Returns (phi, acc): dicts level -> tensor in the caller's input order."""
        if self.lmin is None:  # no hierarchy yet: let the library report the state error
            empty = _ptrs([])
            self._check(lib().fmm_solve(self._h, 0 if lo is None else lo, empty, empty, _stream_ptr(stream)),
                        "fmm_solve")
        lo = self.lmin if lo is None else lo
        phi, acc = out if out is not None else self.alloc_outputs(lo)
        levels = range(lo, self.lmax + 1)
        pp = _ptrs([_data_ptr(phi[l]) for l in levels])
        pa = _ptrs([_data_ptr(acc[l]) for l in levels])
        rc = lib().fmm_solve(self._h, lo, pp, pa, _stream_ptr(stream))
        self._check(rc, "fmm_solve")
        return phi, acc

    def solve_adjoint(self, g_phi: dict, g_acc: dict, lo: int | None = None, out=None, stream=None):
        """Gradient of <g_phi, phi> + <g_acc, acc> of solve(lo) with respect to the mass of
        every leaf: dict level -> float64 tensor, levels lmin..lmax (FP64 solvers only).
        g_phi / g_acc are dicts level -> tensor for levels lo..lmax, in the output dtype."""
        if self.lmin is None:
            empty = _ptrs([])
            self._check(lib().fmm_solve_adjoint(self._h, 0 if lo is None else lo, empty, empty, empty,
                                                _stream_ptr(stream)), "fmm_solve_adjoint")
        import torch
        lo = self.lmin if lo is None else lo
        levels = range(lo, self.lmax + 1)
        if out is None:
            dev = next(iter(g_phi.values())).device if g_phi else "cuda"
            out = {l: torch.empty(self.n[l], dtype=torch.float64, device=dev) for l in range(self.lmin, self.lmax + 1)}
        keep = [g_phi[l] for l in levels] + [g_acc[l] for l in levels]
        pp = _ptrs([_data_ptr(g_phi[l]) for l in levels])
        pa = _ptrs([_data_ptr(g_acc[l]) for l in levels])
        pm = _ptrs([_data_ptr(out[l]) for l in range(self.lmin, self.lmax + 1)])
        rc = lib().fmm_solve_adjoint(self._h, lo, pp, pa, pm, _stream_ptr(stream))
        del keep
        self._check(rc, "fmm_solve_adjoint")
        return out

    def autotune(self, lo: int | None = None, stream=None) -> dict:
        """Time the candidate launch shapes on the current hierarchy and keep the fastest."""
        lo = self.lmin if lo is None else lo
        self._check(lib().fmm_autotune(self._h, lo, _stream_ptr(stream)), "fmm_autotune")
        return self.tuning()

    def set_tuning(self, t: dict) -> None:
        v = np.array([t["split_m2p"], t["split_m2l"], t["near_octs_per_block"]], np.int32)
        self._check(lib().fmm_set_tuning(self._h, v.ctypes.data), "fmm_set_tuning")

    def tuning(self) -> dict:
        out = np.zeros(3, np.int32)
        self._check(lib().fmm_get_tuning(self._h, out.ctypes.data), "fmm_get_tuning")
        return {"split_m2p": int(out[0]), "split_m2l": int(out[1]), "near_octs_per_block": int(out[2])}

    def sync(self):
        self._check(lib().fmm_sync(self._h), "fmm_sync")

    def set_timing(self, on: bool):
        self._check(lib().fmm_set_timing(self._h, int(on)), "fmm_set_timing")

    def direct_sum(self, level: int, sel=None, stream=None):
        """The exact sum (no FMM) at the given cells of `level` (indices into that level's
        input order; None: all of them): (phi, accel) float64 CUDA tensors."""
        import torch
        if sel is None:
            sel = torch.arange(self.n[level], dtype=torch.int64, device="cuda")
        sel = torch.as_tensor(sel, dtype=torch.int64, device="cuda").contiguous()
        n = int(sel.numel())
        phi = torch.empty(n, dtype=torch.float64, device="cuda")
        acc = torch.empty(n, 3, dtype=torch.float64, device="cuda")
        rc = lib().fmm_direct_sum(self._h, level, n, sel.data_ptr() if n else None, phi.data_ptr() if n else None,
                                  acc.data_ptr() if n else None, _stream_ptr(stream))
        self._check(rc, "fmm_direct_sum")
        return phi, acc

    def set_velocities(self, vel, lo: int | None = None, stream=None) -> None:
        """Velocities [n, 3] (float64) of the leaves of levels lo..lmax, for drifting."""
        lo = self.lmin if lo is None else lo
        keep = [v if hasattr(v, "data_ptr") else np.ascontiguousarray(v, dtype=np.float64) for v in vel]
        pv = _ptrs([_data_ptr(v) for v in keep])
        rc = lib().fmm_set_velocities(self._h, lo, pv, _stream_ptr(stream))
        del keep
        self._check(rc, "fmm_set_velocities")

    def set_drift(self, dt=None) -> None:
        """dt[k]: time since level lmin+k was set (None: drifting off)."""
        if dt is None:
            self._check(lib().fmm_set_drift(self._h, None, 0), "fmm_set_drift")
            return
        d = np.ascontiguousarray(dt, dtype=np.float64)
        self._check(lib().fmm_set_drift(self._h, d.ctypes.data, int(d.size)), "fmm_set_drift")

    def set_wait_limit(self, seconds: float) -> None:
        """Limit of every bounded device-side wait (fmm_set_wait_limit)."""
        self._check(lib().fmm_set_wait_limit(self._h, float(seconds)), "fmm_set_wait_limit")

    def set_graphs(self, on: bool) -> None:
        """Replay solves as CUDA graphs (default) or launch every kernel directly."""
        self._check(lib().fmm_set_graphs(self._h, int(on)), "fmm_set_graphs")

    def stage_times(self):
        out = np.zeros(5)
        self._check(lib().fmm_stage_times(self._h, out.ctypes.data), "fmm_stage_times")
        return dict(zip(["upward", "downward", "m2p", "near_m2p", "near"], out.tolist()))

    def solve_unigrid_static(self, level: int, ijk, mass, phi, accel, stream=None):
        """Unigrid solve (level 2..4) that allocates no device memory; all arguments are
        contiguous CUDA tensors: ijk int32 [n, 3], mass float64 [n], phi [n] and accel
        [n, 3] in the output dtype of this solver (see fmm_solve_unigrid_static in
        include/fmm.h).  Anything else is rejected here, before the library is called."""
        import torch
        n = int(ijk.shape[0]) if hasattr(ijk, "shape") and len(ijk.shape) else -1
        out_dt = torch.float32 if self.out_fp32 else torch.float64
        want = ((ijk, torch.int32, (n, 3)), (mass, torch.float64, (n,)), (phi, out_dt, (n,)),
                (accel, out_dt, (n, 3)))
        for name, (t, dt, shape) in zip(("ijk", "mass", "phi", "accel"), want):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and tuple(t.shape) == shape
                    and t.is_contiguous()):
                raise FMMError(-1, f"solve_unigrid_static: {name} must be a contiguous CUDA tensor of dtype "
                                   f"{dt} and shape {shape}")
        rc = lib().fmm_solve_unigrid_static(self._h, level, int(ijk.shape[0]), _data_ptr(ijk), _data_ptr(mass),
                                            _data_ptr(phi), _data_ptr(accel), _stream_ptr(stream))
        self._check(rc, "fmm_solve_unigrid_static")

    def stats(self):
        out = np.zeros(4, np.int64)
        self._check(lib().fmm_stats(self._h, out.ctypes.data), "fmm_stats")
        return dict(zip(["launches", "cub_calls", "solves", "set_levels"], out.tolist()))

    def tree_counts(self):
        out = np.zeros(self.lmax + 1, np.int64)
        self._check(lib().fmm_tree_counts(self._h, out.ctypes.data), "fmm_tree_counts")
        return out

    def tree_export(self, level: int):
        n_oct = int(self.tree_counts()[level])
        keys = np.zeros(n_oct, np.uint64)
        status = np.zeros(8 * n_oct, np.int64)
        nbr = np.zeros(27 * n_oct, np.int64)
        self._check(lib().fmm_tree_export(self._h, level, keys.ctypes.data, status.ctypes.data,
                                          nbr.ctypes.data), "fmm_tree_export")
        return keys, status, nbr.reshape(-1, 27)


def _data_ptr(a):
    if hasattr(a, "data_ptr"):
        return a.data_ptr() if a.numel() else None
    a = np.asarray(a)
    return a.ctypes.data if a.size else None


def batch_solve(solvers, outs=None, los=None, stream=None):
    """Solve every solver's hierarchy in one CUDA graph launch (fmm_batch_solve).

    outs[i] = (phi, acc) dicts of device tensors as from Solver.alloc_outputs (allocated
    here when omitted); los[i] the first solved level (default lmin).  Returns outs."""
    n = len(solvers)
    los = [s.lmin for s in solvers] if los is None else list(los)
    if outs is None:
        outs = [s.alloc_outputs(lo) for s, lo in zip(solvers, los)]
    keep, pp_rows, pa_rows = [], [], []
    for s, lo, (phi, acc) in zip(solvers, los, outs):
        levels = range(lo, s.lmax + 1)
        pp = _ptrs([_data_ptr(phi[l]) for l in levels])
        pa = _ptrs([_data_ptr(acc[l]) for l in levels])
        keep += [pp, pa]
        pp_rows.append(ctypes.cast(pp, ctypes.c_void_p).value)
        pa_rows.append(ctypes.cast(pa, ctypes.c_void_p).value)
    hs = (ctypes.c_void_p * n)(*[s._h for s in solvers])
    lo_arr = (ctypes.c_int * n)(*los)
    pp_arr = (ctypes.c_void_p * n)(*pp_rows)
    pa_arr = (ctypes.c_void_p * n)(*pa_rows)
    rc = lib().fmm_batch_solve(hs, n, lo_arr, pp_arr, pa_arr, _stream_ptr(stream))
    del keep
    if rc:
        raise FMMError(rc, "fmm_batch_solve: " + (lib().fmm_last_error(solvers[0]._h) or b"").decode())
    return outs
