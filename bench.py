#!/usr/bin/env python
"""Benchmark of the adaptive FMM Poisson solver on one B300 per rank.

Metric: cell-updates/s per Poisson solve (leaf cells whose phi and accel are
produced, divided by the device time of one solve), for the mixed-precision
path (split-BF16 tcgen05 M2L/M2P, FP32 P2P) with the FP64 GPU path timed
beside it at the same workload, and the relative RMS acceleration error of
the mixed path against the FP64 path reported with it.

Workload: two-level isolated AMR hierarchy, 64^3 base plus a 32^3 refined
block over the central 16^3 coarse cells, Plummer density (scale 0.05 of the
box) with seeded lognormal noise (sigma 0.3), expansion order p = 6.  Inputs
are synthetic and seeded.

One step = fmm_set_levels (tree build over all levels) + fmm_solve (upward,
downward, M2P, near field, scatter), i.e. every step of the hot path, on
inputs resident in HBM.  The inputs are far smaller than L2, so L2 is flushed
(256 MB write) before each timed step, outside its event pair.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 (torchrun) every rank solves its own copy of the hierarchy on its
own GPU (independent problems, weak scaling); the only collectives are the
barrier and the max of the step time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per Poisson solve, mixed vs FP64 GPU FMM, at <=1e-4 rel force error"
UNIT = "cell-updates/s"
P_ORDER = 6
WORKLOAD = "two-level AMR 64^3 + 32^3 refined block, Plummer a=0.05 + lognormal sigma=0.3, isolated, p=6"
# Peaks measured on the B300s (copy bandwidth; cuBLAS bf16 dense burst and sustained);
# MEASURED_PEAKS.json, when present, takes precedence.
RECORDED_PEAKS = {"hbm_gbs": 6513.0, "bf16_tflops": 1786.0, "bf16_tflops_sustained": 1405.0}
NC = (P_ORDER + 1) * (P_ORDER + 2) * (P_ORDER + 3) // 6
# DRAM bytes (read + write) of the stage-timed M2P launch (k_gemm_tc, in-order
# solve, split-K from the built-in heuristic) of the headline workload, from one
# ncu capture of that launch shape; None until captured for the current kernel.
M2P_TRAFFIC_BYTES = 37023488
# FP32 work per P2P interaction, the usual count for a softened-free gravity
# pair (3 differences, r^2, rsqrt ~4, m/r, m/r^3, 4 accumulations)
FLOP_PER_PAIR = 20


# FP32 / FP64 / MUFU throughput of the B300s, probed once with
# register-only FFMA, DFMA and rsqrt chains over 148 x 8 blocks of 256 threads
# (CUDA events, best of 5); MEASURED_PEAKS.json carries no FP32 figure.
PROBED_PEAKS = {"ffma_tflops": 71.6, "dfma_tflops": 1.18, "rsqrt_tops": 4.69,
                "note": "probed FP32 FFMA peak (register-only FFMA chains, 148 x 8 x 256 threads, CUDA events)"}


def load_peaks():
    for path in (os.path.join(ROOT, "MEASURED_PEAKS.json"),):
        if os.path.exists(path):
            with open(path) as f:
                d = json.load(f)
            out = dict(RECORDED_PEAKS)
            for k in out:
                for kk, v in d.items():
                    if kk == k or kk.endswith(k):
                        try:
                            out[k] = float(v)
                        except (TypeError, ValueError):
                            pass
            return out, "measured (MEASURED_PEAKS.json)"
    return dict(RECORDED_PEAKS), "measured (recorded values for this pool)"


# ---------------------------------------------------------------------------- ranks

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(value: float, dist, device) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------- GPU arm

WORKLOADS = {
    "two_level": WORKLOAD,
    "unigrid16": "unigrid 16^3 Plummer a=0.1, p=6 (a small case for checking the launch paths)",
}


def make_workload(name: str = "two_level"):
    from paper_2607_19489_b300 import workloads as W
    return W.two_level_plummer() if name == "two_level" else W.unigrid_plummer(4)


# ---------------------------------------------------------------------------- work counts

_OFF6 = np.array([[x, y, z] for z in range(-2, 4) for y in range(-2, 4) for x in range(-2, 4)], np.int64)


def _keys(c, level):
    c = np.asarray(c, np.int64)
    return c[..., 0] + (c[..., 1] << level) + (c[..., 2] << (2 * level))


class _CellSet:
    """Membership of level-l cell keys: a dense bitmap up to level 8, else a sorted array."""

    def __init__(self, keys, level):
        self.dense = level <= 8
        if self.dense:
            self.map = np.zeros(1 << (3 * level), bool)
            self.map[keys] = True
        else:
            self.keys = np.sort(keys)

    def test(self, q):
        """q: keys, -1 where invalid."""
        if self.dense:
            return self.map[np.maximum(q, 0)] & (q >= 0)
        if self.keys.size == 0:
            return np.zeros(q.shape, bool)
        i = np.searchsorted(self.keys, q).clip(0, self.keys.size - 1)
        return self.keys[i] == q


def _member(cells, q):
    return cells.test(q)


def work_counts(h, chunk: int = 8192) -> dict:
    """The method's own interaction counts for the leaf targets of a hierarchy
    (Fig. 2): M2P (source box, target) pairs of the bottom intermediate field, P2P
    pairs (level-l leaves of the 3^3 neighbour octs, coarse leaves once each, and
    the coarse leaves of the interaction list), nearest-field children, and
    near-field M2P pairs.  Bookkeeping for the roofline, on the host."""
    lv = list(h.levels)
    leaves, refined = {}, {}
    for k, l in enumerate(lv):
        leaves[l] = np.sort(_keys(h.ijk[k], l))
    cells_next = None
    for l in range(h.lmax, 0, -1):  # refined cells: parents of the next level's cells
        if cells_next is None:
            refined[l] = np.zeros(0, np.int64)
        else:
            refined[l] = np.unique(_keys(cells_next >> 1, l))
        k = l - h.lmin
        mine = h.ijk[k].astype(np.int64) if 0 <= k < len(lv) else np.zeros((0, 3), np.int64)
        ref_cells = np.stack([refined[l] & ((1 << l) - 1), (refined[l] >> l) & ((1 << l) - 1),
                              refined[l] >> (2 * l)], 1) if refined[l].size else np.zeros((0, 3), np.int64)
        cells_next = np.concatenate([mine, ref_cells]) if (mine.size or ref_cells.size) else None
    for l in range(0, h.lmin):
        leaves[l] = np.zeros(0, np.int64)
    # octs (keyed by their parent cell) holding a refined cell, per level
    m2p_rows = {l: np.unique(np.stack([v & ((1 << l) - 1), (v >> l) & ((1 << l) - 1), v >> (2 * l)], 1) >> 1,
                             axis=0).shape[0] if v.size else 0 for l, v in refined.items()}
    leaves = {l: _CellSet(v, l) for l, v in leaves.items()}
    refined = {l: _CellSet(v, l) for l, v in refined.items()}
    empty = _CellSet(np.zeros(0, np.int64), 0)
    out = {"targets": 0, "m2p_pairs": 0, "p2p_pairs": 0, "nearest_pairs": 0, "near_m2p_pairs": 0,
           "m2p_rows": m2p_rows}
    child = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], np.int64)
    for k, l in enumerate(lv):
        T = h.ijk[k].astype(np.int64)
        out["targets"] += T.shape[0]
        n_up = 1 << (l - 1)
        # everything but the self term and the touching test depends on the parent
        # box F only: count per F, weighted by its number of targets
        fk, inv, n_t = np.unique(_keys(T >> 1, l - 1), return_inverse=True, return_counts=True)
        Fs = np.stack([fk & (n_up - 1), (fk >> (l - 1)) & (n_up - 1), fk >> (2 * (l - 1))], 1)
        tmask = np.zeros((fk.size, 8), bool)  # which children of F are targets
        tmask[inv.reshape(-1), (T[:, 0] & 1) | ((T[:, 1] & 1) << 1) | ((T[:, 2] & 1) << 2)] = True
        for i0 in range(0, fk.size, chunk):
            F = Fs[i0:i0 + chunk]
            nt = n_t[i0:i0 + chunk]
            # bottom intermediate field: interaction list of F at level l-1
            S = 2 * (F >> 1)[:, None, :] + _OFF6[None]
            ok = ((S >= 0) & (S < n_up)).all(-1) & (np.abs(S - F[:, None, :]).max(-1) > 1)
            sk = np.where(ok, _keys(np.clip(S, 0, n_up - 1), l - 1), -1)
            out["m2p_pairs"] += int((nt * _member(refined[l - 1], sk).sum(1)).sum())
            out["p2p_pairs"] += int((nt * _member(leaves.get(l - 1, empty), sk).sum(1)).sum())
            # near field: the level-l positions of F's 3^3 neighbour octs
            P = 2 * F[:, None, :] + _OFF6[None]
            inb = ((P >= 0) & (P < (1 << l))).all(-1)
            pk = np.where(inb, _keys(np.clip(P, 0, (1 << l) - 1), l), -1)
            n_leaf = _member(leaves[l], pk).sum(1)
            nk = np.where(inb, _keys(np.clip(P >> 1, 0, n_up - 1), l - 1), -1)
            n_coarse = _member(leaves.get(l - 1, empty), nk).sum(1) // 8
            out["p2p_pairs"] += int((nt * (n_leaf - 1 + n_coarse)).sum())  # every target skips itself
            is_ref = _member(refined[l], pk)
            iface = np.where(is_ref.any(1))[0]
            if iface.size:  # touching refined cells: nearest field; the others: near-field M2P
                t = 2 * F[iface][:, None, :] + child[None]                      # [f, 8, 3]
                touch = np.abs(P[iface][:, None, :, :] - t[:, :, None, :]).max(-1) <= 1  # [f, 8, 216]
                rt = (touch & is_ref[iface][:, None, :]).sum(-1)                 # [f, 8]
                tm = tmask[i0:i0 + chunk][iface]
                out["nearest_pairs"] += 8 * int((rt * tm).sum())
                out["near_m2p_pairs"] += int(((is_ref[iface].sum(1)[:, None] - rt) * tm).sum())
    return out


def rel_rms(a: dict, b: dict) -> float:
    num = sum(float(((a[l] - b[l]) ** 2).sum()) for l in b)
    den = sum(float((b[l] ** 2).sum()) for l in b)
    return float(np.sqrt(num / den))


def host_warm(seconds: float = 1.0):
    """Keeps the calling host core busy for a moment before a timed region.

    Every step has host work between its device stages (the tree build's one
    synchronisation, the solve's graph launch).  On the test machines a host
    core that has idled, even for 0.1 s, runs that work several times slower
    for the next few hundred milliseconds (the graph launch measured 0.08 ms
    instead of 0.011 ms, the step 0.55 ms instead of 0.34 ms), and a busy-wait
    of about a second restores it; steps in a steady loop never see it.  The
    spin touches no GPU state."""
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        pass


def timed_steps(torch, step, K, W, stream, flush):
    for _ in range(W):
        step()
    torch.cuda.synchronize()
    host_warm()
    times = []
    for _ in range(K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    return times


def timed_after(torch, prepare, step, K, W, stream, flush):
    """As timed_steps, with prepare() run before each step outside its event pair."""
    for _ in range(W):
        prepare()
        step()
    torch.cuda.synchronize()
    host_warm()
    times = []
    for _ in range(K):
        flush.zero_()
        prepare()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    return times


def gpu_arm(args, rank, world, local):
    import torch
    from paper_2607_19489_b300 import fmm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, "nccl")
    stream = torch.cuda.current_stream()
    h = make_workload(args.workload)
    n_cells = h.n_cells
    ijk = [torch.as_tensor(a, device=dev).contiguous() for a in h.ijk]
    mass = [torch.as_tensor(m, device=dev).contiguous() for m in h.mass]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def make(precision, **kw):
        s = fmm.Solver(P_ORDER, precision, **kw)
        s.set_levels(h.lmin, h.lmax, ijk, mass)
        out = s.alloc_outputs()
        return s, out

    mixed, out_m = make("mixed")
    fp64, out_d = make("fp64") if not args.quick else (None, None)

    def step_mixed():
        mixed.set_levels(h.lmin, h.lmax, ijk, mass)
        mixed.solve(out=out_m)

    def step_mixed_solve_only():
        mixed.solve(out=out_m)

    def step_fp64():
        fp64.set_levels(h.lmin, h.lmax, ijk, mass)
        fp64.solve(out=out_d)

    # accuracy of the mixed path against the FP64 GPU path (which matches the oracle to 1e-10)
    err_acc = err_phi = None
    if fp64 is not None:
        step_mixed()
        step_fp64()
        torch.cuda.synchronize()
        mixed.sync()
        fp64.sync()
        am = {l: out_m[1][l].cpu().numpy() for l in h.levels}
        ad = {l: out_d[1][l].cpu().numpy() for l in h.levels}
        pm = {l: out_m[0][l].cpu().numpy() for l in h.levels}
        pd = {l: out_d[0][l].cpu().numpy() for l in h.levels}
        err_acc = rel_rms(am, ad)
        err_phi = rel_rms(pm, pd)

    barrier(dist)
    launches0 = mixed.stats()["launches"]
    with ClockSampler(local) as clk:
        t_mixed = timed_steps(torch, step_mixed, args.steps, args.warmup, stream, flush)
    launches1 = mixed.stats()["launches"]
    clocks = clk.summary()
    # solve only: the hierarchy is set (outside the event pair) before every timed
    # solve, so the solve recomputes every stage (an unchanged hierarchy would let
    # it skip the upward pass)
    t_solve = timed_after(torch, lambda: mixed.update_masses(mass), step_mixed_solve_only,
                          args.steps, 3, stream, flush)
    k64 = max(3, min(args.steps, 5))
    t_fp64 = timed_steps(torch, step_fp64, k64, 3, stream, flush) if fp64 is not None else [float("nan")]
    mixed.sync()
    if fp64 is not None:
        fp64.sync()
    # the option that keeps FP64 for the top-of-tree M2M and the L2L chain /
    # local-expansion accumulation: same step, its time and accuracy
    top64 = None
    if fp64 is not None:
        m64, out_t = make("mixed", fp64_top=True)

        def step_top64():
            m64.set_levels(h.lmin, h.lmax, ijk, mass)
            m64.solve(out=out_t)

        t_top = timed_steps(torch, step_top64, min(args.steps, 50), args.warmup, stream, flush)
        m64.sync()
        at = {l: out_t[1][l].cpu().numpy() for l in h.levels}
        top64 = {"ms_per_step": statistics.mean(t_top), "value": world * n_cells / (statistics.mean(t_top) * 1e-3),
                 "rel_rms_accel_vs_fp64": rel_rms(at, ad),
                 "what": "config.fp64_top: FP64 M2M at box levels <= 3 and FP64 L2L / local-expansion accumulation"}
        del m64
    barrier(dist)

    ms_mixed = reduce_max(statistics.mean(t_mixed), dist, dev)
    ms_solve = reduce_max(statistics.mean(t_solve), dist, dev)
    ms_fp64 = reduce_max(statistics.mean(t_fp64), dist, dev)
    value = world * n_cells / (ms_mixed * 1e-3)
    value_fp64 = world * n_cells / (ms_fp64 * 1e-3)

    # per-stage device times of the solve (events inside the library, on this stream)
    mixed.set_timing(True)
    stage = {k: 0.0 for k in ("upward", "downward", "m2p", "near_m2p", "near")}
    reps = max(3, args.steps)
    for _ in range(reps):
        flush.zero_()
        mixed.update_masses(mass)
        mixed.solve(out=out_m)
        mixed.sync()
        for k, v in mixed.stage_times().items():
            stage[k] += v / reps
    mixed.set_timing(False)

    # end to end through the C ABI with pinned host buffers: H2D of inputs, D2H of outputs
    h_ijk = [torch.as_tensor(a).pin_memory() for a in h.ijk]
    h_mass = [torch.as_tensor(m).pin_memory() for m in h.mass]
    h_phi = {l: torch.empty(h.n(l), dtype=torch.float64).pin_memory() for l in h.levels}
    h_acc = {l: torch.empty(h.n(l), 3, dtype=torch.float64).pin_memory() for l in h.levels}
    e2e_solver = fmm.Solver(P_ORDER, "mixed")
    np_ijk = [t.numpy() for t in h_ijk]
    np_mass = [t.numpy() for t in h_mass]
    np_out = ({l: h_phi[l].numpy() for l in h.levels}, {l: h_acc[l].numpy() for l in h.levels})

    def step_e2e():
        e2e_solver.set_levels(h.lmin, h.lmax, np_ijk, np_mass)
        e2e_solver.solve(out=np_out)

    t_e2e = timed_steps(torch, step_e2e, args.steps if not args.quick else 3, 3, stream, flush)
    e2e_solver.sync()
    ms_e2e = reduce_max(statistics.mean(t_e2e), dist, dev)
    h2d = sum(a.nbytes for a in np_ijk) + sum(m.nbytes for m in np_mass)
    d2h = sum(v.nbytes for v in np_out[0].values()) + sum(v.nbytes for v in np_out[1].values())

    peaks, peak_src = load_peaks()
    roofline, kernels = rooflines(h, stage, peaks, peak_src)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3+f32+f64", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOADS[args.workload], "cells": n_cells, "levels": [h.n(l) for l in h.levels], "p": P_ORDER,
                   "step": "fmm_set_levels (tree build) + fmm_solve", "l2": "flushed (256 MB write) before each step",
                   "parallelism": f"replicas x{world} (independent hierarchies)"},
        "fp64_gpu": {"value": value_fp64, "ms_per_step": ms_fp64, "speedup_mixed_over_fp64": value / value_fp64},
        "mixed_fp64_top": top64,
        "accuracy": {"rel_rms_accel_mixed_vs_fp64": err_acc, "rel_rms_phi_mixed_vs_fp64": err_phi,
                     "bar": 1e-4},
        "solve_only": {"value": world * n_cells / (ms_solve * 1e-3), "ms": ms_solve},
        "stages_ms": stage,
        "e2e": {"value": world * n_cells / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
        "gpu_launches": int(launches1 - launches0),
        "roofline": roofline,
        "kernels": kernels,
        "clocks": clocks,
    }
    del mixed, fp64, e2e_solver
    # the extra workloads characterise one GPU: a multi-rank run reports the headline only
    legs = [x for x in args.legs.split(",") if x and x != "none"] if not args.quick and world == 1 else []
    for name in legs:
        fn = {"batched": leg_batched, "adjoint": leg_adjoint, "ats": leg_ats, "sweep": leg_sweep,
              "binary": leg_binary, "delta_l": leg_delta_l, "periodic": leg_periodic}.get(name)
        if fn is None:
            continue
        try:
            line[name] = fn(args, torch, dev, stream, flush)
        except Exception as e:  # an extra workload never hides the headline
            line[name] = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu_baseline and not args.quick:
        line["cpu_baseline"] = cpu_baseline(h, per_level=args.cpu_sample)
    if rank == 0:
        print(json.dumps(line))
    barrier(dist)


def rooflines(h, stage, peaks, peak_src):
    """Roofline of the dominant kernel (the bottom M2P contraction) and of the
    other stages, from the method's own work on this hierarchy (work_counts) and
    the per-stage CUDA-event times of an in-order solve."""
    w = work_counts(h)
    kq = 8 * NC
    # M2P row tiles: per target level l, 128-row tiles over the octs of level l-1
    # holding a refined cell
    issued_mac = sum(-(-w["m2p_rows"][l - 1] // 128) * 128 for l in h.levels if h.n(l)) * 26 * kq * 256 * 3
    useful = 2.0 * 4 * NC * w["m2p_pairs"]
    t = stage["m2p"] * 1e-3
    peak = peaks["bf16_tflops"] / 3.0
    roof = {
        "kernel": "k_gemm_tc (bottom M2P, split-BF16 x3 on tcgen05)",
        "bound": "tensor",
        "achieved": useful / t / 1e12,
        "peak": peak,
        "unit": "TFLOP/s",
        "frac": useful / t / 1e12 / peak,
        "traffic": M2P_TRAFFIC_BYTES,
        "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of the stage-timed M2P launch of this "
                        "workload, one ncu capture (null until captured for this kernel); algorithmic: the "
                        "operator hi+lo (17.9 MB), the gathered multipole rows and the accumulator",
        "peak_note": f"{peak_src} bf16 dense burst / 3 (three bf16 products per split-BF16 product; the kernel is "
                     "timed alone by stage events); useful flops = 2 * 4 * ncoef per (source box, target) pair "
                     f"of the method, {w['m2p_pairs']} pairs = {w['m2p_pairs'] / w['targets']:.1f} sources per target",
        "issued_bf16_tflops": 2.0 * issued_mac / t / 1e12,
        "issued_note": "MACs the contraction issues: 128-row tiles x 26 offsets x 8 ncoef x 256 columns x 3 "
                       "products (dense blocks, zero near-neighbour blocks included)",
        "stage_ms": stage["m2p"],
    }
    kern = {"work": w, "flop_per_pair": FLOP_PER_PAIR}
    fp32 = PROBED_PEAKS["ffma_tflops"]
    p2p = w["p2p_pairs"] + w["nearest_pairs"]
    if stage.get("near"):
        fl = FLOP_PER_PAIR * p2p + 2.0 * 4 * NC * w["targets"]   # P2P + nearest + L2P
        kern["near"] = {"kernel": "k_near (P2P, nearest field, L2P, scatter)", "bound": "fp32",
                        "achieved_tflops": fl / (stage["near"] * 1e-3) / 1e12, "peak_tflops": fp32,
                        "frac": fl / (stage["near"] * 1e-3) / 1e12 / fp32, "ms": stage["near"],
                        "peak_note": PROBED_PEAKS["note"]}
    if stage.get("near_m2p"):
        fl = 2.0 * 4 * NC * w["near_m2p_pairs"]
        kern["near_m2p"] = {"kernel": "k_near_m2p", "bound": "fp32", "achieved_tflops": fl / (stage["near_m2p"] * 1e-3) / 1e12,
                            "peak_tflops": fp32, "frac": fl / (stage["near_m2p"] * 1e-3) / 1e12 / fp32,
                            "ms": stage["near_m2p"]}
    if stage.get("upward"):
        # algorithmic bytes of P2M + M2M: each leaf mass read once (8 B), each cell's
        # total mass written (4 B), each refined cell's multipole row written once in
        # FP32 + bf16 hi + lo (8 B per coefficient) and read once by its parent (4 B)
        n_leaf = sum(h.n(l) for l in h.levels)
        n_ref = sum(np.unique(_keys(h.ijk[k].astype(np.int64) >> 1, l - 1)).size for k, l in enumerate(h.levels))
        nbytes = 12 * n_leaf + 4 * n_ref + 12 * NC * n_ref
        kern["upward"] = {"kernels": "k_leaf_mono, k_leaf_rows, k_m2m, k_m2m_block", "bound": "hbm",
                          "algorithmic_bytes": nbytes, "achieved_gbs": nbytes / (stage["upward"] * 1e-3) / 1e9,
                          "peak_gbs": peaks["hbm_gbs"], "frac": nbytes / (stage["upward"] * 1e-3) / 1e9 / peaks["hbm_gbs"],
                          "ms": stage["upward"]}
    return roof, kern


def profile_solves(args):
    """In-order, stage-timed solves of the headline hierarchy, for ncu: each solve
    launches k_gemm_tc twice (M2L of every box level, then the bottom M2P)."""
    import torch
    from paper_2607_19489_b300 import fmm
    h = make_workload(args.workload)
    s = fmm.Solver(P_ORDER, "mixed")
    s.set_hierarchy(h)
    out = s.alloc_outputs()
    s.set_timing(True)
    for _ in range(args.profile_solves):
        s.update_masses([torch.as_tensor(m, device="cuda") for m in h.mass])
        s.solve(out=out)
        s.sync()
    torch.cuda.synchronize()
    print(json.dumps({"profile_solves": args.profile_solves, "stages_ms": s.stage_times()}))


# ---------------------------------------------------------------------------- extra workloads

def _timed(torch, fn, K, W, stream):
    for _ in range(W):
        fn()
    torch.cuda.synchronize()
    host_warm()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / K


def leg_sweep(args, torch, dev, stream, flush):
    """Speed against accuracy (a Pareto table): the bottom intermediate field (M2P
    as in the paper, or M2L into the parent box + L2P), the orders (p_m, p) = (2, 3)
    (the paper's quadrupoles), (4, 4), (6, 6), (8, 8), and the precision (FP64,
    split-BF16, TF32), on the 32^3 Plummer unigrid and the two-level 64^3 + 32^3
    hierarchy.  Each entry: cell-updates/s of fmm_set_levels + fmm_solve, and the
    relative RMS error against the exact sum (fmm_direct_sum, FP64) on all cells
    (32^3) or 4096 seeded cells per level (64^3 + 32^3)."""
    from paper_2607_19489_b300 import fmm, workloads as W
    cfgs = [("unigrid 32^3 Plummer a=0.1, 1% noise", W.unigrid_plummer(5), None),
            ("two-level 64^3 + 32^3 Plummer a=0.05, lognormal 0.3", W.two_level_plummer(), 4096)]
    orders = [(3, 2), (4, 4), (6, 6), (8, 8)]
    keep = {}   # one context per (p, p_m, precision) keeps its shared tables alive
    rows = []
    t0 = time.perf_counter()
    for cname, h, nsample in cfgs:
        ijk = [torch.as_tensor(a, device=dev).contiguous() for a in h.ijk]
        mass = [torch.as_tensor(m, device=dev).contiguous() for m in h.mass]
        ref = fmm.Solver(4, "fp64")
        ref.set_levels(h.lmin, h.lmax, ijk, mass)
        sel = {l: (torch.arange(h.n(l), device=dev) if nsample is None else
                   torch.as_tensor(np.unique((W.uniform(61, l, np.arange(nsample)) * h.n(l)).astype(np.int64)),
                                   device=dev)) for l in h.levels}
        direct = {l: ref.direct_sum(l, sel[l]) for l in h.levels}
        ref.sync()
        fp64_out = {}
        for p, pm in orders:
            for prec in ("fp64", "mixed", "tf32"):
                for bottom in ("m2p", "m2l"):
                    s = fmm.Solver(p, prec, p_m=pm, bottom=bottom)
                    keep.setdefault((p, pm, prec), s)
                    s.set_levels(h.lmin, h.lmax, ijk, mass)
                    out = s.alloc_outputs(device=dev)

                    def step():
                        s.set_levels(h.lmin, h.lmax, ijk, mass)
                        s.solve(out=out)

                    K = 2 if prec == "fp64" else 10
                    ms = _timed(torch, step, K, 2, stream)
                    s.sync()
                    num_a = den_a = num_p = den_p = 0.0
                    for l in h.levels:
                        ga = out[1][l][sel[l]].double()
                        gp = out[0][l][sel[l]].double()
                        num_a += float(((ga - direct[l][1]) ** 2).sum())
                        den_a += float((direct[l][1] ** 2).sum())
                        num_p += float(((gp - direct[l][0]) ** 2).sum())
                        den_p += float((direct[l][0] ** 2).sum())
                    got = {l: out[1][l][sel[l]].double() for l in h.levels}
                    if prec == "fp64":
                        fp64_out[(p, pm, bottom)] = got
                    ref64 = fp64_out.get((p, pm, bottom))
                    vs64 = None
                    if ref64 is not None and prec != "fp64":
                        vs64 = float(np.sqrt(sum(float(((got[l] - ref64[l]) ** 2).sum()) for l in h.levels) /
                                             sum(float((ref64[l] ** 2).sum()) for l in h.levels)))
                    rows.append({"config": cname, "p": p, "p_m": pm, "bottom": bottom, "precision": prec,
                                 "cells": h.n_cells, "ms": ms, "value": h.n_cells / (ms * 1e-3),
                                 "rel_rms_accel_vs_direct": float(np.sqrt(num_a / den_a)),
                                 "rel_rms_phi_vs_direct": float(np.sqrt(num_p / den_p)),
                                 "rel_rms_accel_vs_fp64": vs64})
                    del s, out
        del ref
    del keep
    return {"unit": UNIT, "step": "fmm_set_levels + fmm_solve (inputs resident)", "runs": rows,
            "reference": "fmm_direct_sum (FP64 exact sum) on the listed cells", "wall_s": time.perf_counter() - t0}


def leg_delta_l(args, torch, dev, stream, flush):
    """Delta l = 1 (the paper's) against Delta l = 2 (the footnote of Sec. 2,
    which Paper I tested on unigrids: a 12^3-cell near field, M2P one box level
    up, M2L one level shorter) on the Plummer unigrids 32^3, 64^3 and 128^3, at
    p = 4 and 6 in FP64, split-BF16 and TF32.  Each entry: cell-updates/s of
    fmm_set_levels + fmm_solve, the in-order stage times of one solve, and the
    relative RMS error against the exact sum (fmm_direct_sum, FP64) on 4096
    seeded cells.  One context per (p, precision, Delta l) serves every grid."""
    from paper_2607_19489_b300 import fmm, workloads as W
    t0 = time.perf_counter()
    grids = []
    for level in (5, 6, 7):
        h = W.unigrid_plummer(level)
        ijk = [torch.as_tensor(a, device=dev).contiguous() for a in h.ijk]
        mass = [torch.as_tensor(m, device=dev).contiguous() for m in h.mass]
        l = h.lmin
        sel = torch.as_tensor(np.unique((W.uniform(67, l, np.arange(4096)) * h.n(l)).astype(np.int64)), device=dev)
        ref = fmm.Solver(4, "fp64")
        ref.set_levels(l, l, ijk, mass)
        d_phi, d_acc = ref.direct_sum(l, sel)
        ref.sync()
        del ref
        grids.append((level, h, ijk, mass, sel, d_phi, d_acc))
    rows = []
    for p in (4, 6):
        for prec in ("fp64", "mixed", "tf32"):
            for dl in (1, 2):
                s = fmm.Solver(p, prec, delta_l=dl)
                for level, h, ijk, mass, sel, d_phi, d_acc in grids:
                    if prec == "fp64" and level == 7:
                        continue  # seconds per solve; the two smaller grids carry the FP64 comparison
                    l = h.lmin
                    s.set_levels(l, l, ijk, mass)
                    out = s.alloc_outputs(device=dev)

                    def step():
                        s.set_levels(l, l, ijk, mass)
                        s.solve(out=out)

                    K = 2 if prec == "fp64" else 10
                    ms = _timed(torch, step, K, 3, stream)
                    s.sync()
                    ga = out[1][l][sel].double()
                    gp = out[0][l][sel].double()
                    s.set_timing(True)
                    s.update_masses(mass)
                    s.solve(out=out)
                    s.sync()
                    st = s.stage_times()
                    s.set_timing(False)
                    rows.append({"grid": f"{2 ** level}^3", "p": p, "precision": prec, "delta_l": dl,
                                 "cells": h.n_cells, "ms": ms, "value": h.n_cells / (ms * 1e-3),
                                 "stages_ms": st,
                                 "rel_rms_accel_vs_direct": float(((ga - d_acc) ** 2).sum().sqrt() /
                                                                  (d_acc ** 2).sum().sqrt()),
                                 "rel_rms_phi_vs_direct": float(((gp - d_phi) ** 2).sum().sqrt() /
                                                                (d_phi ** 2).sum().sqrt())})
                    del out
                del s
    rows.sort(key=lambda r: (r["grid"], r["p"], ["fp64", "mixed", "tf32"].index(r["precision"]), r["delta_l"]))
    return {"unit": UNIT, "step": "fmm_set_levels + fmm_solve (inputs resident)", "runs": rows,
            "workload": "Plummer unigrids (a = 0.1, 1% noise)",
            "reference": "fmm_direct_sum (FP64 exact sum) on 4096 seeded cells", "wall_s": time.perf_counter() - t0}


def leg_periodic(args, torch, dev, stream, flush):
    """Periodic boundaries (the extension Sec. 6 names for cosmology): the
    headline two-level 64^3 + 32^3 hierarchy and the 64^3 Plummer unigrid with
    the box tiled by images and a neutralising background, p = 6, split-BF16 and
    FP64.  Each entry: cell-updates/s of fmm_set_levels + fmm_solve, the
    in-order stage times, and the mixed path's error against the FP64 GPU path
    (relative RMS of accel; phi against max(RMS, G M_total), the periodic
    field's scale)."""
    from paper_2607_19489_b300 import fmm, workloads as W
    rows = []
    t0 = time.perf_counter()
    for cname, h in (("two-level 64^3 + 32^3 Plummer a=0.05, lognormal 0.3", W.two_level_plummer()),
                     ("unigrid 64^3 Plummer a=0.1, 1% noise", W.unigrid_plummer(6))):
        ijk = [torch.as_tensor(a, device=dev).contiguous() for a in h.ijk]
        mass = [torch.as_tensor(m, device=dev).contiguous() for m in h.mass]
        outs = {}
        for prec in ("fp64", "mixed"):
            s = fmm.Solver(P_ORDER, prec, periodic=True)
            s.set_levels(h.lmin, h.lmax, ijk, mass)
            out = s.alloc_outputs(device=dev)

            def step():
                s.set_levels(h.lmin, h.lmax, ijk, mass)
                s.solve(out=out)

            ms = _timed(torch, step, 2 if prec == "fp64" else 50, 3, stream)
            s.sync()
            s.set_timing(True)
            s.update_masses(mass)
            s.solve(out=out)
            s.sync()
            st = s.stage_times()
            s.set_timing(False)
            outs[prec] = ({l: out[0][l].double() for l in h.levels}, {l: out[1][l].double() for l in h.levels})
            rows.append({"config": cname, "precision": prec, "cells": h.n_cells, "ms": ms,
                         "value": h.n_cells / (ms * 1e-3), "stages_ms": st})
            del s, out
        (pm, am), (pd, ad) = outs["mixed"], outs["fp64"]
        num_a = sum(float(((am[l] - ad[l]) ** 2).sum()) for l in h.levels)
        den_a = sum(float((ad[l] ** 2).sum()) for l in h.levels)
        n = sum(h.n(l) for l in h.levels)
        num_p = sum(float(((pm[l] - pd[l]) ** 2).sum()) for l in h.levels)
        rms_p = np.sqrt(sum(float((pd[l] ** 2).sum()) for l in h.levels) / n)
        rows[-1]["rel_rms_accel_vs_fp64"] = float(np.sqrt(num_a / den_a))
        rows[-1]["rms_phi_err_vs_fp64_over_scale"] = float(np.sqrt(num_p / n) / max(rms_p, h.total_mass()))
    return {"unit": UNIT, "step": "fmm_set_levels + fmm_solve (inputs resident), periodic boundaries", "runs": rows,
            "wall_s": time.perf_counter() - t0}


def leg_binary(args, torch, dev, stream, flush):
    """The paper's binary orbit test (Sec. 4, Figs. 5-6): two point masses (GM = 0.01
    each, separation 0.15) deposited by CIC on a grid with lmin = 6 and lmax = 6, 7, 8
    that follows them (nexpand = 2), fixed-step kick-drift-kick leapfrog to t = 8
    (about three orbits), p = 6 mixed; the diagnostics of Fig. 6 at t = 8."""
    from paper_2607_19489_b300 import binary
    runs = []
    for lmax in (6, 7, 8):
        b = binary.Binary(lmin=6, lmax=lmax, p=P_ORDER, precision="mixed", nexpand=2)
        period = 2 * np.pi / b.omega
        t0 = time.perf_counter()
        d = b.run(8.0, period / 200)
        d.update({"lmin": 6, "lmax": lmax, "dt": period / 200, "wall_s": time.perf_counter() - t0,
                  "ms_per_step_wall": 1e3 * (time.perf_counter() - t0) / d["solves"]})
        runs.append(d)
        del b
    return {"workload": "binary orbit, GM = 0.01 each, separation 0.15, CIC, nexpand = 2, KDK leapfrog, "
                        "p=6 mixed", "runs": runs,
            "step": "per solve: grid around the particles (host), CIC deposit, fmm_set_levels + fmm_solve, "
                    "CIC interpolation"}


def leg_batched(args, torch, dev, stream, flush):
    """64 independent hierarchies (32^3/64^3/128^3 bases, 1-3 nested levels,
    Gaussian blobs), p = 6 mixed, one CUDA graph launch per batch; launch
    shapes from the autotuner (one tuned context per base size)."""
    from paper_2607_19489_b300 import fmm, workloads as W
    t0 = time.perf_counter()
    hs = W.batched_blobs(count=64, seed=5)
    gen_s = time.perf_counter() - t0
    solvers, tuned = [], {}
    for h in hs:
        s = fmm.Solver(P_ORDER, "mixed")
        s.set_hierarchy(h, device=dev)
        if h.lmin not in tuned:
            tuned[h.lmin] = s.autotune()
        else:
            s.set_tuning(tuned[h.lmin])
        solvers.append(s)
    outs = [s.alloc_outputs(device=dev) for s in solvers]
    free, total = torch.cuda.mem_get_info(dev)
    cells = int(sum(h.n_cells for h in hs))
    K = max(3, min(args.steps // 20, 20))
    l0 = sum(s.stats()["launches"] for s in solvers)
    masses = [[torch.as_tensor(m, device=dev) for m in h.mass] for h in hs]

    def new_masses():  # every step solves for fresh masses: nothing is reused
        for sv, ms in zip(solvers, masses):
            sv.update_masses(ms)

    def batch():
        new_masses()
        fmm.batch_solve(solvers, outs)

    def one_by_one():
        new_masses()
        for sv, o in zip(solvers, outs):
            sv.solve(out=o)

    ms_batch = _timed(torch, batch, K, 3, stream)
    l1 = sum(s.stats()["launches"] for s in solvers)
    ms_seq = _timed(torch, one_by_one, K, 2, stream)
    for s in solvers:
        s.sync()
    # accuracy of the mixed batch against FP64 solves of the same hierarchies (the FP64
    # path matches the oracle to 1e-10 in the tests): the largest hierarchy of each base size
    acc_err = []
    for i in sorted({min(range(len(hs)), key=lambda j: (hs[j].lmin != b, -hs[j].n_cells)) for b in (5, 6, 7)}):
        ref = fmm.Solver(P_ORDER, "fp64")
        ref.set_hierarchy(hs[i], device=dev)
        rp, ra = ref.solve()
        ref.sync()
        got = outs[i][1]
        num = sum(float(((got[l].double() - ra[l]) ** 2).sum()) for l in ra)
        den = sum(float((ra[l] ** 2).sum()) for l in ra)
        acc_err.append(float(np.sqrt(num / den)))
        del ref
    out = {"workload": "64 isolated hierarchies, bases 32^3/64^3/128^3 by seed, 1-3 nested levels of 1/4-1/2 "
                       "width, 1-8 Gaussian blobs, p=6 mixed", "hierarchies": len(hs), "cells": cells,
           "value": cells / (ms_batch * 1e-3), "unit": UNIT, "ms_per_batch": ms_batch,
           "one_graph_per_hierarchy_ms": ms_seq, "gpu_launches_per_batch": (l1 - l0) // (K + 3),
           "tuning_by_base_level": {str(k): v for k, v in tuned.items()},
           "rel_rms_accel_mixed_vs_fp64": acc_err,
           "device_memory_used_gb": (total - free) / 1e9, "generation_s": gen_s,
           "step": "fmm_update_masses (device copy, all 64) + fmm_batch_solve"}
    del solvers, outs
    return out


def leg_adjoint(args, torch, dev, stream, flush):
    """Nested two-Plummer hierarchy (128^3 base, refined central boxes at levels
    8 and 9), FP64: forward solve and adjoint (loss = sum w . accel)."""
    from paper_2607_19489_b300 import fmm, workloads as W
    h = W.nested_two_plummer()
    s = fmm.Solver(P_ORDER, "fp64")
    ijk = [torch.as_tensor(a, device=dev).contiguous() for a in h.ijk]
    mass = [torch.as_tensor(m, device=dev).contiguous() for m in h.mass]
    s.set_levels(h.lmin, h.lmax, ijk, mass)
    out = s.alloc_outputs(device=dev)
    w = {l: torch.as_tensor(W.normal(31, 300 + l, np.arange(3 * h.n(l))).reshape(-1, 3), device=dev)
         for l in h.levels}
    zero = {l: torch.zeros(h.n(l), dtype=torch.float64, device=dev) for l in h.levels}
    gm = {l: torch.empty(h.n(l), dtype=torch.float64, device=dev) for l in h.levels}
    ms_fwd = _timed(torch, lambda: s.solve(out=out), 2, 1, stream)
    ms_adj = _timed(torch, lambda: s.solve_adjoint(zero, w, out=gm), 2, 1, stream)
    s.sync()
    lhs = sum(float((w[l] * out[1][l]).sum()) for l in h.levels)
    rhs = sum(float((gm[l] * mass[k]).sum()) for k, l in enumerate(h.levels))
    fd = None
    if args.fd_cells > 0:
        # forward differences: the loss is linear in the masses, so
        # (L(m + h e_i) - L(m)) / h = dL/dm_i with no truncation error, and a step
        # of the whole box's mass (h = 1; cells hold ~1e-7) keeps rounding small
        t_fd = time.perf_counter()
        n_all = sum(h.n(l) for l in h.levels)
        offs = np.cumsum([0] + [h.n(l) for l in h.levels])
        picks = np.unique((W.uniform(41, 1, np.arange(args.fd_cells)) * n_all).astype(np.int64))
        step = 1.0
        s.update_masses(mass)
        s.solve(out=out)
        s.sync()
        l0 = sum(float((w[l] * out[1][l]).sum()) for l in h.levels)
        errs = []
        for g in picks:
            k = int(np.searchsorted(offs, g, side="right") - 1)
            j = int(g - offs[k])
            mp = [m.clone() for m in mass]
            mp[k][j] += step
            s.update_masses(mp)
            s.solve(out=out)
            s.sync()
            l1 = sum(float((w[l] * out[1][l]).sum()) for l in h.levels)
            ad = float(gm[h.lmin + k][j])
            errs.append(abs((l1 - l0) / step - ad) / max(abs(ad), 1e-300))
        s.update_masses(mass)
        fd = {"cells": int(len(picks)), "h": step, "kind": "forward differences (exact for the linear map)",
              "max_rel_err": float(max(errs)), "median_rel_err": float(np.median(errs)),
              "wall_s": time.perf_counter() - t_fd}
    res = {"workload": "nested two-Plummer 128^3 + 2 refined levels (central 1/4 and 1/16 volumes), p=6 FP64",
           "finite_differences": fd,
           "cells": h.n_cells, "forward_ms": ms_fwd, "adjoint_ms": ms_adj, "adjoint_over_forward": ms_adj / ms_fwd,
           "dot_identity_rel": abs(lhs - rhs) / max(abs(lhs), 1e-300),
           "check": "<w, accel(m)> = <dL/dm, m> (linear map), and per-cell finite differences"}
    del s
    return res


def leg_ats(args, torch, dev, stream, flush):
    """Lognormal 256^3 base (sigma 1, P(k) ~ k^-2), refined where the cell mass
    exceeds 8x the mean base-cell mass (up to 4 levels); one coarse step = the
    amr_step schedule of full and fine-level-only solves, each after rebuilding
    the active levels with +-1e-3 perturbed masses; p = 6 mixed, FP32 outputs."""
    from paper_2607_19489_b300 import fmm, workloads as W
    t0 = time.perf_counter()
    h = W.lognormal_amr(base=8)
    gen_s = time.perf_counter() - t0
    sched = W.ats_schedule(h.lmin, h.lmax)
    s = fmm.Solver(P_ORDER, "mixed", out_fp32=True)
    ijk = [torch.as_tensor(a, device=dev).contiguous() for a in h.ijk]
    base = [torch.as_tensor(m, device=dev).contiguous() for m in h.mass]
    s.set_levels(h.lmin, h.lmax, ijk, base)
    tuning = s.autotune()
    # perturbed masses of each rebuild, resident before the timed region
    pert = []
    for i, lo in enumerate(sched):
        k0 = lo - h.lmin
        pert.append([base[k] * torch.as_tensor(1.0 + 1e-3 * (2 * W.uniform(77, 1000 * i + k, np.arange(h.n(h.lmin + k))) - 1),
                                               device=dev) for k in range(k0, len(base))])
    outs = {lo: s.alloc_outputs(lo, device=dev) for lo in set(sched)}

    def coarse_step():
        for lo, ms in zip(sched, pert):
            s.set_levels(h.lmin, h.lmax, ijk[lo - h.lmin:], ms, lo=lo)
            s.solve(lo, out=outs[lo])

    K = max(3, min(args.steps // 40, 10))
    ms_step = _timed(torch, coarse_step, K, 3, stream)
    # one more coarse step with an event pair around every solve of the schedule
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(sched) + 1)]
    host_warm()
    evs[0].record(stream)
    for i, (lo, ms) in enumerate(zip(sched, pert)):
        s.set_levels(h.lmin, h.lmax, ijk[lo - h.lmin:], ms, lo=lo)
        s.solve(lo, out=outs[lo])
        evs[i + 1].record(stream)
    evs[-1].synchronize()
    per_solve = [{"lo": lo, "ms": evs[i].elapsed_time(evs[i + 1]),
                  "cells": sum(h.n(l) for l in range(lo, h.lmax + 1))} for i, lo in enumerate(sched)]
    # Each kind of solve alone, as a subcycle loop runs it: the stream idle and
    # the host core busy before it (a solve that follows a 60 ms one in the
    # schedule starts on a host core that idled meanwhile, and its launch work
    # then runs several times slower), median of 20 rebuild + solve pairs.
    per_lo = {}
    for lo, ms in zip(sched, pert):
        if lo in per_lo or lo == h.lmin:
            continue
        tt = []
        for _ in range(20):
            torch.cuda.synchronize()
            host_warm(0.05)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.set_levels(h.lmin, h.lmax, ijk[lo - h.lmin:], ms, lo=lo)
            s.solve(lo, out=outs[lo])
            e1.record(stream)
            e1.synchronize()
            tt.append(e0.elapsed_time(e1))
        per_lo[str(lo)] = statistics.median(tt)
    # in-order stage times of each kind of solve in the schedule (one rebuild + solve per lo)
    s.set_timing(True)
    stages = {}
    for lo, ms in zip(sched, pert):
        if lo in stages:
            continue
        s.set_levels(h.lmin, h.lmax, ijk[lo - h.lmin:], ms, lo=lo)
        s.solve(lo, out=outs[lo])
        s.sync()
        stages[lo] = s.stage_times()
    s.set_timing(False)
    s.set_levels(h.lmin, h.lmax, ijk, base)
    ms_full = _timed(torch, lambda: (s.set_levels(h.lmin, h.lmax, ijk, base), s.solve(out=outs[h.lmin])), K, 2, stream)
    s.sync()
    updated = sum(sum(h.n(l) for l in range(lo, h.lmax + 1)) for lo in sched)
    # accuracy of the mixed, FP32-output solve against an FP64 solve of the same masses
    s.set_levels(h.lmin, h.lmax, ijk, base)
    mp, ma = s.solve(out=outs[h.lmin])
    ref = fmm.Solver(P_ORDER, "fp64")
    ref.set_levels(h.lmin, h.lmax, ijk, base)
    rp, ra = ref.solve()
    ref.sync()
    s.sync()
    num = sum(float(((ma[l].double() - ra[l]) ** 2).sum()) for l in ra)
    den = sum(float((ra[l] ** 2).sum()) for l in ra)
    err_ats = float(np.sqrt(num / den))
    del ref
    res = {"workload": h.name + ", p=6 mixed, FP32 outputs", "cells": h.n_cells,
           "levels": [h.n(l) for l in h.levels], "schedule_lo": sched,
           "value": updated / (ms_step * 1e-3), "unit": UNIT, "ms_per_coarse_step": ms_step,
           "per_solve": per_solve, "solve_alone_ms_by_lo": per_lo,
           "stages_ms_by_lo": {str(k): v for k, v in sorted(stages.items())},
           "cell_updates_per_coarse_step": updated, "full_rebuild_and_solve_ms": ms_full,
           "tuning": tuning, "generation_s": gen_s, "rel_rms_accel_mixed_vs_fp64": err_ats,
           "step": "per solve of the schedule: fmm_set_levels(lo) with perturbed masses + fmm_solve(lo)"}
    del s
    return res


# ---------------------------------------------------------------------------- CPU oracle

def cpu_baseline(h, per_level: int):
    """The oracle as it stands, all host threads, on a bounded sample of targets."""
    import oracle
    from paper_2607_19489_b300 import workloads as W
    sel = {l: np.unique((W.uniform(11, 700 + l, np.arange(per_level)) * h.n(l)).astype(np.int64))
           for l in h.levels}
    n = int(sum(v.size for v in sel.values()))
    threads = oracle.lib().oracle_max_threads()
    t0 = time.perf_counter()
    oracle.solve(h, P_ORDER, sel=sel, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} seeded target cells ({per_level} per level) of the same hierarchy; "
                      f"wall time {dt:.1f} s includes the oracle's tree, merged-tree and local-expansion setup"}


def reference_arm(args, rank, world):
    if rank != 0:
        return
    h = make_workload(args.workload)
    per = []
    cb = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(h, per_level=args.ref_sample)
        if i >= args.warmup:
            per.append(cb["value"])
    value = statistics.mean(per)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)", "impl": "reference",
            "config": {"workload": WORKLOADS[args.workload], "cells": h.n_cells, "p": P_ORDER},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": cb["cores"],
                             "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=4000, help="oracle targets per level for cpu_baseline")
    ap.add_argument("--ref-sample", type=int, default=1000, help="oracle targets per level per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="two_level", choices=sorted(WORKLOADS),
                    help="two_level: the measured configuration; unigrid16: a small check of the launch paths")
    ap.add_argument("--fd-cells", type=int, default=100,
                    help="adjoint leg: finite differences on this many seeded cells (one FP64 solve each)")
    ap.add_argument("--legs", default="sweep,batched,adjoint,ats,binary,delta_l,periodic",
                    help="extra workloads reported beside the headline (comma list, or 'none')")
    ap.add_argument("--quick", action="store_true",
                    help="the mixed headline and its stage times only (no FP64 arm, e2e, legs or CPU baseline)")
    ap.add_argument("--profile-solves", type=int, default=0,
                    help="for profilers: set the headline hierarchy, then run this many in-order, stage-timed mixed "
                         "solves (the launch shapes the roofline times) and exit without a JSON line")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.profile_solves:
        profile_solves(args)
        return
    gpu_arm(args, rank, world, local)


if __name__ == "__main__":
    main()
