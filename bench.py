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


def load_peaks():
    for path in (os.path.join(ROOT, "MEASURED_PEAKS.json"), "/root/repo/MEASURED_PEAKS.json"):
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
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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

def make_workload():
    from paper_2607_19489_b300 import workloads as W
    return W.two_level_plummer()


def rel_rms(a: dict, b: dict) -> float:
    num = sum(float(((a[l] - b[l]) ** 2).sum()) for l in b)
    den = sum(float((b[l] ** 2).sum()) for l in b)
    return float(np.sqrt(num / den))


def timed_steps(torch, step, K, W, stream, flush):
    for _ in range(W):
        step()
    torch.cuda.synchronize()
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


def gpu_arm(args, rank, world, local):
    import torch
    from paper_2607_19489_b300 import fmm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, "nccl")
    stream = torch.cuda.current_stream()
    h = make_workload()
    n_cells = h.n_cells
    ijk = [torch.as_tensor(a, device=dev).contiguous() for a in h.ijk]
    mass = [torch.as_tensor(m, device=dev).contiguous() for m in h.mass]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def make(precision):
        s = fmm.Solver(P_ORDER, precision)
        s.set_levels(h.lmin, h.lmax, ijk, mass)
        out = s.alloc_outputs()
        return s, out

    mixed, out_m = make("mixed")
    fp64, out_d = make("fp64")

    def step_mixed():
        mixed.set_levels(h.lmin, h.lmax, ijk, mass)
        mixed.solve(out=out_m)

    def step_mixed_solve_only():
        mixed.solve(out=out_m)

    def step_fp64():
        fp64.set_levels(h.lmin, h.lmax, ijk, mass)
        fp64.solve(out=out_d)

    # accuracy of the mixed path against the FP64 GPU path (which matches the oracle to 1e-10)
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
    t_solve = timed_steps(torch, step_mixed_solve_only, args.steps, 3, stream, flush)
    k64 = max(3, min(args.steps, 5))
    t_fp64 = timed_steps(torch, step_fp64, k64, 3, stream, flush)
    mixed.sync()
    fp64.sync()
    barrier(dist)

    ms_mixed = reduce_max(statistics.mean(t_mixed), dist, dev)
    ms_solve = reduce_max(statistics.mean(t_solve), dist, dev)
    ms_fp64 = reduce_max(statistics.mean(t_fp64), dist, dev)
    value = world * n_cells / (ms_mixed * 1e-3)
    value_fp64 = world * n_cells / (ms_fp64 * 1e-3)

    # per-stage device times of the solve (events inside the library, on this stream)
    mixed.set_timing(True)
    stage = {k: 0.0 for k in ("upward", "downward", "m2p", "near")}
    reps = max(3, args.steps)
    for _ in range(reps):
        flush.zero_()
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

    t_e2e = timed_steps(torch, step_e2e, args.steps, 3, stream, flush)
    e2e_solver.sync()
    ms_e2e = reduce_max(statistics.mean(t_e2e), dist, dev)
    h2d = sum(a.nbytes for a in np_ijk) + sum(m.nbytes for m in np_mass)
    d2h = sum(v.nbytes for v in np_out[0].values()) + sum(v.nbytes for v in np_out[1].values())

    peaks, peak_src = load_peaks()
    n_tgt = n_cells
    m2p_useful = 2.0 * 189 * 4 * NC * n_tgt                       # per solve (all target levels)
    rows = sum(int(mixed.tree_counts()[l - 1]) for l in h.levels)  # upper bound on M2P rows
    roofline = {
        "kernel": "k_gemm_tc (bottom M2P, split-BF16 x3 on tcgen05)",
        "bound": "tensor",
        "achieved": m2p_useful / (stage["m2p"] * 1e-3) / 1e12,
        "peak": peaks["bf16_tflops_sustained"] / 3.0,
        "unit": "TFLOP/s",
        "traffic": None,
        "peak_note": f"{peak_src} bf16 dense sustained / 3 (three bf16 products per split-BF16 product); "
                     "achieved counts useful flops 2*189*4*ncoef per target cell",
        "stage_ms": stage["m2p"],
    }
    roofline["frac"] = roofline["achieved"] / roofline["peak"]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3+f32+f64", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "cells": n_cells, "levels": [h.n(l) for l in h.levels], "p": P_ORDER,
                   "step": "fmm_set_levels (tree build) + fmm_solve", "l2": "flushed (256 MB write) before each step",
                   "parallelism": f"replicas x{world} (independent hierarchies)"},
        "fp64_gpu": {"value": value_fp64, "ms_per_step": ms_fp64, "speedup_mixed_over_fp64": value / value_fp64},
        "accuracy": {"rel_rms_accel_mixed_vs_fp64": err_acc, "rel_rms_phi_mixed_vs_fp64": err_phi,
                     "bar": 1e-4},
        "solve_only": {"value": world * n_cells / (ms_solve * 1e-3), "ms": ms_solve},
        "stages_ms": stage,
        "e2e": {"value": world * n_cells / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
        "gpu_launches": int(launches1 - launches0),
        "roofline": roofline,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(h, per_level=args.cpu_sample)
    if rank == 0:
        print(json.dumps(line))
    barrier(dist)
    del rows


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
    h = make_workload()
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
            "config": {"workload": WORKLOAD, "cells": h.n_cells, "p": P_ORDER},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": cb["cores"],
                             "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=4000, help="oracle targets per level for cpu_baseline")
    ap.add_argument("--ref-sample", type=int, default=1000, help="oracle targets per level per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    gpu_arm(args, rank, world, local)


if __name__ == "__main__":
    main()
