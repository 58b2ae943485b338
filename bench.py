#!/usr/bin/env python
"""Benchmark of the collision-operator hot path on GB300.

One step = one evaluation of Q(f, f) (reconstruction, loss sums, fused point generation +
spreading, cosine transform + deconvolution, combine).  The headline is the 2D hard-sphere
workload: d = 2, N = 64 (65^2 modes), M = 32 circle points, S = 3, gamma = 1, algebraic map,
f = three Maxwellians + a Gaussian-windowed positive perturbation (seeded synthetic input,
projected on the GPU), in the FP32-spreading path (tol 1e-6; loss, transform, deconvolution
and moments in FP64).  Beside it the line carries a row per single-plan workload (2D Maxwell
molecules N = 16, 2D hard spheres N = 64, 3D BKW N = 16, 3D gamma = 1/2 bi-Maxwellian N = 24):
FP32 and FP64 timings, the error against the oracle's stored values on seeded modes and against
the FP64 path on all modes, the mode-level conservation residuals, the spreading roofline, and
the CPU oracle timed on a bounded sample; and the 4096-cell batched workload.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on bounded samples
of the headline workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Q(f,f) evals/s and NU points/s at stated rel err; FP32/batched vs FP64, % roofline"
UNIT = "Q evals/s"
# Single-plan workloads: name -> (workloads.py constructor, description).  The default run
# measures all of them; --workload restricts it to one (for profiling).
WORKLOADS = {
    "2d-maxwell": ("c1_2d_maxwell", "2D Maxwell molecules (gamma=0), N=16, M=8 circle points, S=2, algebraic map"),
    "2d-hard-spheres": ("c2_2d_vhs", "2D hard spheres (gamma=1), N=64 (65^2 modes), M=32 circle points, S=3, "
                                     "algebraic map"),
    "3d-bkw": ("c3_3d_bkw", "3D Maxwell molecules on the BKW datum (K=3/5), N=16, M=32 antipodal Fibonacci "
                            "points, S=2, algebraic map"),
    "3d-bimaxwell": ("c4_3d_bimaxwell", "3D VHS gamma=1/2 on a bi-Maxwellian (T=0.6/1.4/1.4), N=24, M=32 "
                                        "antipodal Fibonacci points, S=3, algebraic map"),
}
HEADLINE = "2d-hard-spheres"
# DRAM bytes (read + write) of one launch of the FP32 spreading kernel on the headline workload,
# from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum), valid only while the code
# of the kernel's sources (comments aside) hashes to source_sha16 (reported as null otherwise).
PROFILED_TRAFFIC = {"kernel": "k_spread_f32<2,6,0>", "bytes": 292608, "source_sha16": "1662833d363ae60e"}
KERNEL_SOURCES = ("spread_impl.cuh", "spread_f32_2d.cu", "pgb_internal.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-full", action="store_true",
                    help="run the CPU oracle in full (all outer nodes) for the 2D workloads and the 3D BKW one "
                         "instead of a bounded sample (minutes of CPU time)")
    ap.add_argument("--fp64-steps", type=int, default=-1,
                    help="timed steps of the FP64 path (-1: --steps for 2D workloads, 2 for the 3D BKW one, "
                         "none for the 3D bi-Maxwellian)")
    ap.add_argument("--no-fp64-3d", action="store_true", help="skip the FP64 path of the 3D workloads")
    ap.add_argument("--tol32", type=float, default=1e-6)
    ap.add_argument("--upsampfac", type=float, default=0.0)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=2)
    ap.add_argument("--batched-cells", type=int, default=0,
                    help="run the batched workload on its first K cells only (0: all 4096; for profiling)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=None,
                    help="measure this single-plan workload only (for profiling)")
    ap.add_argument("--batched-only", action="store_true",
                    help="measure the batched workload only, beside the headline's FP32 path (for profiling)")
    ap.add_argument("--sphere-points", type=int, default=0,
                    help="override the workload's number of sphere points M (0: the workload's own; for "
                         "profiling the same kernel on a smaller case)")
    return ap.parse_args()


def code_lines(text):
    """The source's code without // comments and blank lines (comment edits keep the hash)."""
    out = []
    for line in text.splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code:
            out.append(code)
    return "\n".join(out)


def kernel_source_sha16():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2105_08806_gb300", "csrc", name), encoding="utf-8") as fh:
            h.update(code_lines(fh.read()).encode())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, enabled: bool = True):
        self.enabled = enabled
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        if not self.enabled:
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.enabled or self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- distributed
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(values, world, device="cpu"):
    """Element-wise maximum over ranks (the job's timing is its slowest rank)."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def aggregate_throughput(ms_per_step, world):
    """Whole-job evaluations per second: every rank evaluates its own problem each step."""
    return world * 1000.0 / ms_per_step


# ------------------------------------------------------------ CPU oracle timing
def cpu_baseline(workload, budget_s=8.0, full=False):
    """The FP64 oracle, as it stands, on the host cores: the first n outer nodes i of the
    workload's triple sum (all j, all sigma_m, all modes), n sized to about budget_s seconds
    (every node with full=True), scaled to one evaluation."""
    from oracle import oracle as O

    d, N, M, S, g = workload.d, workload.N, workload.M, workload.S, workload.gamma
    ft = O.project(workload, d, N, S, 1).ravel()
    nnode = N ** d
    threads = O.default_threads()
    if full:
        n2 = nnode
    else:
        n = min(nnode, max(threads, 8))
        t0 = time.perf_counter()
        O.collide_parts(ft, d, N, M, S, g, r=1, outer=(0, n), nthreads=threads)
        per_node = (time.perf_counter() - t0) / n
        n2 = int(min(nnode, max(n, budget_s / per_node)))
        n2 = min(nnode, max(threads, (n2 // threads) * threads))
    t0 = time.perf_counter()
    O.collide_parts(ft, d, N, M, S, g, r=1, outer=(0, n2), nthreads=threads)
    dt2 = time.perf_counter() - t0
    evals_per_s = (n2 / nnode) / dt2
    sample = (f"all {nnode} outer nodes" if n2 == nnode else f"outer nodes 0..{n2 - 1} of {nnode}") + \
        f" (all j, all {M} sigma, all {(N + 1) ** d} modes) in {dt2:.2f} s" + \
        ("" if n2 == nnode else f", scaled by {nnode}/{n2}")
    return {"value": evals_per_s, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
            "seconds_per_eval": 1.0 / evals_per_s}


# ------------------------------------------------------------ single plans
def oracle_samples(name):
    """(flat mode indices, gain, loss) stored by tests/golden/make_oracle_samples.py from oracle/."""
    import numpy as np

    path = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.txt")
    a = np.loadtxt(path, comments="#", ndmin=2)
    d = a.shape[1] - 2
    modes = a[:, :d].astype(np.int64)
    return modes, a[:, d], a[:, d + 1]


def flat_index(modes, N):
    import numpy as np

    idx = np.zeros(modes.shape[0], dtype=np.int64)
    for l in range(modes.shape[1]):
        idx = idx * (N + 1) + modes[:, l]
    return idx


class Timer:
    """Device-timed evaluations of one plan on one stream, the L2 flushed between steps."""

    def __init__(self, stream, flush, barrier):
        self.stream, self.flush, self.barrier = stream, flush, barrier

    def run(self, plan, ft, out, steps, warmup):
        import torch

        for _ in range(warmup):
            plan.collide(ft, out)
        self.stream.synchronize()
        plan.set_timing(True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        stages = []
        self.barrier()
        t0 = time.perf_counter()
        for k in range(steps):
            with torch.cuda.stream(self.stream):
                self.flush.fill_(float(k))
            evs[k][0].record(self.stream)
            plan.collide(ft, out)
            evs[k][1].record(self.stream)
            stages.append(plan.stage_times())
        self.barrier()
        wall = time.perf_counter() - t0
        plan.set_timing(False)
        return [a.elapsed_time(b) for a, b in evs], stages, wall


STAGES = ["reconstruct", "loss", "spread", "transform"]


def mean_stages(stages):
    return {n: statistics.mean(s[i] for s in stages) for i, n in enumerate(STAGES)}


def errors_vs_oracle(Q, N, name):
    """Relative L2 error on the stored oracle modes, against |Q| and against the gain |Q+| there."""
    import numpy as np

    modes, gain, loss = oracle_samples(name)
    ref = gain - loss
    e = np.linalg.norm(Q[flat_index(modes, N)] - ref)
    return {"modes": int(len(ref)), "rel_l2_Q": float(e / np.linalg.norm(ref)),
            "rel_l2_gain": float(e / np.linalg.norm(gain))}


def spread_roofline(info, d, spread_ms, peaks):
    """Shared-memory additions of the spreading kernel: w^d for each of the M N^d (N^d + 1)/2 points
    of the unordered node pairs (the points the kernel skips exactly, whose contributions all round
    to zero, included), per launch, over the launch's time; peak = the measured conflict-free
    int32 shared-atomic rate of the whole GPU."""
    adds = info["points"] * info["kernel_width"] ** d
    achieved = adds / (spread_ms * 1e-3)
    return {"bound": "alu", "achieved": achieved / 1e9, "peak": peaks["shared_atomics_free"] / 1e9,
            "unit": "G shared-memory additions/s", "frac": achieved / peaks["shared_atomics_free"],
            "additions_per_launch": adds,
            "peak_basis": "measured: int32 shared atomics, every lane on its own bank, all SMs (pg_boltz_probe_pipes)",
            "frac_of_random_address_atomics": achieved / peaks["shared_atomics_random"]}


def measure_config(name, args, dev, stream, timer, peaks, world):
    """One single-plan workload: FP32 path (the tolerance of --tol32) and FP64 path (tol 1e-13)."""
    import numpy as np
    import torch

    from paper_2105_08806_gb300 import PG_PREC_FP32, PG_PREC_FP64, Plan
    from paper_2105_08806_gb300 import workloads as Wl

    w = getattr(Wl, WORKLOADS[name][0])()
    d, N, M, S, gamma = w.d, w.N, w.M, w.S, w.gamma
    if args.sphere_points > 0:
        M = args.sphere_points
    plan32 = Plan(d, N, M, S, gamma, args.tol32, precision=PG_PREC_FP32, upsampfac=args.upsampfac)
    plan32.set_stream(stream)
    info = plan32.info()
    # input: f at the projection nodes (seeded workload density), projected on the GPU
    v = np.array(plan32.project_nodes())
    grids = np.meshgrid(*([v] * d), indexing="ij")
    fv = torch.as_tensor(w(np.stack([g.ravel() for g in grids], 1)), device=dev)
    ft = torch.empty((N + 1) ** d, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        plan32.project(fv, ft)
    Q32 = torch.empty_like(ft)
    ms32, st32, wall32 = timer.run(plan32, ft, Q32, args.steps, args.warmup)
    mom32 = plan32.moments()
    mean32 = reduce_max([statistics.mean(ms32)], world, dev)[0]
    stages32 = mean_stages(st32)
    q32 = Q32.cpu().numpy()
    row = {
        "workload": WORKLOADS[name][1] + ("" if M == w.M else f" (M overridden to {M})"),
        "d": d, "N": N, "M": M, "S": S, "gamma": gamma,
        "fp32": {
            "tol": args.tol32, "kernel_width": info["kernel_width"], "n_grid": info["n_grid"],
            "slabs": info["slabs"], "spread_blocks": info["spread_blocks"], "steps": len(ms32),
            "kernels_per_collide": info["kernels_per_collide"],
            "ms_per_eval": mean32, "evals_per_s": aggregate_throughput(mean32, world),
            "points_per_eval": info["points"], "points_per_s": aggregate_throughput(mean32, world) * info["points"],
            "points_per_s_paper_convention": aggregate_throughput(mean32, world) * M * (N + 2) ** (2 * d),
            "stages_ms": stages32,
            "mode_mass_rel": abs(mom32["mass"]) / abs(mom32["mass_gain"]),
            "mode_energy_rel": abs(mom32["energy"]) / abs(mom32["energy_gain"]),
            "roofline": spread_roofline(info, d, stages32["spread"], peaks),
        },
        "_wall_s": wall32,
    }
    if M == w.M:
        row["fp32"]["rel_err_vs_oracle_sampled"] = errors_vs_oracle(q32, N, name)
    plan32.close()
    # FP64 path: the same steps for the 2D workloads; 3D FP64 evaluations take seconds (3D BKW) to
    # minutes (the gamma = 1/2 bi-Maxwellian) each
    n64 = args.fp64_steps if args.fp64_steps >= 0 else (args.steps if d == 2 else (2 if N <= 16 else 0))
    if d == 3 and args.no_fp64_3d:
        n64 = 0
    if n64 > 0:
        plan64 = Plan(d, N, M, S, gamma, 1e-13, precision=PG_PREC_FP64)
        plan64.set_stream(stream)
        Q64 = torch.empty_like(ft)
        ms64, st64, _ = timer.run(plan64, ft, Q64, n64, 1 if d == 3 else min(args.warmup, 3))
        mom64 = plan64.moments()
        info64 = plan64.info()
        plan64.close()
        mean64 = reduce_max([statistics.mean(ms64)], world, dev)[0]
        q64 = Q64.cpu().numpy()
        e = float(np.linalg.norm(q32 - q64))
        row["fp64"] = {"tol": 1e-13, "kernel_width": info64["kernel_width"], "slabs": info64["slabs"],
                       "steps": len(ms64), "ms_per_eval": mean64, "evals_per_s": aggregate_throughput(mean64, world),
                       "stages_ms": mean_stages(st64),
                       "mode_mass_rel": abs(mom64["mass"]) / abs(mom64["mass_gain"]),
                       "mode_energy_rel": abs(mom64["energy"]) / abs(mom64["energy_gain"])}
        if M == w.M:
            row["fp64"]["rel_err_vs_oracle_sampled"] = errors_vs_oracle(q64, N, name)
        row["fp32"]["rel_err_vs_fp64_path_all_modes"] = {"rel_l2_Q": e / float(np.linalg.norm(q64)),
                                                         "rel_l2_gain": e / mom64["norm_gain"]}
        row["norm_Q_over_norm_gain"] = float(np.linalg.norm(q64)) / mom64["norm_gain"]
        row["speedup_fp32_vs_fp64"] = mean64 / mean32
    else:
        row["fp64"] = {"skipped": "not timed by default: one FP64 evaluation takes about 77 s here "
                                  "(--fp64-steps 1 times it)" if (d == 3 and N > 16 and args.fp64_steps < 0)
                       else "--no-fp64-3d or --fp64-steps 0"}
        row["norm_Q_over_norm_gain"] = float(np.linalg.norm(q32)) / mom32["norm_gain"]
    return row


def headline_extras(args, dev, stream, timer, world):
    """The headline workload end to end through the public API (pinned host f~ in, host Q out,
    every step) and its screened variant."""
    import numpy as np
    import torch

    from paper_2105_08806_gb300 import PG_PREC_FP32, Plan
    from paper_2105_08806_gb300 import workloads as Wl

    w = getattr(Wl, WORKLOADS[HEADLINE][0])()
    d, N, M, S, gamma = w.d, w.N, w.M, w.S, w.gamma
    plan = Plan(d, N, M, S, gamma, args.tol32, precision=PG_PREC_FP32, upsampfac=args.upsampfac)
    plan.set_stream(stream)
    v = np.array(plan.project_nodes())
    grids = np.meshgrid(*([v] * d), indexing="ij")
    fv = torch.as_tensor(w(np.stack([g.ravel() for g in grids], 1)), device=dev)
    ft = torch.empty((N + 1) ** d, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        plan.project(fv, ft)
    stream.synchronize()
    fh = ft.cpu().pin_memory()
    qh = torch.empty_like(fh).pin_memory()
    fd = torch.empty_like(ft)
    Q = torch.empty_like(ft)
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            timer.flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            fd.copy_(fh, non_blocking=True)
        plan.collide(fd, Q)
        with torch.cuda.stream(stream):
            qh.copy_(Q, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if k >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    plan.close()
    mean_e2e = reduce_max([statistics.mean(e2e_ms)], world, dev)[0]
    e2e = {"value": aggregate_throughput(mean_e2e, world), "unit": UNIT, "ms_per_step": mean_e2e,
           "h2d_bytes_per_step": 8 * (N + 1) ** d, "d2h_bytes_per_step": 8 * (N + 1) ** d}
    # screened variant: node pairs whose summed strength bound is below 0.05 tol B are skipped
    plan_sc = Plan(d, N, M, S, gamma, args.tol32, precision=PG_PREC_FP32, upsampfac=args.upsampfac, screen=True)
    plan_sc.set_stream(stream)
    Qsc = torch.empty_like(ft)
    ms_sc, _, _ = timer.run(plan_sc, ft, Qsc, args.steps, args.warmup)
    plan_sc.close()
    q = Qsc.cpu().numpy()
    screened = {"ms_per_step": statistics.mean(ms_sc), "value": 1000.0 / statistics.mean(ms_sc),
                "rel_err_vs_oracle_sampled": errors_vs_oracle(q, N, HEADLINE),
                "note": "screen=1: node pairs whose summed strength bound is below 0.05 tol B are skipped"}
    return e2e, screened


# ------------------------------------------------------------------ batched
def batched_inputs(cells, stream, dev):
    """Each cell's density projected on the GPU with a plan of its N; the packed f~."""
    import numpy as np
    import torch

    from paper_2105_08806_gb300 import Plan

    d = 2
    fts, plans = [], {}
    for w in cells:
        if w.N not in plans:
            plans[w.N] = Plan(d, w.N, 8, w.S, 0.0, 1e-6)
            plans[w.N].set_stream(stream)
        pl = plans[w.N]
        v = np.array(pl.project_nodes())
        G = np.meshgrid(v, v, indexing="ij")
        fv = torch.as_tensor(w(np.stack([x.ravel() for x in G], 1)), device=dev)
        out = torch.empty((w.N + 1) ** d, dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            pl.project(fv, out)
        fts.append(out)
    stream.synchronize()
    for pl in plans.values():
        pl.close()
    return fts


def time_batched(bp, f, Q, steps, stream):
    import torch

    ms = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bp.collide(f, Q)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.mean(ms)


def run_batched(steps, stream, dev, ncells=0, fp64_cells=256):
    """The 4096-cell batched 2D workload: N in {16,24,32}, M in {8,16,32}, gamma in {0,1}, S=3,
    FP32 spreading (tol 1e-6), one graph-replayed pg_boltz_collide_batched per step; against one
    pg_boltz_collide per cell, and against the FP64 path (batched, tol 1e-13) on the first
    fp64_cells cells."""
    import numpy as np
    import torch

    from paper_2105_08806_gb300 import PG_PREC_FP32, PG_PREC_FP64, BatchedPlan, Plan
    from paper_2105_08806_gb300 import workloads as Wl

    cells = Wl.c5_batched_2d()
    if ncells > 0:
        cells = cells[:ncells]
    d = 2
    fts = batched_inputs(cells, stream, dev)
    f = torch.cat(fts)
    Q = torch.empty_like(f)
    bp = BatchedPlan(d, [w.N for w in cells], [w.M for w in cells], [w.S for w in cells],
                     [w.gamma for w in cells], 1e-6, precision=PG_PREC_FP32)
    bp.set_stream(stream)
    # launch shape and work-item size of the persistent spreading kernel picked by the library's
    # autotuner on this data (untimed)
    tuned = bp.autotune(f, Q, trials=1)
    info = bp.info()
    bp.collide(f, Q)  # capture + first replay
    stream.synchronize()
    t = time_batched(bp, f, Q, steps, stream)
    bp.close()
    # the same cells one pg_boltz_collide each (one plan per (N, M, S, gamma), reused across cells)
    single = {}
    for w in cells:
        key = (w.N, w.M, w.S, w.gamma)
        if key not in single:
            single[key] = Plan(d, w.N, w.M, w.S, w.gamma, 1e-6, precision=PG_PREC_FP32)
            single[key].set_stream(stream)
    offs = [0]
    for x in fts:
        offs.append(offs[-1] + x.numel())
    Qs = torch.empty_like(f)
    t_single = []
    for rep in range(2):  # the first pass warms up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for c, w in enumerate(cells):
            single[(w.N, w.M, w.S, w.gamma)].collide(f[offs[c]:offs[c + 1]], Qs[offs[c]:offs[c + 1]])
        b.record(stream)
        b.synchronize()
        t_single.append(a.elapsed_time(b))
    for pl in single.values():
        pl.close()
    # FP32 against FP64 batched plans on the first cells
    sub = cells[:min(fp64_cells, len(cells))]
    fsub = f[:offs[len(sub)]].contiguous()
    cmp = {}
    for prec, tol in ((PG_PREC_FP32, 1e-6), (PG_PREC_FP64, 1e-13)):
        b2 = BatchedPlan(d, [w.N for w in sub], [w.M for w in sub], [w.S for w in sub], [w.gamma for w in sub], tol,
                         precision=prec)
        b2.set_stream(stream)
        Qb = torch.empty_like(fsub)
        b2.collide(fsub, Qb)
        stream.synchronize()
        cmp[prec] = (time_batched(b2, fsub, Qb, 1, stream), Qb.cpu().numpy())
        b2.close()
    e = float(np.linalg.norm(cmp[PG_PREC_FP32][1] - cmp[PG_PREC_FP64][1]) / np.linalg.norm(cmp[PG_PREC_FP64][1]))
    return {"cells": len(cells), "ms_per_batch": t, "cell_evals_per_s": len(cells) * 1000.0 / t,
            "points_per_s": info["points"] * 1000.0 / t, "points_per_batch": info["points"],
            "spread_blocks": info["spread_blocks"], "spread_threads": info["spread_threads"],
            "autotuned": {"threads": tuned[0], "blocks": tuned[1], "item_points": tuned[2], "ms": tuned[3]},
            "one_call_per_cell_ms": t_single[-1], "speedup_vs_one_call_per_cell": t_single[-1] / t,
            "fp64_sample": {"cells": len(sub), "fp32_ms": cmp[PG_PREC_FP32][0], "fp64_ms": cmp[PG_PREC_FP64][0],
                            "speedup_vs_fp64_path": cmp[PG_PREC_FP64][0] / cmp[PG_PREC_FP32][0],
                            "rel_err_fp32_vs_fp64": e},
            "steps": steps, "launches_per_call": info["launches_per_collide"],
            "workload": f"{len(cells)} 2D cells, N in {{16,24,32}}, M in {{8,16,32}}, gamma in {{0,1}}, S=3, "
                        "FP32 tol 1e-6, CUDA graph"}


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch

    from paper_2105_08806_gb300 import workloads as Wl
    from paper_2105_08806_gb300._lib import probe_pipes, probe_shared_atomics
    from paper_2105_08806_gb300.build import build

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    timer = Timer(stream, flush, barrier)
    f32, f64, atom_free = probe_pipes(stream)
    peaks = {"fp32_fma": f32, "fp64_fma": f64, "shared_atomics_free": atom_free,
             "shared_atomics_random": probe_shared_atomics(stream),
             "basis": "measured on this GPU: pg_boltz_probe_pipes (FMA chains, conflict-free shared atomics) and "
                      "pg_boltz_probe_shared_atomics (random addresses of a 16,900-cell tile)"}
    head = args.workload or HEADLINE
    names = [head] + ([] if (args.workload or args.batched_only) else [n for n in WORKLOADS if n != head])
    with ClockSampler(local, enabled=not args.no_clocks) as clk:
        rows = {head: measure_config(head, args, dev, stream, timer, peaks, world)}
    clocks = clk.summary()
    for n in names[1:]:
        rows[n] = measure_config(n, args, dev, stream, timer, peaks, world)
    e2e, screened = (headline_extras(args, dev, stream, timer, world)
                     if head == HEADLINE and args.sphere_points == 0 and not args.batched_only else (None, None))
    batched = None
    if not args.no_batched and not args.workload:
        batched = run_batched(max(1, args.batched_steps), stream, dev, args.batched_cells)
    if rank == 0 and not args.no_cpu_baseline and args.sphere_points == 0:
        for n in names:
            w = getattr(Wl, WORKLOADS[n][0])()
            rows[n]["cpu_baseline"] = cpu_baseline(w, full=args.cpu_full and n != "3d-bimaxwell")
    h = rows[head]
    wall = h.pop("_wall_s")
    for r in rows.values():
        r.pop("_wall_s", None)
    r32 = h["fp32"]
    roof = dict(r32["roofline"])
    roof["kernel"] = f"k_spread_f32<{h['d']},{r32['kernel_width']},0>"
    same_kernel = PROFILED_TRAFFIC["source_sha16"] == kernel_source_sha16() and head == HEADLINE
    roof["traffic"] = PROFILED_TRAFFIC["bytes"] if same_kernel else None
    res = {
        "metric": METRIC,
        "value": r32["evals_per_s"],
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r32["ms_per_eval"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (the workload's seeded density, projected on the GPU)",
        "config": {
            "workload": h["workload"],
            "spread_precision": f"fp32 (tol {args.tol32:g}); loss, transform, deconvolution, moments fp64",
            "kernel_width": r32["kernel_width"], "n_grid": r32["n_grid"], "points_per_eval": r32["points_per_eval"],
            "spread_blocks": r32["spread_blocks"],
            "l2": "flushed between timed steps (256 MiB write, outside the step events)",
            "parallelism": f"replicas x{world} (independent evaluations, no collective)",
        },
        "points_per_s": r32["points_per_s"],
        "points_per_s_paper_convention": r32["points_per_s_paper_convention"],
        "rel_err_vs_oracle_sampled": r32.get("rel_err_vs_oracle_sampled"),
        "rel_err_fp32_vs_fp64_path": r32.get("rel_err_vs_fp64_path_all_modes"),
        "fp64_path": h["fp64"],
        "speedup_fp32_vs_fp64": h.get("speedup_fp32_vs_fp64"),
        "screened": screened,
        "stages_ms": r32["stages_ms"],
        "roofline": roof,
        "peaks": peaks,
        "e2e": e2e,
        "gpu_launches": r32["kernels_per_collide"] * args.steps,
        "clocks": clocks,
        "wall_s_timed_region": wall,
        "configs": rows,
        "batched": batched,
    }
    if "cpu_baseline" in h:
        res["cpu_baseline"] = h["cpu_baseline"]
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 CPU oracle, as it stands, on the host cores: each step sums the triple sum of the
    headline workload over a block of outer nodes (all j, all sigma, all modes), a bounded sample
    of one evaluation; value = evaluations per second extrapolated from the sampled fraction."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2105_08806_gb300 import workloads as Wl

    w = getattr(Wl, WORKLOADS[HEADLINE][0])()
    d, N, M, S, g = w.d, w.N, w.M, w.S, w.gamma
    ft = O.project(w, d, N, S, 1).ravel()
    nnode = N ** d
    threads = O.default_threads()
    n = threads  # outer nodes per sampled step
    times = []
    for k in range(args.warmup + args.steps):
        lo = (k * n) % nnode
        t0 = time.perf_counter()
        O.collide_parts(ft, d, N, M, S, g, r=1, outer=(lo, min(nnode, lo + n)), nthreads=threads)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    step_s = statistics.mean(times)
    frac = n / nnode
    value = frac / step_s
    res = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * step_s, "step_fraction_of_eval": frac,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[HEADLINE][1],
                   "implementation": "FP64 CPU oracle (direct triple sum), host cores",
                   "step": f"{n} of {nnode} outer nodes (all j, sigma, modes): value = fraction / step time"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"each step: {n} outer nodes of {nnode} (all j, sigma, modes), scaled by {nnode}/{n}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(res))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
