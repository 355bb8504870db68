#!/usr/bin/env python
"""Benchmark of one backward-Euler Oseen time step of the P2/P1 Navier-Stokes
discretisation (assembly + preconditioned FGMRES solve) through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fs|reference]

A "step" is one full pass of the hot path: per-step convection assembly,
right-hand side and boundary rows, then the Krylov solve to a relative FP64
residual of 1e-14.  The default workload is the 2D channel 512x96
(98,304 triangles, 445,411 DOF, nu = 1e-3, dt = 1e-3).  Prints one JSON line.
Under torchrun each rank runs an independent replica (the single-mesh path
does not shard); the whole-job value is the steps of all ranks divided by the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NS steps/s & DOF/s vs plain FP64 GPU path; % HBM roofline; p50/p99 latency"
L2_FLUSH_BYTES = 256 << 20  # > 135 MB of L2


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="fs", choices=["fs", "reference"])
    p.add_argument("--workload", default="channel", choices=["channel", "unit_square", "cube"])
    p.add_argument("--precision", default="fp32_refine", choices=["fp32_refine", "fp64"])
    p.add_argument("--fp64-steps", type=int, default=20,
                   help="steps of the plain FP64 path timed for the comparison")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--schedule", default="auto",
                   help="schedule 'V,P[,S,M]' (fused-tail row thresholds of the velocity and "
                        "pressure hierarchies, SpMV and smoothing slot-group depths), or 'auto' "
                        "to run the autotuner at set-up; fix it when a profiler distorts the "
                        "autotuner's timings")
    p.add_argument("--coarse-degree", type=int, default=0, choices=[0, 2, 3],
                   help="Chebyshev degree of the smoothing below the finest multigrid level "
                        "(0: the library default, 2)")
    p.add_argument("--fine-degree", type=int, default=0, choices=[0, 2, 3],
                   help="Chebyshev degree on the finest multigrid level (0: the library "
                        "default, 2)")
    p.add_argument("--smoother-ratios", default="4,6,8,12,16",
                   help="candidate Chebyshev interval ratios the smoother tuner times at "
                        "set-up on every workload, after the degree pairs (2,2), (1,2), (2,1), "
                        "(1,1) ('' keeps the library defaults: ratio 8, degree 2)")
    p.add_argument("--smoother", default="",
                   help="fixed smoother 'COARSE,FINEST,RATIO' (degrees and Chebyshev interval "
                        "ratio) instead of the set-up tuner, for profiler runs, under which the "
                        "tuner's step timings are distorted")
    p.add_argument("--smoother-steps", type=int, default=5,
                   help="steps the smoother autotuner times per candidate (channel; the "
                        "cube and the batch take 3)")
    p.add_argument("--serial-launches", type=int, default=0, choices=[0, 1],
                   help="1: plain serialised kernel launches instead of programmatic dependent "
                        "launches (the library default)")
    p.add_argument("--no-graph", action="store_true",
                   help="launch the solver's kernels one by one instead of replaying captured "
                        "CUDA graphs (for per-kernel profilers, which cannot see kernels inside "
                        "graphs with conditional nodes)")
    p.add_argument("--roofline-kernel", default="cgs_upd", choices=sorted(KERNELS),
                   help="kernel of the roofline line: the largest single kernel of the "
                        "channel step's ncu launch list (the CGS2 update pass)")
    p.add_argument("--batch-steps", type=int, default=20,
                   help="timed steps of the 96-instance batched workload (0: skip)")
    p.add_argument("--cube-steps", type=int, default=10,
                   help="timed FP32+refinement steps of the cube 48^3 (0: skip)")
    p.add_argument("--cube-fp64-steps", type=int, default=5,
                   help="timed FP64 steps of the cube 48^3")
    p.add_argument("--serve-requests", type=int, default=96,
                   help="requests of each serving run (0: skip)")
    p.add_argument("--serve-rate", type=float, default=200.0,
                   help="mean arrival rate of the saturation run (requests/s)")
    p.add_argument("--ipcs-steps", type=int, default=10,
                   help="timed IPCS steps of the 256x256 unit square (0: skip)")
    p.add_argument("--picard", type=int, default=1,
                   help="time the steady Picard solve of the Sec. 3.3 example (0: skip)")
    p.add_argument("--cpu-baseline-steps", type=int, default=1,
                   help="full oracle steps of the workload timed for cpu_baseline")
    return p.parse_args(argv)


# kernels timed by fs_profile_kernel: name -> (id attribute, description)
KERNELS = {
    "spmv": ("FS_KERNEL_SPMV", "k_spmv_full (saddle-point SpMV, SELL-32, solver arithmetic)"),
    "spmv_fp64": ("FS_KERNEL_SPMV_FP64", "k_spmv_full (FP64, refinement residual)"),
    "cheb": ("FS_KERNEL_CHEB", "k_mg (Chebyshev step, finest P2 level, SELL-32)"),
    "assemble": ("FS_KERNEL_ASSEMBLE_CONV", "k_assemble_conv (per-step convection, FP64)"),
    "cgs_dot": ("FS_KERNEL_CGS_DOT", "k_seg_dot (CGS2 dots h = V^T w, j = 15)"),
    "cgs_upd": ("FS_KERNEL_CGS_UPD", "k_seg_upd (CGS2 update w -= V h, re-dot, norm; j = 15)"),
    "cgs_fin": ("FS_KERNEL_CGS_FIN", "k_seg_fin (CGS2 final update and normalisation; j = 15)"),
}


SMOOTHER_DEGREES = ((2, 2), (1, 2), (2, 1), (1, 1))


FIXED_SMOOTHER = None  # (coarse degree, finest degree, ratio) from --smoother


def tune_smoother(fs, S, ratios, nsteps):
    """Set-up, untimed: the smoother's degrees (coarse levels, finest level)
    and then its Chebyshev interval, each picked by timing `nsteps` steps
    from the problem's current state under every candidate (the library
    restores the state afterwards); or the fixed smoother of --smoother."""
    if FIXED_SMOOTHER:
        c, f, r = FIXED_SMOOTHER
        return fs.fs_autotune_smoother(S.prob, [(r, c, f)], nsteps=1)["best"]
    if not ratios:
        return None
    return fs.fs_tune_smoother(S.prob, nsteps=nsteps, degrees=SMOOTHER_DEGREES, ratios=ratios)


def parse_ratios(text):
    return tuple(int(q) for q in text.split(",") if q.strip())


def workload(name):
    import fs_workloads as W
    return {"channel": W.C2, "unit_square": W.C1, "cube": W.C3}[name]


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms (reads only)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["smax"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def traffic_from_profiles(kernel, wl_name):
    """DRAM bytes per launch from the committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        for line in open(path):
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel \
                    and parts[1] == wl_name:
                return float(parts[2])
    except OSError:
        pass
    return None


# ---------------------------------------------------------------------------
def oracle_full_step(wl):
    """One full oracle step of the workload at its own size, single-threaded:
    COO assembly, right-hand side and boundary rows, then the sparse direct
    solve with FP64 refinement (ILU(0)-GMRES stagnates on the do-nothing
    channel).  Returns seconds."""
    from oracle import oracle as O
    P = O.Problem(dim=wl.dim, n=wl.n, lo=wl.lo, hi=wl.hi, problem=wl.problem, nu=wl.nu,
                  dt=wl.dt, jitter=wl.jitter, seed=wl.seed, side_mask=wl.side_mask,
                  pin_p0=wl.pin_p0, init=wl.init)
    t0 = time.perf_counter()
    P.step(rtol=1e-14, method="lu")
    return time.perf_counter() - t0


def reference_arm(args, rank):
    """The oracle on the host cores as the reference arm.  Each timed step is
    one full oracle step of the workload at its full size (about a minute on
    one core), so at most two are timed; the warm-up loads the oracle once
    on a small channel (the CPU program has nothing else to warm)."""
    if rank != 0:
        return 0
    import fs_workloads as W
    wl = workload(args.workload)
    from oracle import oracle as O
    O.build()
    if args.warmup > 0:
        oracle_full_step(W.channel(16, 4))
    k = max(1, min(args.steps, 2))
    secs = [oracle_full_step(wl) for _ in range(k)]
    total = sum(secs)
    value = k / total
    sample = (f"{k} full oracle steps of {wl.name} ({wl.ndof} DOF; COO assembly + sparse LU "
              f"with FP64 refinement to 1e-14), single-threaded; {args.steps} requested, at "
              f"most 2 timed so the run ends within minutes")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": k, "steps_requested": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / k, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "ndof": wl.ndof, "cells": wl.ncell, "nu": wl.nu,
                   "dt": wl.dt, "rtol": 1e-14},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def aggregate_time(total_s, dist):
    """Slowest rank's time (the whole job runs until its last rank ends)."""
    if dist is None:
        return total_s
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([total_s], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
def batched_run(torch, fs, steps, warmup=3, opts=None, ratios=()):
    """The batched workload: 96 unit-square instances, N and Re drawn
    log-uniform from the seed, one problem over their union (one launch per
    phase for all instances), FP32 inner / FP64 refinement."""
    import fs_workloads as W
    import numpy as np
    wls = W.batched_instances()
    t0 = time.perf_counter()
    B = fs.Stepper.from_workloads(wls, precision=fs.FS_PREC_FP32_REFINE)
    setup_s = time.perf_counter() - t0
    try:
        tune = fs.fs_autotune(B.prob, reps=3)
        smoother = tune_smoother(fs, B, ratios, 3)
        for _ in range(warmup):
            fs.fs_step(B.prob, 1, opts)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.cuda.nvtx.range_push("batch_step")  # profilers can select these steps
            fs.fs_step(B.prob, 1, opts)
            torch.cuda.nvtx.range_pop()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = fs.fs_instance_stats(B.prob)
        ndof = B.info["n_dof"]
    finally:
        B.close()
    per_step = sum(ms) / len(ms) / 1e3
    return {"workload": "96 unit squares, N log-uniform [16,256], Re log-uniform [1,2000], "
                        "dt 1e-3, seed 0", "instances": len(wls), "ndof_total": ndof,
            "ms_per_step": 1e3 * per_step, "steps_per_s": 1.0 / per_step,
            "instance_steps_per_s": len(wls) / per_step, "dof_per_s": ndof / per_step,
            "setup_s": setup_s, "timed_steps": steps, "schedule": tune, "smoother": smoother,
            "iters_max": max(x["iters"] for x in st),
            "iters_median": float(np.median([x["iters"] for x in st])),
            "status_ok": all(x["status"] == 0 for x in st),
            "rel_res_max": max(x["rel_res"] for x in st)}


def serving_run(fs, count, rate, budget=150 << 30, slots=32):
    """The first `count` requests of the seeded serving stream (2D N
    log-uniform in [16,512], 3D N in [8,48], Re in [1,2000], 10-100 steps,
    Bernoulli(1/2) 2D/3D, exponential gaps at `rate` requests/s), admitted by
    the native loop under the HBM budget; latency = completion - arrival on
    the wall clock."""
    import fs_workloads as W
    import numpy as np
    reqs = W.serving_requests(count=count, rate=rate)
    srv = fs.Server(budget, slots)
    try:
        t0 = time.perf_counter()
        pending = list(reqs)
        done = []
        peak = 0
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.pop(0)
                srv.submit(r.workload, r.workload.steps, r.arrival)
            srv.progress(now)
            done += srv.completed()
            peak = max(peak, srv.status()["bytes_reserved"])
            if time.perf_counter() - t0 > 900:
                break
        span = time.perf_counter() - t0
    finally:
        srv.close()
    lat = np.array([d["finished"] - d["arrival"] for d in done])
    steps = sum(d["nsteps"] for d in done)
    byid = {r.rid: r for r in reqs}
    dofsteps = sum(byid[d["id"] - 1].workload.ndof * d["nsteps"] for d in done)
    return {"requests": len(reqs), "completed": len(done),
            "ok": sum(1 for d in done if d["status"] == 0), "rate_per_s": rate,
            "latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "requests_per_s": len(done) / span, "steps_per_s": steps / span,
            "dof_steps_per_s": dofsteps / span, "makespan_s": span,
            "hbm_budget_gb": budget / 2**30, "peak_reserved_gb": peak / 2**30, "slots": slots,
            "mean_ndof": float(np.mean([r.workload.ndof for r in reqs])),
            "mean_steps": float(np.mean([r.workload.steps for r in reqs]))}


def serving_block(fs, count, rate):
    """Saturation run at the stream's own rate, then the same requests at a
    sustainable rate (70% of the measured saturation request rate)."""
    sat = serving_run(fs, count, rate)
    sus_rate = 0.7 * sat["requests_per_s"]
    sus = serving_run(fs, count, sus_rate)
    return {"workload": f"first {count} requests of the seeded stream: Poisson arrivals, 2D N "
                        f"log-uniform [16,512] / 3D N [8,48] (Bernoulli 1/2), Re log-uniform "
                        f"[1,2000], 10-100 steps, dt 1e-3, FP32 inner / FP64 refinement, "
                        f"HBM budget 150 GB, seed 0",
            "saturation": sat, "sustainable": sus}


def ipcs_block(torch, fs, stream, flush, steps, warmup=3):
    """Incremental pressure correction (three FP64 CG solves per step) on the
    256x256 unit square with the Sec. 4.1 solution, nu = 1e-2, dt = 1e-3,
    beside the coupled Oseen step (FP32 inner / FP64 refinement) of the same
    workload."""
    import fs_workloads as W
    import numpy as np
    wl = W.unit_square(256, jitter=0.0, nu=1e-2, dt=1e-3)
    out = {"workload": wl.name, "ndof": wl.ndof, "nu": wl.nu, "dt": wl.dt, "timed_steps": steps}
    S = fs.Stepper.from_workload(wl, precision=fs.FS_PREC_FP64, stream=stream.cuda_stream)
    try:
        fs.fs_step_ipcs(S.prob, warmup)
        ms, its = [], []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            stream.synchronize()
            t0 = time.perf_counter()
            st = fs.fs_step_ipcs(S.prob, 1)[0]   # synchronises
            ms.append(1e3 * (time.perf_counter() - t0))
            its.append(st["iters"])
        out["ipcs"] = {"steps_per_s": 1e3 * len(ms) / sum(ms), "ms_per_step": sum(ms) / len(ms),
                       "cg_iters_per_stage": [float(np.mean([i[k] for i in its]))
                                              for k in range(3)],
                       "timing": "host wall clock around the synchronising call"}
    finally:
        S.close()
    S = fs.Stepper.from_workload(wl, precision=fs.FS_PREC_FP32_REFINE, stream=stream.cuda_stream)
    try:
        for _ in range(warmup):
            fs.fs_step(S.prob, 1)
        t, st = time_steps(torch, fs, S, stream, steps, flush)
        out["coupled_fp32_refine"] = {"steps_per_s": 1e3 * len(t) / sum(t),
                                      "ms_per_step": sum(t) / len(t),
                                      "iters_per_step": float(np.mean([q["iters"] for q in st]))}
    finally:
        S.close()
    return out


def picard_block(fs, n=64):
    """The steady example of Sec. 3.3 (nu = 1, no time derivative) on an
    n x n square: Picard iteration to 1e-10 from zero, each linear solve
    FP32 inner / FP64 refinement to 1e-12 (without the mass term the system
    is far worse conditioned than a time step's)."""
    import math
    import numpy as np
    import fs_workloads as W
    wl = W.unit_square(n, problem=W.STEADY_POLY, jitter=0.0, nu=1.0, dt=math.inf)
    S = fs.Stepper.from_workload(wl, precision=fs.FS_PREC_FP32_REFINE)
    try:
        x0, t0 = S.state()
        fs.fs_set_state(S.prob, np.zeros_like(x0), t0)
        t = time.perf_counter()
        st = fs.fs_solve_steady(S.prob, nl_tol=1e-10, opts=fs.fs_default_solve_opts(rtol=1e-12),
                                raise_on_error=False)
        secs = time.perf_counter() - t
    finally:
        S.close()
    return {"workload": f"steady example (Sec. 3.3) on {wl.name}, nu = 1", "ndof": wl.ndof,
            "seconds": secs, "status": st["status"], "picard_iters": st["picard_iters"],
            "krylov_iters": st["krylov_iters"], "update": st["update"],
            "rel_res": st["rel_res"]}


def cube_block(torch, fs, stream, flush, steps, steps64, warmup=3, ratios=()):
    """The cube 48^3 (2,855,668 DOF): FP32+refinement and FP64 steps/s, the
    per-step difference between the two paths' states, and the L2-cold
    fractions of its SpMV and smoothing step (working sets above the L2)."""
    import fs_workloads as W
    import numpy as np
    wl = W.C3
    out = {"workload": wl.name, "ndof": wl.ndof, "cells": wl.ncell, "nu": wl.nu, "dt": wl.dt}
    res = {}
    states = {}
    for prec, k in ((fs.FS_PREC_FP32_REFINE, steps), (fs.FS_PREC_FP64, steps64)):
        S = fs.Stepper.from_workload(wl, precision=prec, stream=stream.cuda_stream)
        try:
            fs.fs_autotune(S.prob, reps=3)
            smoother = tune_smoother(fs, S, ratios, 3)
            xs = []
            for _ in range(warmup):
                fs.fs_step(S.prob, 1)
                xs.append(fs.fs_get_state(S.prob)[0])
            t, st = time_steps(torch, fs, S, stream, k, flush)
            name = "fp32_refine" if prec == fs.FS_PREC_FP32_REFINE else "fp64"
            res[name] = {"steps_per_s": 1e3 * len(t) / sum(t), "ms_per_step": sum(t) / len(t),
                         "timed_steps": k, "dof_per_s": 1e3 * len(t) * wl.ndof / sum(t),
                         "iters_per_step": float(np.mean([q["iters"] for q in st])),
                         "rel_res_max": max(q["rel_res"] for q in st), "smoother": smoother}
            states[name] = xs
            if prec == fs.FS_PREC_FP32_REFINE:
                peak, kind = measured_peak_hbm()
                kern = {}
                for kname in ("spmv", "cheb"):
                    ms, by = fs.fs_profile_kernel(S.prob, getattr(fs, KERNELS[kname][0]),
                                                  reps=10, cold=True)
                    kern[kname] = {"ms_cold": ms, "alg_bytes": by, "gbs": by / ms / 1e6,
                                   "frac": by / ms / 1e6 / peak}
                out["kernels_l2_cold"] = kern
        finally:
            S.close()
    out.update(res)
    out["vs_fp64_path"] = res["fp32_refine"]["steps_per_s"] / res["fp64"]["steps_per_s"]
    # the two paths' states after each of the warm-up steps (same steps,
    # both stopped at a relative residual of 1e-14)
    out["per_step_rel_l2_fp32_refine_vs_fp64"] = [
        float(np.linalg.norm(a - b) / np.linalg.norm(b))
        for a, b in zip(states["fp32_refine"], states["fp64"])]
    out["oracle_parity"] = ("per-step parity against the oracle is tested on the 16^3 cube "
                            "(5 free-running steps, rel L2 <= 1e-9) and on the 512x96 channel "
                            "(tests/test_gpu_fullsize_parity.py); at 48^3 the test checks "
                            "sampled rows and the FP64 residual")
    return out


# ---------------------------------------------------------------------------
def time_steps(torch, fs, S, stream, steps, flush, opts=None):
    """Per-step CUDA-event times (ms) of fs_step on the problem's stream;
    L2 flushed (256 MB write) before each step, outside the timed window."""
    out = []
    stats = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = fs.fs_step(S.prob, 1, opts)[0]
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
        stats.append(st)
    return out, stats


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)

    import numpy as np
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the CUDA path has no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__ as G
    G.build()
    import fs_workloads as W
    from paper_2605_25403_gb300 import fs

    wl = workload(args.workload)
    ratios = parse_ratios(args.smoother_ratios)
    global FIXED_SMOOTHER
    if args.smoother:
        FIXED_SMOOTHER = tuple(int(q) for q in args.smoother.split(","))
    prec = fs.FS_PREC_FP32_REFINE if args.precision == "fp32_refine" else fs.FS_PREC_FP64
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # ---- plain FP64 GPU path (the in-repo baseline) ----------------------
    fp64 = None
    k64 = args.fp64_steps
    if prec != fs.FS_PREC_FP64 and k64 > 0:
        S64 = fs.Stepper.from_workload(wl, precision=fs.FS_PREC_FP64, stream=stream.cuda_stream)
        fs.fs_set_schedule(S64.prob, 0, 0, 0, 0, args.coarse_degree, args.serial_launches,
                           fine_degree=args.fine_degree)
        tune64 = fs.fs_autotune(S64.prob, reps=5)
        smooth64 = tune_smoother(fs, S64, ratios, args.smoother_steps)
        for _ in range(args.warmup):
            fs.fs_step(S64.prob, 1)
        t64, st64 = time_steps(torch, fs, S64, stream, k64, flush)
        fp64 = {"steps_per_s": 1e3 * len(t64) / sum(t64),
                "ms_per_step": sum(t64) / len(t64),
                "step_ms_p50": float(np.percentile(t64, 50)),
                "step_ms_max": float(max(t64)),
                "iters_per_step": float(np.mean([s["iters"] for s in st64])),
                "iters_max": int(max(s["iters"] for s in st64)),
                "cycles_per_step": float(np.mean([s["cycles"] for s in st64])),
                "rel_res_max": max(s["rel_res"] for s in st64), "schedule": tune64,
                "smoother": smooth64}
        S64.close()

    # ---- the timed path ----------------------------------------------------
    S = fs.Stepper.from_workload(wl, precision=prec, stream=stream.cuda_stream)
    # set-up, untimed: pick the multigrid schedule by timing the candidates
    if args.schedule == "auto":
        fs.fs_set_schedule(S.prob, 0, 0, 0, 0, args.coarse_degree, args.serial_launches,
                           fine_degree=args.fine_degree)
        tune = fs.fs_autotune(S.prob, reps=5)
    else:
        fs.fs_set_schedule(S.prob, *(int(q) for q in args.schedule.split(",")))
        tune = {"fixed": fs.fs_get_schedule(S.prob)}
    smoother = tune_smoother(fs, S, ratios, args.smoother_steps)
    for _ in range(args.warmup):
        fs.fs_step(S.prob, 1)
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = fs.fs_launch_count()
    opts = fs.fs_default_solve_opts(use_graph=0) if args.no_graph else None
    torch.cuda.nvtx.range_push("bench_timed")  # profilers can select the timed steps
    times, stats = time_steps(torch, fs, S, stream, args.steps, flush, opts)
    torch.cuda.nvtx.range_pop()
    launches = fs.fs_launch_count() - l0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total_s = aggregate_time(sum(times) / 1e3, dist)
    value = world * args.steps / total_s
    ms_per_step = 1e3 * total_s / args.steps

    # ---- end to end through the C ABI with host buffers --------------------
    # a second problem of the same workload, schedule and warm-up, so that
    # its steps cover the same window of the run as the device-timed ones
    # (the solves' starting guesses extrapolate the state history, so later
    # steps of a transient can be cheaper)
    ndof = S.info["n_dof"]
    sched = fs.fs_get_schedule(S.prob)
    SE = fs.Stepper.from_workload(wl, precision=prec, stream=stream.cuda_stream)
    fs.fs_set_schedule(SE.prob, sched["tail_rows_velocity"], sched["tail_rows_pressure"],
                       sched["spmv_group"], sched["smooth_group"], sched["coarse_degree"],
                       sched["serial_launches"], sched["persistent_precond"],
                       sched["fine_degree"], sched["cheb_ratio"], sched["schur"])
    for _ in range(max(0, args.warmup - 1)):
        fs.fs_step(SE.prob, 1)
    xh = torch.empty(ndof, dtype=torch.float64).pin_memory()
    xn = xh.numpy()
    x0, t0 = fs.fs_get_state(SE.prob)
    xn[:] = x0
    tcur = t0
    e2e_ms = []
    e2e_iters = []
    # the first pass (the last warm-up step) is not timed: the timed passes
    # are steps warmup+1 .. warmup+steps, as on the device-timed path
    for k in range(args.steps + 1):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fs.fs_set_state(SE.prob, xn, tcur)                # H2D of the step's input
        st = fs.fs_step(SE.prob, 1)[0]
        x_new, tcur = fs.fs_get_state(SE.prob)           # D2H of the step's result
        e1.record(stream)
        e1.synchronize()
        xn[:] = x_new
        if k > 0:
            e2e_ms.append(e0.elapsed_time(e1))
            e2e_iters.append(st["iters"])
    e2e_val = world * len(e2e_ms) / (sum(e2e_ms) / 1e3)
    SE.close()

    # ---- roofline of the dominant kernel ----------------------------------
    # every hot kernel timed on the timed problem's own data and stream, warm
    # (back-to-back launches) and with a cold L2 (each launch after a read of
    # twice the L2 size); the roofline takes the cold figure
    peak, peak_kind = measured_peak_hbm()
    kernels = {}
    for name, (attr, desc) in KERNELS.items():
        kid = getattr(fs, attr)
        ms, by = fs.fs_profile_kernel(S.prob, kid, reps=20)
        msc, _ = fs.fs_profile_kernel(S.prob, kid, reps=20, cold=True)
        kernels[name] = {"ms": ms, "ms_cold": msc, "alg_bytes": by, "gbs": by / ms / 1e6,
                         "gbs_cold": by / msc / 1e6, "frac_cold": by / msc / 1e6 / peak}
    kernels["precond"] = {"ms": fs.fs_profile_kernel(S.prob, fs.FS_KERNEL_PRECOND, reps=10)[0],
                          "unit": "one block-preconditioner application (graph of 10)"}
    kname = args.roofline_kernel
    achieved = kernels[kname]["gbs_cold"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind, "kernel": KERNELS[kname][1],
                "timing": "L2-cold, each launch after a read of twice the L2 size, CUDA events "
                          "on the problem's stream",
                "traffic": traffic_from_profiles(kname, wl.name)}

    # ---- CPU baseline: the oracle on a bounded sample ---------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.cpu_baseline_steps > 0:
        k = args.cpu_baseline_steps
        secs = sum(oracle_full_step(wl) for _ in range(k))
        cpu = {"value": k / secs, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{k} full oracle step(s) of {wl.name} ({wl.ndof} DOF: COO assembly, "
                         f"right-hand side, boundary rows, sparse LU with FP64 refinement to "
                         f"1e-14) in {secs:.1f} s, single-threaded plain C + SuperLU"}

    S.close()

    def block(enabled, fn, *a):
        """A secondary workload: its result, or the error that stopped it (the
        headline line is printed either way)."""
        if not enabled:
            return None
        try:
            return fn(*a)
        except Exception as e:  # noqa: BLE001 - recorded in the JSON line
            return {"error": f"{type(e).__name__}: {e}"}

    batch = block(args.batch_steps > 0, batched_run, torch, fs, args.batch_steps, 3, opts,
                  ratios)
    cube = block(args.cube_steps > 0, cube_block, torch, fs, stream, flush, args.cube_steps,
                 args.cube_fp64_steps, 3, ratios)
    serving = block(args.serve_requests > 0, serving_block, fs, args.serve_requests,
                    args.serve_rate)
    ipcs = block(args.ipcs_steps > 0, ipcs_block, torch, fs, stream, flush, args.ipcs_steps)
    picard = block(args.picard > 0, picard_block, fs)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    iters = [s["iters"] for s in stats]
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp32+fp64" if prec == fs.FS_PREC_FP32_REFINE else "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "ndof": ndof, "cells": wl.ncell, "nu": wl.nu,
                   "dt": wl.dt, "precision": args.precision, "rtol": 1e-14,
                   "l2": "flushed before every timed step and every e2e step (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "graphs": not args.no_graph},
        "dof_per_s": value * ndof,
        "step_ms_p50": statistics.median(times),
        "step_ms_p99": float(np.percentile(times, 99)),
        "iters_per_step": float(np.mean(iters)),
        "refinements_per_step": float(np.mean([s["refinements"] for s in stats])),
        "cycles_per_step": float(np.mean([s["cycles"] for s in stats])),
        "rel_res_max": max(s["rel_res"] for s in stats),
        "fp64_path": fp64,
        "vs_fp64_path": (value / world) / fp64["steps_per_s"] if fp64 else None,
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": "steps/s", "h2d_bytes_per_step": 8 * ndof,
                "d2h_bytes_per_step": 8 * ndof},
        "e2e_iters_per_step": float(np.mean(e2e_iters)),
        "gpu_launches": launches,
        "schedule": tune, "smoother": smoother,
        "roofline": roofline,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "batched": batch,
        "cube": cube,
        "serving": serving,
        "ipcs": ipcs,
        "picard_steady": picard,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
