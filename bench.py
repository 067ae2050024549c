#!/usr/bin/env python
"""Benchmark of the fused D2Q9 stream + collide + sensor step (MLUPS and HBM roofline).

Workload: 4096 x 4096 periodic D2Q9 lattice in FP32, tau = 0.6, seeded smooth density /
velocity perturbations (max |drho| = 1e-2, max |u| = 0.1 c_s) on a density step
rho_L / rho_R = 2 at x = 2048; every step is an output step: Knudsen sensor tagged
against 1e-3 (refine flag), non-equilibrium sensor against 1e-4 (switch flag), the
Kullback-Leibler sensor field stored, per-tile (16 x 16) tag counts and FP64
conservation sums.  The timed region is one kss_step(K) call: K such steps in one
cooperative multi-step launch (each block of a step waits only for its neighbours'
previous step); the same steps as one launch each are timed alongside.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload batch64    # the batched workload (below)
  python bench.py --workload adjoint512 # the adjoint workload (below)
  python bench.py --workload fp16dev8192 [--fp16-error]  # the precision workload (below)
  python bench.py --workload aar4096    # adaptive algorithm refinement (below)
  python bench.py --workload shear128   # the FP64 correctness case (below)

Batched workload (--workload batch64): 64 uneven periodic lattices (sizes 64^2 ..
1024^2, tau ~ U[0.51, 1.5], Mach ~ U[0.01, 0.15], seed 13618, 15.8 M cells in all), the
same sensors, flags and sums every step, advanced by one launch per step for all of
them (replayed as a CUDA graph), against the same 64 lattices stepped one launch per
lattice per step.

Adaptive-algorithm-refinement workload (--workload aar4096): the same 4096^2 lattice
with the two-relaxation model in the switched region (tau2 = 1/2 + (3/16)/(tau - 1/2)):
output steps with the {Kn, KL, neq} set and neq as the switch sensor (the region then
follows the flags), the same with the quasi-equilibrium sensor as the switch, all of
Table 1 with that switch, and plain steps in a fixed 40 % region, each against the same
steps with BGK only.

Correctness workload (--workload shear128): the decaying shear wave on a 128^2 FP64
lattice (u_x = 0.01 sin(2 pi y / 128), tau = 0.8), 2000 steps in one call with the Kn and
KL sensors, flags (Kn > 1e-3), tile counts and sums every 10 steps.  The lattice (1.2 MB per
buffer) lives in L2, so its rate is reported as it is, with no bandwidth fraction.

N > 1 (launched by torchrun) runs one independent lattice per rank (replicas, weak
scaling); rank 0 prints one JSON line.  --impl reference times the CPU oracle on the
host cores on a bounded window of the same workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 4096
TAU = 0.6
THR_R, THR_S = 1e-3, 1e-4
TILE = 16
# algorithmic bytes per lattice update of the fused FP32 output step:
# 9 population loads + 9 stores (4 B each) + the KL sensor value (4 B) + the flag byte
BYTES_PER_LUP = 9 * 4 + 9 * 4 + 4 + 1
METRIC = "MLUPS with sensors fused and % of HBM roofline, 1xGB300"
WORKLOAD = ("D2Q9 FP32 4096x4096 periodic, tau=0.6, smooth perturbations (amp 1e-2, "
            "Mach<=0.1) + density step 2:1 at x=2048; fused stream+collide+sensors "
            "(Kn refine 1e-3, neq switch 1e-4, KL field) + flags + tile counts + sums "
            "every step")
CSRC = os.path.join(ROOT, "paper_2603_13618_gb300", "csrc")
PROFILE = os.path.join(ROOT, "profiles", "step_std_f32_4096.md")


def kernel_hash() -> str:
    """sha256 (first 16 hex digits) over every file of the CUDA sources (kernels, launch
    decisions, runtimes), by name in sorted order: any edit there changes it."""
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        path = os.path.join(CSRC, name)
        if os.path.isfile(path):
            h.update(name.encode() + b"\0")
            with open(path, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(path=PROFILE):
    """DRAM bytes per step of the fused step from a committed ncu summary, or None if
    the summary is missing or was taken on different kernel sources."""
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]{16})", txt)
    t = re.search(r"dram_bytes_per_step:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != kernel_hash():
        return None
    return float(t.group(1))


def kernel_name(choice: str) -> str:
    tma = choice == "tma"
    return ("step_tma_kernel<float, MODE_STD> (bulk-copy staged), one launch per step" if tma
            else "step_kernel_multi<float, MODE_STD> (each warp's next row staged in shared "
                 "memory by cp.async; all steps in one cooperative launch, blocks waiting on "
                 "their neighbours' previous step)")


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during timing (and, for
    the headline, during about a second of the same untimed launches after it)."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def workload_fields(nx=NX, ny=NY, x0=0, y0=0, wx=None, wy=None):
    from paper_2603_13618_gb300 import inputs

    return inputs.smooth_jump(NX, NY, seed=2603, kmax=8, x0=x0, y0=y0, wx=wx, wy=wy)


def _oracle_rate(f, seconds, threads, max_steps=1 << 30):
    """Fused oracle steps ({Kn, KL, neq}: Kn refine, neq switch, KL field, flags, tile
    counts, sums, collide) on the state f for about `seconds`; (MLUPS, steps, s)."""
    import oracle

    oracle.set_threads(threads)
    try:
        steps, t0 = 0, time.perf_counter()
        while steps < max_steps:
            oracle.run(f, TAU, 1, oracle.SENSOR_ID["kn"], THR_R, oracle.SENSOR_ID["neq"], THR_S,
                       TILE, full=False)
            steps += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                break
    finally:
        oracle.set_threads(1)
    return f.shape[1] * f.shape[2] * steps / el / 1e6, steps, el


def cpu_baseline(seconds: float = 8.0, window: int = 1024):
    """The oracle as it stands on a window of the workload, with the GPU headline's
    sensor set: on all host cores (the reported value) and on one thread."""
    import oracle

    rho, ux, uy = workload_fields(x0=NX // 2 - window // 2, y0=NY // 2 - window // 2,
                                  wx=window, wy=window)
    f = oracle.init_equilibrium(rho, ux, uy)
    cores = oracle.host_cores()
    threads = cores if oracle.lib().orc_have_openmp() else 1
    v1, n1, t1 = _oracle_rate(f, seconds, 1)
    vn, nn, tn = _oracle_rate(f, seconds, threads)
    return {"value": vn, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"{nn} fused oracle step(s) ({{Kn, KL, neq}}: Kn refine 1e-3, neq switch "
                      f"1e-4, KL field, flags, tile counts, sums) on the central "
                      f"{window}x{window} window of the workload, {tn:.1f} s, {threads} "
                      f"threads (row sweeps split over the host cores)",
            "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1,
                              "sample": f"{n1} step(s) of the same, {t1:.1f} s, 1 thread"}}


BATCH_METRIC = "MLUPS with sensors fused, 64 uneven lattices batched, 1xGB300"


def run_batch(args):
    """The batched workload: 64 uneven lattices, all K steps in one cooperative launch
    (against one launch per step, as a graph and directly, and one lattice at a time)."""
    import torch

    from paper_2603_13618_gb300 import inputs, kss

    torch.cuda.set_device(0)
    specs = inputs.batch_specs()
    cells = sum(s * s for s, _, _, _ in specs)
    b = kss.Batch([dict(nx=s, ny=s, tau=tau) for s, tau, _, _ in specs], precision="fp32",
                  refine_sensor="kn", refine_threshold=THR_R, switch_sensor="neq",
                  switch_threshold=THR_S, record=("kl",), output_every=1, tile=TILE,
                  stream="torch")
    for k, (s, _, mach, fs) in enumerate(specs):
        b[k].set_fields(*inputs.batch_fields(s, mach, fs))
    if args.batch_rows:  # a fixed decomposition (profiling captures): multi-step launch
        b.set_tuning(rows=args.batch_rows, ctas_per_sm=0, graph=1, multi_step=1)
        tuning = b.tuning
    else:
        tuning = b.autotune(None, steps=20) if not args.no_tune else b.tuning
    stream = torch.cuda.current_stream()
    K = args.steps
    b.step(args.warmup)
    b.step(K)          # records the K-step graph for both buffer parities
    b.step(K)
    torch.cuda.synchronize()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    with ClockSampler(0) as clk:
        total_ms = timed(lambda: b.step(K))
    clocks = clk.summary()
    value = cells * K / (total_ms * 1e-3) / 1e6
    multi = bool(b.tuning["multi_step"])
    # the multi-step launch at each CTA height (the tuner times per-step launches)
    multi_rows = {}
    for rows in (16, 32, 64):
        b.set_tuning(rows=rows, ctas_per_sm=0, graph=1, multi_step=1)
        b.step(args.warmup)
        multi_rows[rows] = timed(lambda: b.step(K)) / K
    # the same steps as one launch per step: a captured graph, then direct launches
    b.set_tuning(rows=tuning["rows"], ctas_per_sm=tuning["ctas_per_sm"], graph=1,
                 multi_step=0)
    b.step(K)
    b.step(K)
    graph_ms = timed(lambda: b.step(K))
    b.set_tuning(rows=tuning["rows"], ctas_per_sm=tuning["ctas_per_sm"], graph=0,
                 multi_step=0)
    direct_ms = timed(lambda: b.step(K))
    # the 64 lattices stepped one at a time: one launch per lattice per step
    ks = max(4, K // 10)

    def separate():
        for k in range(len(specs)):
            b[k].step(ks)

    separate()
    sep_ms = timed(separate)
    sep_value = cells * ks / (sep_ms * 1e-3) / 1e6
    peak, peak_kind = measured_peak()
    kern_ms = total_ms / K
    achieved = BYTES_PER_LUP * cells / (kern_ms * 1e-3) / 1e9
    line = {
        "metric": BATCH_METRIC, "value": value, "unit": "MLUPS", "n_gpus": 1, "steps": K,
        "warmup": args.warmup, "ms_per_step": kern_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "64 periodic D2Q9 FP32 lattices, sizes from {64..1024}^2, "
                               "tau ~ U[0.51,1.5], Mach ~ U[0.01,0.15], seed 13618; Kn "
                               "refine 1e-3, neq switch 1e-4, KL field, flags, tile "
                               "counts and sums every step",
                   "cells": cells, "lattices": len(specs), "tuning": tuning,
                   "l2": "inputs larger than L2: 1.14 GB of populations per step"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": profile_traffic(BATCH_PROFILE) if multi else None,
                     "algorithmic_bytes_per_launch": BYTES_PER_LUP * cells,
                     "kernel_ms": kern_ms,
                     "kernel": ("batch_kernel_multi<float, MODE_STD> (all steps in one "
                                "cooperative launch, rows staged in shared memory by "
                                "cp.async)" if multi
                                else "batch_step_kernel<float, MODE_STD>")},
        "multi_step_ms_by_rows": multi_rows,
        "graph_of_per_step_launches": {"value": cells * K / (graph_ms * 1e-3) / 1e6,
                                       "unit": "MLUPS", "ms_per_step": graph_ms / K},
        "direct_launches": {"value": cells * K / (direct_ms * 1e-3) / 1e6, "unit": "MLUPS",
                            "ms_per_step": direct_ms / K},
        "separate_lattices": {"value": sep_value, "unit": "MLUPS", "steps": ks,
                              "ms_per_step": sep_ms / ks,
                              "launches_per_step": len(specs)},
        "speedup_vs_separate": value / sep_value,
        "gpu_launches": 1 if multi else K,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    b.close()
    return 0


ADJ_METRIC = "adjoint MLUPS (forward with checkpoints + reverse sweep), 1xGB300"


def adjoint_roofline(n, N, E, ms):
    """Algorithmic bytes of one gradient over its time: the forward's N - 1 plain steps and
    the recomputed ones (72 B/LUP; every segment but the last, whose states the forward
    pass keeps), the N - 1 reverse steps (108 B/LUP: f read, lambda read and written), the
    objective and the projection (72 B/LUP each).  The 512^2 working set (9.4 MB per
    state) lives mostly in L2, so HBM is not the limit: the latency of each dependent
    reverse step is (the cooperative sweep's blocks wait on their neighbours)."""
    peak, kind = measured_peak()
    recompute = 0
    s0 = ((N - 2) // E) * E if N >= 2 else -1
    first = True
    while s0 >= 0:
        if not first:
            recompute += min(s0 + E - 1, N - 2) - s0
        first = False
        s0 -= E
    lups = n * n
    bytes_ = lups * (72 * (N - 1) + 72 * recompute + 108 * (N - 1) + 72 * 2)
    achieved = bytes_ / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": kind, "traffic": None,
            "algorithmic_bytes_per_gradient": bytes_,
            "note": "working set mostly in L2 (512^2: 9.4 MB per state): bound by the latency "
                    "of the dependent reverse steps, not by HBM"}


def adjoint_launches(N, E, multi=True):
    """Kernel launches of one gradient: the forward pass (equilibrium, N - 1 plain steps,
    the last segment's states among them, and the objective), then per segment of the
    reverse sweep, last first: one cooperative launch of its reverse steps that also
    recomputes the previous segment, and the ordered addition of its totals (multi); or
    its recomputed plain steps (all but the last segment) and one launch per reverse step.
    Then the final projection."""
    fwd = 1 + (N - 1) + 1
    bwd = 1
    s0 = ((N - 2) // E) * E if N >= 2 else -1
    first = True
    while s0 >= 0:
        last = min(s0 + E - 1, N - 2)
        if multi:
            bwd += 2
        else:
            bwd += (0 if first else last - s0) + (last - s0 + 1)
        first = False
        s0 -= E
    return fwd + bwd


def run_adjoint(args):
    """The adjoint workload: time(forward + backward) against time(200 plain steps)."""
    import numpy as np
    import torch

    from paper_2603_13618_gb300 import inputs, kss

    torch.cuda.set_device(0)
    n, N, E, tau = 512, 200, 20, 0.6
    r, u, v = inputs.random_smooth(n, n, seed=1361, kmax=8, drho_amp=1e-2, mach=0.1)
    dr, du, dv = (torch.tensor(a, device="cuda") for a in (r, u, v))
    stream = torch.cuda.current_stream()
    adj = kss.Adjoint(n, n, N, precision="fp32", checkpoint_every=E)
    lat = kss.Lattice(n, n, precision="fp32", tau=tau, output_every=0)

    def timed(fn, reps):
        for _ in range(max(1, args.warmup // 10)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def gradient():
        adj.forward(dr, du, dv, tau)
        return adj.backward(device=True)

    def plain():
        lat.set_fields(dr, du, dv)
        lat.step(N)

    reps = max(3, args.steps // 100)
    with ClockSampler(0) as clk:
        t_adj = timed(gradient, reps)
        t_fwd = timed(plain, reps)
    g, gt = gradient()

    # the same gradient with one segment (checkpoint_every = N): the forward pass keeps every
    # state (N x 9.4 MB in HBM), the reverse sweep is one cooperative launch and recomputes
    # nothing; reported beside the workload's checkpoint interval, not in place of it
    adj_all = kss.Adjoint(n, n, N, precision="fp32", checkpoint_every=N)

    def gradient_all():
        adj_all.forward(dr, du, dv, tau)
        return adj_all.backward(device=True)

    t_all = timed(gradient_all, reps)
    g_all, gt_all = gradient_all()
    adj_all.close()
    cells = n * n
    line = {
        "metric": ADJ_METRIC, "value": cells * N / (t_adj * 1e-3) / 1e6, "unit": "MLUPS",
        "n_gpus": 1, "steps": reps, "warmup": max(1, args.warmup // 10),
        "ms_per_step": t_adj / N, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "gradient of the summed KL sensor of step 200 in rho0 and "
                               "tau, 512x512 FP32, checkpoint every 20, tau=0.6, seed 1361",
                   "nx": n, "ny": n, "nsteps": N, "checkpoint_every": E},
        "roofline": adjoint_roofline(n, N, E, t_adj),
        "ms_gradient": t_adj, "ms_forward_plain": t_fwd, "adjoint_over_forward": t_adj / t_fwd,
        "grad_tau": gt, "grad_rho0_norm": float(torch.linalg.vector_norm(g)),
        "gpu_launches_per_gradient": adjoint_launches(N, E, multi=True),
        "gpu_launches_per_gradient_one_launch_per_reverse_step": adjoint_launches(N, E, False),
        "every_state_kept": {"checkpoint_every": N, "ms_gradient": t_all,
                             "adjoint_over_forward": t_all / t_fwd,
                             "state_bytes": 9 * 4 * cells * N,
                             "grad_tau": gt_all,
                             "grad_rho0_max_abs_diff": float((g_all - g).abs().max())},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    adj.close()
    lat.close()
    return 0


FP16_METRIC = "MLUPS with sensors fused, FP16 deviation storage, and % of HBM roofline, 1xGB300"


def run_fp16(args):
    """The precision workload: FP16 deviation storage against FP32 storage."""
    import numpy as np
    import torch

    from paper_2603_13618_gb300 import inputs, kss

    torch.cuda.set_device(0)
    n = args.size or 8192
    amp, tau, kexp = 1e-3, 0.6, 20
    gen = dict(seed=8192, kmax=8, drho_amp=amp, mach=amp / inputs.CS, jump=1.0)
    rho, ux, uy = inputs.smooth_jump(n, n, **gen)
    stream = torch.cuda.current_stream()
    K = args.steps
    peak, peak_kind = measured_peak()
    cells = n * n
    runs = {}
    with ClockSampler(0) as clk:
        for name, prec, out in (("fp16dev", "fp16dev", 1), ("fp32", "fp32", 1),
                                ("fp16dev_plain", "fp16dev", 0), ("fp32_plain", "fp32", 0)):
            lat = kss.Lattice(n, n, precision=prec, tau=tau, refine_sensor="kn",
                              refine_threshold=THR_R, switch_sensor="neq",
                              switch_threshold=THR_S, record=("kl",), output_every=out,
                              tile=TILE, dev_exp=kexp)
            lat.set_fields(rho, ux, uy)
            lat.step(args.warmup)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K)]
            for k in range(K):
                ev[2 * k].record(stream)
                lat.step(1)
                ev[2 * k + 1].record(stream)
            torch.cuda.synchronize()
            total = ev[0].elapsed_time(ev[-1])
            kern = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(K)) / K
            # the same K steps as one kss_step(K) call (a multi-step launch where the
            # library takes one, else a replayed graph of one-step launches)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(K)
            e1.record(stream)
            torch.cuda.synchronize()
            call = e0.elapsed_time(e1) / K
            bpl = (18 if prec == "fp16dev" else 36) * 2 + (5 if out else 0)
            achieved = bpl * cells / (kern * 1e-3) / 1e9
            runs[name] = {"value": cells * K / (total * 1e-3) / 1e6, "unit": "MLUPS",
                          "ms_per_step": total / K, "kernel_ms": kern, "bytes_per_lup": bpl,
                          "achieved_gbs": achieved, "frac": achieved / peak,
                          "one_call_ms_per_step": call,
                          "one_call_frac": bpl * cells / (call * 1e-3) / 1e9 / peak}
            lat.close()
    clocks = clk.summary()
    err = None
    if args.fp16_error:
        err = fp16_error(n, tau, kexp, gen)
    main = runs["fp16dev"]
    line = {
        "metric": FP16_METRIC, "value": main["value"], "unit": "MLUPS", "n_gpus": 1, "steps": K,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16 storage / f32 arithmetic",
        "data": "synthetic",
        "config": {"workload": f"D2Q9 {n}x{n} periodic, smooth perturbations amplitude 1e-3 "
                               "(density and velocity), tau=0.6, FP16 deviation storage "
                               "K=20, Kn refine 1e-3, neq switch 1e-4, KL field, flags, tile "
                               "counts, sums every step", "nx": n, "ny": n,
                   "l2": f"inputs larger than L2: {cells * 36 / 1e9:.2f} GB of populations "
                         "per step"},
        "roofline": {"bound": "hbm", "achieved": main["achieved_gbs"], "peak": peak,
                     "unit": "GB/s", "frac": main["frac"], "peak_kind": peak_kind,
                     "traffic": profile_traffic(FP16_PROFILE) if n == 8192 else None,
                     "algorithmic_bytes_per_launch": main["bytes_per_lup"] * cells,
                     "kernel_ms": main["kernel_ms"],
                     "kernel": "step_kernel<__half, MODE_STD, pull, store>"},
        "variants": runs,
        "speedup_vs_fp32": main["value"] / runs["fp32"]["value"],
        "error_vs_fp64": err,
        "gpu_launches": K,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


AAR_PROFILE = os.path.join(ROOT, "profiles", "step_aar_std_f32_4096.md")
BATCH_PROFILE = os.path.join(ROOT, "profiles", "batch_multi_f32_64lattices.md")
FP16_PROFILE = os.path.join(ROOT, "profiles", "step_std_f16dev_8192.md")
AAR_METRIC = ("MLUPS with adaptive algorithm refinement (two-relaxation collision in the "
              "switched region) and sensors fused, 1xGB300")


def run_aar(args):
    """The adaptive-algorithm-refinement workload (one launch per step)."""
    import numpy as np
    import torch

    from paper_2603_13618_gb300 import inputs, kss

    torch.cuda.set_device(0)
    n = args.size or 4096
    cells = n * n
    rho, ux, uy = workload_fields(n, n)
    tau2 = 0.5 + (3.0 / 16.0) / (TAU - 0.5)
    region = inputs.random_region(n, n, seed=4096)
    stream = torch.cuda.current_stream()
    K = args.steps
    peak, peak_kind = measured_peak()
    variants = (
        # name, tau2, switch sensor, output_every, record, bytes per LUP
        ("aar_std", tau2, "neq", 1, ("kl",), 72 + 5 + 2),
        ("bgk_std", 0.0, "neq", 1, ("kl",), 72 + 5),
        ("aar_qe", tau2, "qe", 1, ("kl",), 72 + 5 + 2),
        ("aar_all_sensors", tau2, "qe", 1, ("kl", "alpha"), 72 + 5 + 2),
        ("aar_plain", tau2, "neq", 0, (), 72 + 1),
        ("bgk_plain", 0.0, "neq", 0, (), 72),
    )
    runs = {}
    with ClockSampler(0) as clk:
        for name, t2, sw, out, rec, bpl in variants:
            lat = kss.Lattice(n, n, precision="fp32", tau=TAU, tau2=t2, refine_sensor="kn",
                              refine_threshold=THR_R, switch_sensor=sw,
                              switch_threshold=THR_S, record=rec, output_every=out,
                              tile=TILE)
            lat.set_fields(rho, ux, uy)
            if t2 and not out:
                lat.set_aar_region(region)
            lat.step(args.warmup)
            torch.cuda.synchronize()
            # the K steps as one call (a multi-step launch for output steps, a replayed
            # graph for plain ones), then as single launches, each timed on its own
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(K)
            e1.record(stream)
            torch.cuda.synchronize()
            total = e0.elapsed_time(e1)
            k1 = min(K, 100)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * k1)]
            for k in range(k1):
                ev[2 * k].record(stream)
                lat.step(1)
                ev[2 * k + 1].record(stream)
            torch.cuda.synchronize()
            kern = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(k1)) / k1
            achieved = bpl * cells / (total / K * 1e-3) / 1e9
            r = {"value": cells * K / (total * 1e-3) / 1e6, "unit": "MLUPS",
                 "ms_per_step": total / K, "single_launch_ms": kern, "bytes_per_lup": bpl,
                 "achieved_gbs": achieved, "frac": achieved / peak}
            if t2:
                r["switched_fraction"] = float(np.mean(lat.get_aar_region()))
            runs[name] = r
            lat.close()
    main = runs["aar_std"]
    line = {
        "metric": AAR_METRIC, "value": main["value"], "unit": "MLUPS", "n_gpus": 1,
        "steps": K, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"D2Q9 FP32 {n}x{n} periodic as the headline workload, "
                               f"two-relaxation model tau=0.6, tau2={tau2:.4g} in the cells "
                               "switched by neq > 1e-4 at the previous step; Kn refine 1e-3, "
                               "KL field, flags, tile counts, sums every step",
                   "nx": n, "ny": n, "tau": TAU, "tau2": tau2,
                   "l2": f"inputs larger than L2: {cells * 72 / 1e9:.2f} GB of populations "
                         "per step"},
        "roofline": {"bound": "hbm", "achieved": main["achieved_gbs"], "peak": peak,
                     "unit": "GB/s", "frac": main["frac"], "peak_kind": peak_kind,
                     "traffic": (profile_traffic(AAR_PROFILE) if n == 4096 else None),
                     "algorithmic_bytes_per_launch": main["bytes_per_lup"] * cells,
                     "kernel_ms_per_step": main["ms_per_step"],
                     "kernel": "step_kernel_multi<float, MODE_STD, AAR> (all K steps in one "
                               "cooperative launch, rows staged in shared memory by "
                               "cp.async)"},
        "variants": runs,
        "aar_cost_vs_bgk": main["ms_per_step"] / runs["bgk_std"]["ms_per_step"],
        "gpu_launches": 1,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


SHEAR_METRIC = "MLUPS, 128^2 FP64 shear wave, sensors and flags every 10 steps, 1xGB300"


def run_shear(args):
    """The FP64 correctness workload, timed as one 2000-step call."""
    import torch

    from paper_2603_13618_gb300 import inputs, kss

    torch.cuda.set_device(0)
    n, tau, steps = 128, 0.8, 2000
    rho, ux, uy = inputs.shear_wave(n, n, 0.01)
    lat = kss.Lattice(n, n, precision="fp64", tau=tau, refine_sensor="kn",
                      refine_threshold=1e-3, switch_sensor="neq", switch_threshold=1e-4,
                      record=("kn", "kl"), output_every=10)
    stream = torch.cuda.current_stream()
    times = []
    for rep_ in range(1 + max(1, args.warmup // 10)):
        lat.set_fields(rho, ux, uy)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    t = min(times[1:])  # the first call records the step graphs
    _, counts, step = lat.read_stats()
    line = {
        "metric": SHEAR_METRIC, "value": n * n * steps / (t * 1e-3) / 1e6, "unit": "MLUPS",
        "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": t / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "D2Q9 FP64 128x128 periodic shear wave u_x = 0.01 sin(2 pi y/128), "
                               "tau = 0.8, 2000 steps in one call; Kn (refine 1e-3) and KL "
                               "fields, flags, tile counts and sums every 10 steps",
                   "nx": n, "ny": n, "l2": "the lattice lives in L2 (1.2 MB per buffer): no "
                                           "bandwidth fraction is meaningful"},
        "refine_count_at_step_2000": int(counts[0]), "step": int(step),
        "gpu_launches": steps,
    }
    print(json.dumps(line), flush=True)
    lat.close()
    return 0


def fp16_error(n, tau, kexp, gen, steps=500, window=256):
    """Errors of FP16 deviation and FP32 storage after `steps` steps against the FP64
    oracle on the central window (the oracle runs the window's domain of dependence)."""
    import numpy as np

    import oracle
    from paper_2603_13618_gb300 import inputs, kss

    x0 = n // 2 - window // 2
    halo = steps
    wr, wu, wv = inputs.smooth_jump(n, n, x0=x0 - halo, y0=x0 - halo, wx=window + 2 * halo,
                                    wy=window + 2 * halo, **gen)
    t0 = time.perf_counter()
    oracle.set_threads(oracle.host_cores())  # (bit-identical to one thread)
    try:
        f = oracle.step(oracle.init_equilibrium(wr, wu, wv), tau, steps - 1)
        sens, nonpos = oracle.sensor_fields(f, tau, pull=True)
        f = oracle.step(f, tau)
        rr, ru, rv = oracle.moments(f)
    finally:
        oracle.set_threads(1)
    t_orc = time.perf_counter() - t0
    c = slice(halo, halo + window)
    ref = {"rho": rr[c, c], "ux": ru[c, c], "uy": rv[c, c]}
    for s in ("kn", "kl", "neq"):
        ref[s] = sens[oracle.SENSOR_ID[s]][c, c]
    rf, _, _ = oracle.flags(ref["kn"], THR_R, ref["neq"], THR_S, nonpos[c, c], TILE)
    rho, ux, uy = inputs.smooth_jump(n, n, **gen)
    out = {"steps": steps, "window": window, "oracle_s": t_orc}
    win = (slice(x0, x0 + window), slice(x0, x0 + window))
    for prec in ("fp16dev", "fp32"):
        lat = kss.Lattice(n, n, precision=prec, tau=tau, record=("kn", "kl", "neq"),
                          output_every=steps, dev_exp=kexp)
        lat.set_fields(rho, ux, uy)
        lat.step(steps)
        got = dict(zip(("rho", "ux", "uy"), (a[win] for a in lat.read_moments())))
        for s in ("kn", "kl", "neq"):
            got[s] = lat.read_sensor(s)[win]
        fl = lat.read_flags()[0][win]
        lat.close()
        e = {}
        for key in got:
            d = np.abs(got[key] - ref[key])
            scale = np.max(np.abs(ref[key])) if key != "rho" else 1.0
            e[key] = {"max_abs": float(np.max(d)), "max_rel_to_field_max": float(np.max(d) / scale)}
        e["flags_mismatch"] = int(np.sum((fl & 3) != (rf & 3)))
        out[prec] = e
    return out


def run_reference(args):
    """The oracle on the host cores, one bounded window of the workload per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    window = 256
    rho, ux, uy = workload_fields(x0=NX // 2 - window // 2, y0=NY // 2 - window // 2,
                                  wx=window, wy=window)
    f = oracle.init_equilibrium(rho, ux, uy)
    threads = oracle.host_cores() if oracle.lib().orc_have_openmp() else 1
    oracle.set_threads(threads)

    def one():
        oracle.run(f, TAU, 1, oracle.SENSOR_ID["kn"], THR_R, oracle.SENSOR_ID["neq"], THR_S,
                   TILE, full=False)

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = time.perf_counter() - t0
    oracle.set_threads(1)
    value = window * window * args.steps / el / 1e6
    sample = (f"each step: one fused oracle step ({{Kn, KL, neq}}, flags, tile counts, sums) "
              f"on the central {window}x{window} window, {threads} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY,
                   "sample": f"{window}x{window} central window per step"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


# ---- replicas (N > 1 under torchrun): one independent lattice per rank ----

def dist_env():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init_replicas(world, backend="nccl", device=None):
    """The process group of an N > 1 run (None for one process).  The ranks exchange no
    lattice data: only the timing barrier and the maximum of the timings."""
    if world <= 1:
        return None
    import torch.distributed as dist

    if device is not None:
        dist.init_process_group(backend, device_id=device)
    else:
        dist.init_process_group(backend)
    return dist


def max_over_ranks(value, dist, device="cpu"):
    """The largest of the ranks' values (the job's time is that of its slowest rank)."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, cells, steps, ms):
    """Lattice updates of all ranks per second (weak scaling: each rank a full lattice)."""
    return world * cells * steps / (ms * 1e-3) / 1e6


def deferred_fraction(lat):
    """Share of the last step's cells that the fused pass defers to the exact per-cell
    recomputation: Kn >= 1/16 or a non-positive population (Kn = +Inf); the fused
    pass's other condition (|u|^2 >= 0.3) does not occur at Mach 0.1."""
    import numpy as np

    kn = lat.read_sensor("kn")
    return float(np.mean(~(kn < 0.0625)))


def tau_sweep(lat0, k, warmup, stream, peak, barrier):
    """The timed call (one kss_step(k), all steps fused output steps) at each tau of the
    configuration on a fresh lattice, with the deferred share of its last step."""
    import torch

    from paper_2603_13618_gb300 import kss

    rho, ux, uy = workload_fields()
    out = {}
    for tau in (0.51, 0.6, 0.8, 1.0):
        if tau == TAU:
            lat = lat0
            lat.set_fields(rho, ux, uy)
        else:
            lat = kss.Lattice(NX, NY, precision="fp32", tau=tau, refine_sensor="kn",
                              refine_threshold=THR_R, switch_sensor="neq",
                              switch_threshold=THR_S, record=("kl",), output_every=1,
                              tile=TILE, stream="torch")
            lat.set_fields(rho, ux, uy)
        lat.step(warmup)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(k)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / k
        gbs = BYTES_PER_LUP * NX * NY / (ms * 1e-3) / 1e9
        out[str(tau)] = {"ms_per_step": ms, "frac": gbs / peak, "steps": k,
                         "deferred_fraction": deferred_fraction(lat),
                         "refine_count": int(lat.read_stats()[1][0])}
        if lat is not lat0:
            lat.close()
    return out


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2603_13618_gb300 import kss

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_replicas(world, "nccl", torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    rho, ux, uy = workload_fields()
    lat = kss.Lattice(NX, NY, precision="fp32", tau=TAU, refine_sensor="kn",
                      refine_threshold=THR_R, switch_sensor="neq", switch_threshold=THR_S,
                      record=("kl",), output_every=1, tile=TILE, stream="torch",
                      kernel=args.kernel)
    lat.set_fields(rho, ux, uy)
    stream = torch.cuda.current_stream()
    lat.step(args.warmup)
    barrier()

    K = args.steps
    # the timed region: one kss_step(K) call -- K fused steps, each with its sensors,
    # flags, tile counts and sums, in one cooperative multi-step launch (one launch per
    # step for the TMA kernel)
    multi = args.kernel != "tma"
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        t_host = time.perf_counter()
        e0.record(stream)
        lat.step(K)
        e1.record(stream)
        barrier()
        t_host = time.perf_counter() - t_host
        # (untimed) the same launches for about a second more, so that the clock samples
        # of a short timed region are taken under its load rather than at idle
        t_load = time.perf_counter()
        while time.perf_counter() - t_load < 1.0:
            lat.step(max(K, 20))
            torch.cuda.synchronize()
    clocks = clk.summary()
    total_ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    cells = NX * NY
    value = whole_job_mlups(world, cells, K, total_ms)
    kern_ms = total_ms / K  # per step (the launch covers all K steps)
    achieved = BYTES_PER_LUP * cells / (kern_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    sums, counts, step = lat.read_stats()

    # the same steps as one launch per step, each timed on its own
    k1 = min(K, 200)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(k1)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(k1)]
    barrier()
    for k in range(k1):
        starts[k].record(stream)
        lat.step(1)
        ends[k].record(stream)
    barrier()
    per_launch = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    single = {"ms_per_step": starts[0].elapsed_time(ends[-1]) / k1,
              "kernel_ms": sum(per_launch) / k1, "steps": k1}
    single["frac"] = BYTES_PER_LUP * cells / (single["kernel_ms"] * 1e-3) / 1e9 / peak

    # end to end through the C ABI with host buffers: each step copies its input fields
    # from pinned host memory, runs one fused step and reads the flags, tile counts and
    # stats back to pinned host memory.  The FP32 lattice's fields go in as FP32
    # (kss_set_fields_f32: the same state as the same values in FP64, half the bytes over
    # the host link); the leg with FP64 fields (kss_set_fields) is reported beside it.
    e2e = e2e_fp64 = None
    if rank == 0 or world > 1:
        import numpy as np

        pin = [torch.from_numpy(a).pin_memory() for a in (rho, ux, uy)]
        pin32 = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
                 for a in (rho, ux, uy)]
        fl = torch.empty((NY, NX), dtype=torch.uint8).pin_memory()
        tl = torch.empty((2, lat.nty, lat.ntx), dtype=torch.int32).pin_memory()
        ke = max(3, min(20, K // 10))

        def e2e_leg(fields, esize, call):
            for _ in range(2):
                lat.set_fields(*fields)
                lat.step(1)
                lat.read_flags(out=(fl, tl))
                lat.read_stats()
            barrier()
            t0 = time.perf_counter()
            for _ in range(ke):
                lat.set_fields(*fields)
                lat.step(1)
                lat.read_flags(out=(fl, tl))
                lat.read_stats()
            barrier()
            el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
            h2d = 3 * esize * cells
            d2h = cells + 4 * 2 * lat.nty * lat.ntx + 8 * 3 + 8 * 3 + 8 * 3
            return {"value": whole_job_mlups(world, cells, ke, el * 1e3), "unit": "MLUPS",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": ke,
                    "calls_per_step": [call, "kss_step(1)", "kss_read_flags(host)",
                                       "kss_read_stats"]}

        e2e = e2e_leg(pin32, 4, "kss_set_fields_f32(host)")
        e2e_fp64 = e2e_leg(pin, 8, "kss_set_fields(host)")

    # end to end for a caller that keeps the state on the device: K steps, each followed
    # by reading its flags, tile counts, KL field and sums back to pinned host memory
    e2e_stepping = None
    if rank == 0 or world > 1:
        ks = max(3, min(20, K // 10))
        klh = torch.empty((NY, NX), dtype=torch.float64).pin_memory()
        lat.set_fields(*pin)
        for _ in range(2):
            lat.step(1)
            lat.read_flags(out=(fl, tl))
            lat.read_sensor("kl", out=klh)
            lat.read_stats()
        barrier()
        t0 = time.perf_counter()
        for _ in range(ks):
            lat.step(1)
            lat.read_flags(out=(fl, tl))
            lat.read_sensor("kl", out=klh)
            lat.read_stats()
        barrier()
        el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        d2h = cells + 8 * cells + 4 * 2 * lat.nty * lat.ntx + 8 * 3 + 8 * 3 + 8 * 3
        e2e_stepping = {"value": whole_job_mlups(world, cells, ks, el * 1e3), "unit": "MLUPS",
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h, "steps": ks,
                        "calls_per_step": ["kss_step(1)", "kss_read_flags(host)",
                                           "kss_read_sensor(kl, host)", "kss_read_stats"]}

    # the kernel's work depends on the data: cells it cannot prove exact in the fused pass
    # (Kn >= 1/16, or a non-positive population) are recomputed in the CTA epilogue; the
    # same workload at the other relaxation times of the configuration, K' steps each
    sweep = None
    if rank == 0 and not args.no_tau_sweep:
        sweep = tau_sweep(lat, min(K, 100), args.warmup, stream, peak, barrier)

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": total_ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "tau": TAU,
                       "precision": "fp32", "tile": TILE, "output_every": 1,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2: 1.21 GB of populations per step "
                             "vs 126 MB L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": profile_traffic(),
                         "algorithmic_bytes_per_step": BYTES_PER_LUP * cells,
                         "steps_per_launch": K if multi else 1,
                         "kernel_ms_per_step": kern_ms,
                         "kernel": kernel_name(args.kernel)},
            "single_step_launches": single,
            "cpu_baseline": base,
            "e2e": e2e,
            "e2e_fp64_fields": e2e_fp64,
            "e2e_stepping": e2e_stepping,
            "tau_sweep": sweep,
            "gpu_launches": 1 if multi else K,
            "clocks": clocks,
            "host_s": t_host,
            "check": {"sum_rho": sums[0], "refine": int(counts[0]), "switch": int(counts[1]),
                      "nonpos": int(counts[2]), "step": step},
        }
        print(json.dumps(line), flush=True)
    lat.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tau-sweep", action="store_true",
                    help="skip the timed calls at the other relaxation times")
    ap.add_argument("--kernel", default="auto", choices=["auto", "vector", "tma"],
                    help="step kernel (auto: the library's choice)")
    ap.add_argument("--size", type=int, default=None,
                    help="lattice edge (default 4096; 8192 for fp16dev8192; smaller sizes "
                         "for profiling captures only)")
    ap.add_argument("--fp16-error", action="store_true",
                    help="fp16dev8192: also measure the error against the FP64 oracle")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batch64", "adjoint512", "fp16dev8192", "aar4096",
                             "shear128"],
                    help="single: the 4096^2 lattice (default); batch64: 64 uneven "
                         "lattices; adjoint512: the gradient of the KL objective")
    ap.add_argument("--no-tune", action="store_true",
                    help="batch64: keep the default work decomposition")
    ap.add_argument("--batch-rows", type=int, default=0,
                    help="batch64: CTA height of a fixed multi-step decomposition instead of "
                         "the autotuner's choice")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    global NX, NY
    NX = NY = args.size or 4096
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "adjoint512":
        return run_adjoint(args)
    if args.workload == "fp16dev8192":
        return run_fp16(args)
    if args.workload == "aar4096":
        return run_aar(args)
    if args.workload == "shear128":
        return run_shear(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
