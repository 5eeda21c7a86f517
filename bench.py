#!/usr/bin/env python3
"""Throughput of the FFT-based ETD step (Mpoint-steps/s).

Workload: the 3D coupled phi-u system with stabilised ETDRK2 and a narrow band, 256^3 on
[-pi, pi)^3, ellipsoid membrane (1.2, 0.9, 0.9), seeded protein field on the band,
tau = 1e-4, FP32 storage/FFT with FP64 phi-function tables and reductions.

Our arm (default): W untimed steps, then K steps timed with CUDA events on the plan's
stream between barriers; value = points * K * ranks / max-over-ranks time.  Each step
moves ~2 GB through HBM, far more than L2, so no flush is needed.  `e2e` repeats the
measurement through the public API with host buffers (pinned upload of phi and u, one
step, download of phi and u, every step).  `roofline` reports the dominant kernel class:
algorithmic bytes of its launches in the timed region / their event-timed duration.
`cpu_baseline` times the FP64 CPU oracle on a bounded sample (rank 0 only).

--impl reference: the FP64 CPU oracle itself, on a bounded sample of the same workload.
Multi-GPU (torchrun): independent replicas, one per GPU, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import platform
import os
import shutil
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpoint-steps/s, 3D coupled ETDRK2 256^3: FP32 vs FP64 at rel L2<=1e-5; % HBM peak"
UNIT = "Mpoint-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # default window: steps 4-500 of the 500-step c3 run (the whole job after 3 warm-up steps);
    # the first steps carry larger band-solve iteration counts (U^0 is grid-scale noise), so a
    # short early window would misstate the run's throughput
    ap.add_argument("--steps", type=int, default=497)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=64, help="grid of the oracle sample")
    ap.add_argument("--cpu-steps", type=int, default=6)
    ap.add_argument("--fp64-steps", type=int, default=19, help="steps of the FP64 comparison leg (0: skip)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-sweep leg")
    ap.add_argument("--no-sec2", action="store_true", help="skip the Sec. 2.2 Krylov-scheme leg")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def allreduce_max(x: float, world: int) -> float:
    """Max over ranks (identity for one rank).  Works with the nccl and gloo backends."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    devc = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=devc)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(world: int, points: int, steps: int, ms_max: float) -> float:
    """Whole-job throughput in Mpoint-steps/s: units all replicas processed / slowest time."""
    return world * points * steps / (ms_max / 1e3) / 1e6


KERNEL_SOURCES = ("df32.cuh", "fft.cuh", "kernels.cuh", "ops.cuh")


def source_hash():
    """sha256 over the sources that define the measured kernels (the FFT passes with their tile
    choice, the spectral operators and epilogues, the pointwise kernels and the band solve):
    ties recorded ncu counters to the kernels they measured.  The plan's host orchestration and
    the kernels no recorded counter covers (the Krylov scheme's) are left out."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2606_04347_gb300", "csrc")
    for name in sorted(KERNEL_SOURCES):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def recorded_traffic(kind, grid, prec, algo_per_launch):
    """DRAM bytes per launch of a kernel class, from the committed ncu summary, if that summary
    was taken on the kernels as they are now (same source hash); else None.  A class whose
    work per launch varies (the band CG: iterations x band nodes) is recorded as the ratio of
    measured DRAM bytes to algorithmic bytes of the captured launch and scaled to this run's
    average launch by its algorithmic bytes."""
    path = os.path.join(ROOT, "profiles", "traffic_c3.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as f:
        for ln in f:
            parts = ln.split()
            if len(parts) == 2 and not ln.startswith("#"):
                rec[parts[0]] = parts[1]
    if rec.get("source_sha256") != source_hash():
        return None
    v = rec.get(f"{kind}_{grid}_{prec}")
    if v is not None:
        return float(v)
    r = rec.get(f"{kind}_{grid}_{prec}_ratio")
    return float(r) * algo_per_launch if r is not None else None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, period_ms=20):
        self.idx = gpu_index
        self.period = period_ms
        self.proc = None
        self.lines = []        # (host time the sample arrived, csv line)
        self.window = None     # (t0, t1): host times bracketing the timed region

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        self.proc = subprocess.Popen([exe, f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                      "-i", str(self.idx), "-lms", str(self.period)],
                                     stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # samples that arrived while the timed region ran (one period of slack for the pipe);
        # all samples if none did
        lines = [ln for t, ln in self.lines]
        scope = "whole sampler run"
        if self.window:
            t0, t1 = self.window
            inside = [ln for t, ln in self.lines if t0 <= t <= t1 + self.period / 1e3]
            if inside:
                lines, scope = inside, "timed region"
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "scope": scope, "period_ms": self.period}


def oracle_sample(size, steps):
    """FP64 CPU oracle on a bounded sample of the same workload: (Mpoint-steps/s, desc)."""
    from oracle import etd as oetd
    from paper_2606_04347_gb300 import workloads as wl
    p, phi, u, _ = wl.workload("c3", n=size)
    cs = oetd.CoupledStepper(p)
    cs.step(phi, u)          # first step outside the timing (A0, caches)
    t0 = time.perf_counter()
    cs.run(phi, u, steps)
    dt = time.perf_counter() - t0
    return size ** 3 * steps / dt / 1e6, f"c3 workload at {size}^3, {steps} ETDRK2 steps, numpy FP64", dt


def _fixed_sample(name, size, steps):
    from oracle import etd as oetd
    from paper_2606_04347_gb300 import workloads as wl
    p, phi, u, _ = wl.workload(name, n=size)
    st = oetd.FixedStepper(p, phi)
    u = st.step(u)
    t0 = time.perf_counter()
    st.run(u, steps)
    dt = time.perf_counter() - t0
    return float(np.prod(p.shape)) * steps / dt / 1e6, dt


def _pool_worker(args):
    size, steps = args
    v, _, dt = oracle_sample(size, steps)
    return size ** 3 * steps, dt


def host_info():
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    model = ln.split(":", 1)[1].strip() + f" ({platform.machine()})"
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def cpu_baselines(a):
    """The FP64 oracle as it stands on this machine's host cores: the c3 sample on one core (the
    reported value), the same sample in one process per core at once (all-core throughput), and
    samples of the fixed-membrane workloads c1 (128^2 ETD1) and c2 (at 32^3, ETDRK2)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    v, desc, secs = oracle_sample(a.cpu_sample, a.cpu_steps)
    out = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc, "seconds": round(secs, 2),
           "host": host_info()}
    nproc = os.cpu_count() or 1
    workers = max(1, min(nproc, 16))
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_pool_worker, [(a.cpu_sample, 2)] * workers))
    wall = time.perf_counter() - t0
    out["all_cores"] = {"value": sum(r[0] for r in res) / wall / 1e6, "unit": UNIT, "processes": workers,
                        "sample": f"c3 at {a.cpu_sample}^3, 2 ETDRK2 steps in each of {workers} processes "
                                  f"(one per core, process start-up included)", "seconds": round(wall, 2)}
    c1, t1 = _fixed_sample("c1", 128, 10)
    c2, t2 = _fixed_sample("c2", 32, 3)
    out["c1"] = {"value": c1, "unit": UNIT, "sample": "c1 128^2 fixed membrane, 10 ETD1 steps, one core",
                 "seconds": round(t1, 2)}
    out["c2"] = {"value": c2, "unit": UNIT, "sample": "c2 at 32^3 fixed membrane, 3 ETDRK2 steps, one core",
                 "seconds": round(t2, 2)}
    return out


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import etd as oetd
    from paper_2606_04347_gb300 import workloads as wl
    # the sample grid: the largest power of two <= --cpu-sample whose W + K steps stay within
    # about 18 Mpoint-steps (2-3 minutes of the oracle on one core)
    size = a.cpu_sample
    while size > 16 and size ** 3 * (a.steps + a.warmup) > 18e6:
        size //= 2
    p, phi, u, _ = wl.workload("c3", n=size)
    cs = oetd.CoupledStepper(p)
    phi, u = cs.run(phi, u, a.warmup)
    t0 = time.perf_counter()
    cs.run(phi, u, a.steps)
    dt = time.perf_counter() - t0
    v = size ** 3 * a.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * dt / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"c3 coupled ETDRK2 ellipsoid, bounded sample at {size}^3 of the 256^3 run",
                   "grid": size, "tau": p.tau},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{size}^3 grid, {a.steps} steps per timed run", "host": host_info()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def batch_leg(stream, peak):
    """The batched fixed-membrane sweep: 48 runs (64^3 / 96^3 / 128^3, seeds 100-147), FP32-mixed
    ETDRK2, 200 steps each, tiles autotuned per grid, 6-step blocks replayed as one CUDA graph.
    Timed: steps 3-200 of every run (the first two run eagerly, then the graph is recorded and
    replayed 33 times).  Bytes: each run's algorithmic bytes per step, from one single-plan
    replay of the same steps with per-launch counters; the same single plans, one run at a
    time with default tiles and no graph, give the comparison time."""
    import torch
    from paper_2606_04347_gb300 import Batch, Plan
    from paper_2606_04347_gb300 import workloads as wl
    runs = []
    for seed in range(100, 148):
        p, phi, u, nsteps = wl.c4_run(seed, 1)
        runs.append((p.replace(cg_rtol=1e-5), phi, u))
    t0 = time.perf_counter()
    b = Batch([r[0] for r in runs], stream=stream, autotune=True)
    t_plan = time.perf_counter() - t0
    phis = [torch.tensor(r[1], dtype=torch.float32, device="cuda") for r in runs]
    us = [torch.tensor(r[2], dtype=torch.float32, device="cuda") for r in runs]
    b.step(phis, us, 2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(None, us, 198)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    from paper_2606_04347_gb300.abi import EtdError
    try:
        diag, check = b.check(None, us), "ok"
    except EtdError as ex:
        diag, check = [], str(ex)
    tiles = {}
    for i, r in enumerate(runs):
        tiles.setdefault(r[0].n[0], b.info(i))
    graph = b.info(0)["graph"]
    b.close()
    del phis, us
    pts = sum(r[0].n[0] ** 3 for r in runs)
    # one run at a time (default tiles, eager), with the per-launch counters for the bytes
    t_single, nbytes = 0.0, 0.0
    for p, phi, u in runs:
        plan = Plan(p, stream=stream)
        f = torch.tensor(phi, dtype=torch.float32, device="cuda")
        ud = torch.tensor(u, dtype=torch.float32, device="cuda")
        plan.step(f, ud, 2)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        plan.step(None, ud, 198)
        f1.record(stream)
        torch.cuda.synchronize()
        t_single += f0.elapsed_time(f1)
        plan.timing(True)
        plan.step(None, ud, 6)
        nbytes += sum(v[2] for v in plan.timing_read().values()) / 6 * 198
        plan.timing(False)
        plan.close()
    achieved = nbytes / (ms / 1e3) / 1e9
    finite = check == "ok" and all(d["band_size"] > 0 for d in diag)
    return {
        "workload": "c4: 48 fixed-membrane OK runs, grids 64^3/96^3/128^3 (16/21/11), eps in [0.03,0.08], "
                    "sigma in [10,200], S in {1,2,4}, tau in {1e-3,2e-3,5e-3}, seeds 100-147, ETDRK2 FP32, 200 steps",
        "value": pts * 198 / (ms / 1e3) / 1e6, "unit": UNIT, "ms_steps_3_to_200": ms, "graph": graph,
        "tiles_by_grid": {str(k): {kk: vv for kk, vv in v.items() if kk != "graph"} for k, v in tiles.items()},
        "autotune_and_plans_s": round(t_plan, 2),
        "one_run_at_a_time": {"value": pts * 198 / (t_single / 1e3) / 1e6, "ms": t_single},
        "speedup_over_one_at_a_time": t_single / ms,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "bytes_per_step": nbytes / 198},
        "all_runs_finite": finite, "check": check,
    }


def sec2_leg(stream, peak):
    """The g^{1/2}-split scheme of Sec. 2.2 (Lanczos phi_j(tau L) on the band) in the paper's 2D
    rate-study setting: 256^2 on [-1,1]^2, circle, eps_phi = eps_u = 10 h, ETDRK2 (M = 200),
    tau = 1e-4, FP64, band solve to 1e-11.  5 warm-up steps, then 100 steps timed with CUDA events;
    a second pass of the same 100 steps with per-launch counters gives the time per kernel class
    and the Krylov class's algorithmic bytes (15 elements + 24 B of couplings/indices per band
    node per Lanczos step, plus the norms and combinations)."""
    import torch
    from paper_2606_04347_gb300 import Plan
    from paper_2606_04347_gb300 import workloads as wl
    p, phi, u0 = wl.paper2d("circle", 10.0, 2, 0)
    p = p.replace(model=2, cg_rtol=1e-11)
    plan = Plan(p, stream=stream)
    u = torch.tensor(u0, device="cuda")
    d = plan.step(torch.tensor(phi, device="cuda"), u, 5, diag=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nst = 100
    e0.record(stream)
    d = plan.step(None, u, nst, diag=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    plan.timing(True)
    plan.step(None, u, nst)
    kt = plan.timing_read()
    plan.timing(False)
    plan.close()
    kms, kn, kb = kt["krylov"]
    ach = kb / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    return {
        "workload": "Sec. 2.2 scheme, 2D 256^2 [-1,1]^2 circle, eps_phi = eps_u = 10h, ETDRK2, tau=1e-4, FP64",
        "value": 256 * 256 * nst / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms / nst,
        "band_size": d["band_size"], "krylov_dim_last": d["krylov_dim_last"], "cg_iters_last": d["cg_iters_last"],
        "kernel_ms_per_step": {k: round(v[0] / nst, 4) for k, v in kt.items() if v[1]},
        "launches_per_step": {k: v[1] / nst for k, v in kt.items() if v[1]},
        "krylov_roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                            "algo_bytes_per_step": kb / nst,
                            "note": "latency-bound: a band of ~5.7k nodes, host convergence check every 8 steps"},
    }


def run_ours(a):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    from paper_2606_04347_gb300 import Plan
    from paper_2606_04347_gb300 import workloads as wl
    prec = 1 if a.precision == "fp32" else 0
    p, phi0, u0, _ = wl.workload("c3", n=a.size, precision=prec)
    # band-solve tolerance: FP64 solves to 1e-12; the FP32 form stops at 1e-4 (both stages),
    # where the FP32-vs-FP64 differences of phi, u and the energy after 20 steps at 256^3 match
    # those of tighter solves (u 4.4e-6 against 4.3e-6 at 1e-5; a predictor at 1e-3 gives 1.7e-5)
    p = p.replace(cg_rtol=1e-4 if prec else 1e-12, cg_rtol_pred=1e-4 if prec else 0.0)
    dt_ = torch.float32 if prec else torch.float64
    stream = torch.cuda.current_stream()
    plan = Plan(p, stream=stream)
    phi = torch.tensor(phi0, dtype=dt_, device="cuda")
    u = torch.tensor(u0, dtype=dt_, device="cuda")
    npts = a.size ** 3

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    plan.step(phi, u, a.warmup)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0 = time.perf_counter()
    e0.record(stream)
    plan.step(phi, u, a.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    h1 = time.perf_counter()
    barrier()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk.mark(h0, h1)
    clocks = clk.stop()
    ms = allreduce_max(ms, world)
    value = aggregate(world, npts, a.steps, ms)
    d = plan.step(phi, u, 0, diag=True)
    # the same window again (a fresh plan from the same input, the same warm-up steps, the same
    # timed steps) with per-launch events: kernel classes, launch count and rooflines of exactly
    # the headline's steps; the headline value above is timed without them
    plan_t = Plan(p, stream=stream)
    phi_t = torch.tensor(phi0, dtype=dt_, device="cuda")
    u_t = torch.tensor(u0, dtype=dt_, device="cuda")
    plan_t.step(phi_t, u_t, a.warmup)
    torch.cuda.synchronize()
    # counters are read every 100 steps (the plan keeps events for 16384 launches)
    kt, ms_t, left = {}, 0.0, a.steps
    while left > 0:
        chunk = min(100, left)
        plan_t.timing(True)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        plan_t.step(phi_t, u_t, chunk)
        f1.record(stream)
        torch.cuda.synchronize()
        ms_t += f0.elapsed_time(f1)
        for k, v in plan_t.timing_read().items():
            o = kt.get(k, (0.0, 0, 0.0))
            kt[k] = (o[0] + v[0], o[1] + v[1], o[2] + v[2])
        left -= chunk
    plan_t.timing(False)
    plan_t.close()
    del phi_t, u_t

    # dominant kernel class and its roofline
    dom = max(kt, key=lambda k: kt[k][0])
    dms, dn, dbytes = kt[dom]
    peak, peak_src = peaks()
    achieved = dbytes / (dms / 1e3) / 1e9 if dms > 0 else 0.0
    launches = int(sum(v[1] for v in kt.values()))
    # whole step: every class's algorithmic bytes of the headline's steps over the headline's
    # device time (timed without per-launch events)
    step_bytes = sum(v[2] for v in kt.values())
    step_achieved = step_bytes / (ms / 1e3) / 1e9

    # FP64 form of the same step on the same GPU (outside the timed region): speed-up of the
    # FP32-mixed form and agreement of the two after the same number of steps
    fp64 = None
    if a.fp64_steps > 0 and prec == 1:
        p64 = p.replace(precision=0, cg_rtol=1e-12, cg_rtol_pred=0.0)
        plan64 = Plan(p64, stream=stream)
        phi64 = torch.tensor(phi0, dtype=torch.float64, device="cuda")
        u64 = torch.tensor(u0, dtype=torch.float64, device="cuda")
        phi32 = torch.tensor(phi0, dtype=torch.float32, device="cuda")
        u32 = torch.tensor(u0, dtype=torch.float32, device="cuda")
        plan64.step(phi64, u64, 1)
        plan.step(phi32, u32, 1)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        plan64.step(phi64, u64, a.fp64_steps)
        f1.record(stream)
        plan.step(phi32, u32, a.fp64_steps)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / a.fp64_steps
        G = 18.0 * (phi64 * phi64 - phi64) ** 2

        def rel(x, y, sel=None, wt=None):
            x = x.double()
            if sel is not None:
                x, y = x[sel], y[sel]
            if wt is not None:
                return float(torch.sqrt((wt * (x - y) ** 2).sum() / (wt * y ** 2).sum()))
            return float(torch.linalg.vector_norm(x - y) / torch.linalg.vector_norm(y))

        d64 = plan64.energy(phi64, u64)
        d32 = plan.energy(phi32, u32)
        # the FP64 form against a measured FP64 rate: cuBLAS DGEMM (4096^3) on this GPU, and the
        # FFT flops of the step (19 real transforms of 2.5 N log2 N flops each, the standard count;
        # the pointwise and band-solve flops are left out, so the fraction is a lower bound)
        A = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
        B = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
        torch.matmul(A, B)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(3):
            torch.matmul(A, B)
        g1.record(stream)
        torch.cuda.synchronize()
        dgemm_tflops = 3 * 2 * 4096 ** 3 / (g0.elapsed_time(g1) / 1e3) / 1e12
        del A, B
        fft_flops = 19 * 2.5 * npts * math.log2(npts)
        fp64_ach = fft_flops / (ms64 / 1e3) / 1e12
        e64, e32 = d64["energy"], d32["energy"]
        fp64 = {"ms_per_step": ms64, "value": npts / (ms64 / 1e3) / 1e6, "unit": UNIT,
                "speedup_fp32_over_fp64": ms64 / (ms / a.steps), "steps_compared": a.fp64_steps + 1,
                "rel_l2_phi": rel(phi32, phi64), "rel_l2_u_G": rel(u32, u64, wt=G),
                "rel_l2_u": rel(u32, u64), "rel_l2_u_recovery": rel(u32, u64, G > p.recover_delta),
                "rel_l2_u_core": rel(u32, u64, G > 0.1), "rel_energy": abs(e32 - e64) / abs(e64),
                "max_bound_fp32": d32["max_bound"], "max_bound_fp64": d64["max_bound"],
                "roofline": {"bound": "fp64", "achieved": fp64_ach, "peak": dgemm_tflops, "unit": "TFLOP/s",
                             "frac": fp64_ach / dgemm_tflops, "flops_per_step": fft_flops,
                             "peak_source": "measured cuBLAS DGEMM 4096^3 on this GPU",
                             "flops": "FFT only: 19 real transforms x 2.5 N log2 N"}}
        plan64.close()

    batch = None
    if not a.no_batch and rank == 0 and prec == 1:
        batch = batch_leg(stream, peak)
    sec2 = None
    if not a.no_sec2 and rank == 0:
        sec2 = sec2_leg(stream, peak)

    # end to end through the public API with host buffers
    esize = 4 if prec else 8
    h_phi = torch.from_numpy(phi0.astype(np.float32 if prec else np.float64)).pin_memory()
    h_u = torch.from_numpy(u0.astype(np.float32 if prec else np.float64)).pin_memory()
    # each end-to-end step is an independent call on fresh host input (copy in, one step, copy
    # out); two plans on two streams take alternate steps, so one step's host copies overlap
    # the other's kernels (every copy and every kernel stays inside the timed region)
    lanes = []
    for _ in range(2):
        st = torch.cuda.Stream()
        lanes.append((Plan(p, stream=st), st, torch.empty_like(phi), torch.empty_like(u),
                      torch.empty_like(h_phi).pin_memory(), torch.empty_like(h_u).pin_memory()))
    for pl, st, dphi, du, _, _ in lanes:      # first call of each plan, untimed
        with torch.cuda.stream(st):
            dphi.copy_(h_phi, non_blocking=True)
            du.copy_(h_u, non_blocking=True)
            pl.step(dphi, du, 1)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(a.e2e_steps):
        pl, st, dphi, du, hphi, hu = lanes[k % 2]
        with torch.cuda.stream(st):
            dphi.copy_(h_phi, non_blocking=True)
            du.copy_(h_u, non_blocking=True)
            pl.step(dphi, du, 1)
            hphi.copy_(dphi, non_blocking=True)
            hu.copy_(du, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    for ln in lanes:
        ln[0].close()
    del lanes
    barrier()
    t_e2e = allreduce_max(t_e2e, world)
    e2e = aggregate(world, npts, a.e2e_steps, 1e3 * t_e2e)

    line = None
    if rank == 0:
        cpu = None
        if not a.no_cpu_baseline and world == 1:
            cpu = cpu_baselines(a)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec else "f64", "data": "synthetic",
            "config": {"workload": f"c3: 3D coupled phi-u, stabilised ETDRK2, narrow band, {a.size}^3 on "
                                   "[-pi,pi)^3, ellipsoid (1.2,0.9,0.9), seed 2, tau=1e-4",
                       "grid": a.size, "precision": "fp32 storage/FFT, fp64 tables+reductions" if prec else "fp64",
                       "parallelism": f"replicas x{world}",
                       "l2": "per-step traffic ~2 GB >> 129 MB L2: no flush needed",
                       "band_size": d["band_size"], "cg_iters_last": d["cg_iters_last"]},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src,
                         "traffic": recorded_traffic(dom, a.size, a.precision, dbytes / max(dn, 1)),
                         "algo_bytes_per_launch": dbytes / max(dn, 1), "avg_launch_ms": dms / max(dn, 1)},
            "step_roofline": {"bound": "hbm", "bytes_per_step": step_bytes / a.steps,
                              "bytes_per_point_step": step_bytes / a.steps / npts, "achieved": step_achieved,
                              "peak": peak, "unit": "GB/s", "frac": step_achieved / peak},
            "fp64_gpu": fp64,
            "batch_c4": batch,
            "sec2_2d": sec2,
            "kernel_ms": {k: round(v[0], 3) for k, v in kt.items()},
            "kernel_ms_steps": a.steps, "timed_with_events_ms_per_step": ms_t / a.steps,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 2 * npts * esize,
                    "d2h_bytes_per_step": 2 * npts * esize, "steps": a.e2e_steps,
                    "how": "one etd_step call per step on pinned host input and output, two plans on two streams "
                           "taking alternate steps"},
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
