#!/usr/bin/env python3
"""Benchmark of the coupled LBM hot path on GB300.

Workload (default): the FP32 fused flow + heat kernel on a single 4096 x 2048
analytic eye (tau 0.6, Ra 1e5, TM permeability 0.5 cells^2, upright).  One
benchmark step is one check interval of the steady-state loop: 99 plain time
steps plus one time step with the fused FP64 observable reductions (IOP,
fluxes, mass, peak speed, wall shear, residual against the previous
snapshot), i.e. 100 lattice updates of every active cell.  The default of 200
steps is the 20,000 time steps of the workload.

Printed metric: MLUPS over active (fluid + porous) cells.  Inputs are
resident in HBM; the per-step working set (~150 MB of populations in active
tiles) exceeds the 129 MB L2.

--impl reference times the FP64 C oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 4096, 2048
CHECK = 100
KERNEL_SOURCES = ["paper_2102_12663_gb300/csrc/kernel_body.cuh",
                  "paper_2102_12663_gb300/csrc/lbm_internal.cuh",
                  "paper_2102_12663_gb300/csrc/step_lp.cu"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_fp32_traffic.json")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the
    timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def eye_params():
    from paper_2102_12663_gb300 import workloads as W
    return W.config_params(W.CONFIG_FP32)


def oracle_sample(seconds_budget: float = 15.0, threads: int | None = None):
    """Times the FP64 C oracle on the 4096 x 2048 eye: a bounded number of
    steps after initialisation.  Returns (MLUPS over active cells, steps,
    cores, seconds)."""
    import numpy as np

    import oracle as O
    threads = threads or os.cpu_count() or 1
    O.set_threads(threads)
    m, g = O.eye_mask(NX, NY, 45.0)
    n_active = int(((m == 0) | (m == 1)).sum())
    st = O.State(g, O.make_params(**eye_params()), m)
    t0 = time.perf_counter()
    st.run(1)
    one = time.perf_counter() - t0
    steps = max(1, int(seconds_budget / max(one, 1e-3)))
    t0 = time.perf_counter()
    st.run(steps)
    dt = time.perf_counter() - t0
    del st
    return n_active * steps / dt / 1e6, steps, threads, dt


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    per_step = []
    n_active = None
    for k in range(args.warmup + args.steps):
        mlups, steps, cores, dt = oracle_sample(seconds_budget=8.0)
        if k >= args.warmup:
            per_step.append(mlups)
    value = statistics.median(per_step)
    line = {
        "impl": "reference", "metric": "coupled MLUPS (active cells)", "value": value,
        "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "eye 4096x2048, FP64 CPU oracle, bounded sample per step",
                   "cores": cores},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{steps} time steps of the 4096x2048 eye per bench step"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2102_12663_gb300 import lbm
    lbm.load(build_if_missing=True)
    stream = torch.cuda.Stream(device=dev)
    pp = eye_params()
    dom = lbm.Domain(dict(nx=NX, ny=NY, angle_deg=45.0), precision="f32", device=dev, stream=stream)
    dom.set_launch(**LAUNCH)
    dom.set_params(pp)
    info = dom.info()
    n_active = info["n_active"]
    step_bytes = dom.step_bytes()

    def bench_step():
        dom.run_to_steady(0.0, check_every=CHECK, max_steps=CHECK)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            bench_step()
        stream.synchronize()

        # dominant kernel alone: average duration of the plain fused step
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nk = 200
        ev0.record(stream)
        dom.step(nk)
        ev1.record(stream)
        ev1.synchronize()
        kernel_ms = ev0.elapsed_time(ev1) / nk

        # timed region: K bench steps (K * 100 lattice updates)
        if world > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                              if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit()
                              else local)
        clocks.start()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            bench_step()
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        total_ms = e0.elapsed_time(e1)
        clk = clocks.stop()

        # end to end through the public API: parameters in (host -> device
        # descriptor upload) and observables out (device -> host) every step
        h2d = 0
        d2h = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            dom.set_params(pp)
            bench_step()
            dom.observables()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        h2d = 312  # descriptor bytes uploaded by set_params
        d2h = 2 * 12 * 8  # residual check + observables read-back

    t_max = total_ms
    if world > 1:
        t = torch.tensor([total_ms, e2e_s], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max, e2e_s = float(t[0]), float(t[1])
    updates = n_active * CHECK * args.steps * world
    value = updates / (t_max * 1e-3) / 1e6
    e2e_value = updates / e2e_s / 1e6
    peak, peak_kind = hbm_peak()
    achieved = step_bytes / (kernel_ms * 1e-3) / 1e9
    traffic = None
    try:
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        if tr.get("kernel_hash") == kernel_hash() and tr.get("launch") == LAUNCH:
            traffic = tr.get("dram_bytes_per_launch")
    except Exception:
        pass
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mlups_cpu, steps_cpu, cores, dt = oracle_sample(seconds_budget=12.0)
        cpu = {"value": mlups_cpu, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{steps_cpu} time steps of the 4096x2048 eye ({dt:.1f} s, FP64, OpenMP rows)"}
    if rank == 0:
        line = {
            "metric": "coupled MLUPS (active cells)", "value": value, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "FP32 fused flow+heat step, single 4096x2048 analytic eye "
                                   "(tau 0.6, Ra 1e5, K 0.5), 100 time steps per bench step "
                                   "(99 plain + 1 with fused FP64 observables)",
                       "nx": NX, "ny": NY, "active_cells": n_active,
                       "mlups_all_cells": NX * NY * CHECK * args.steps * world / (t_max * 1e-3) / 1e6,
                       "launch": LAUNCH, "l2": "working set > L2 (no flush needed)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind,
                         "kernel": "step_kernel<StF32,false>", "kernel_ms": kernel_ms,
                         "algorithmic_bytes_per_launch": step_bytes},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * (CHECK + 1),
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    dom.close()
    return 0


LAUNCH = dict(tile_w=64, block_rows=1, rows_per_thread=4, blocks_per_sm=0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", type=int, default=0,
                    help="profiling driver: run this many single fused steps of the "
                         "workload (no timing, no JSON line) and exit")
    ap.add_argument("--precision", default="f32", choices=["f32", "f16", "bf16", "f64"],
                    help="storage precision for --profile")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)
    return run_gpu(args)


def run_profile(args):
    """A short, fixed sequence of single-step launches for ncu captures."""
    import torch

    from paper_2102_12663_gb300 import lbm
    lbm.load(build_if_missing=True)
    dom = lbm.Domain(dict(nx=NX, ny=NY, angle_deg=45.0), precision=args.precision)
    dom.set_launch(**LAUNCH)
    dom.set_params(eye_params())
    for _ in range(args.profile):
        dom.step(1)
    torch.cuda.synchronize()
    print(f"profile driver: {args.profile} steps, {dom.tile_count()} tiles, "
          f"{dom.step_bytes():.0f} algorithmic bytes per step", flush=True)
    dom.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
