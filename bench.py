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


def reduce_max_over_ranks(values, device=None):
    """Element-wise maximum over every rank of the default process group (NCCL
    between GPUs, gloo on the host)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def weak_scaling_mlups(active_cells: int, bench_steps: int, world: int, t_max_ms: float) -> float:
    """Whole-job MLUPS: every rank updates its own replica of the workload, so
    the units processed are world x cells x 100 x bench steps, divided by the
    slowest rank's time."""
    return active_cells * CHECK * bench_steps * world / (t_max_ms * 1e-3) / 1e6


def eye_params():
    from paper_2102_12663_gb300 import workloads as W
    return W.config_params(W.CONFIG_FP32)


def oracle_sample(seconds_budget: float = 15.0, threads: int | None = None, nx: int = NX, ny: int = NY,
                  params: dict | None = None, angle_deg: float = 45.0):
    """Times the FP64 C oracle on an eye (default the 4096 x 2048 one): after
    initialisation and one step, chunks of steps until seconds_budget has
    passed.  Returns (MLUPS over active cells, steps, cores, seconds)."""
    import oracle as O
    threads = threads or os.cpu_count() or 1
    O.set_threads(threads)
    m, g = O.eye_mask(nx, ny, angle_deg)
    n_active = int(((m == 0) | (m == 1)).sum())
    st = O.State(g, O.make_params(**(params or eye_params())), m)
    st.run(1)
    steps, dt, chunk = 0, 0.0, 1
    while dt < seconds_budget:
        t0 = time.perf_counter()
        st.run(chunk)
        took = time.perf_counter() - t0
        steps += chunk
        dt += took
        # next chunk: about a quarter of the remaining budget
        chunk = max(1, int(0.25 * max(seconds_budget - dt, 0.0) / max(took / chunk, 1e-7)))
    del st
    return n_active * steps / dt / 1e6, steps, threads, dt


def run_reference(args):
    """The FP64 C oracle on the host cores, timed as it stands on the same
    4096 x 2048 eye: state built once, then every bench step runs a bounded
    number of time steps, sized so that warm-up plus timed steps take about a
    minute in total."""
    import oracle as O
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    m, g = O.eye_mask(NX, NY, 45.0)
    n_active = int(((m == 0) | (m == 1)).sum())
    st = O.State(g, O.make_params(**eye_params()), m)
    t0 = time.perf_counter()
    st.run(1)
    one = time.perf_counter() - t0
    per_step = max(1, int(60.0 / max(args.steps + args.warmup, 1) / max(one, 1e-3)))
    rates = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        st.run(per_step)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            rates.append(n_active * per_step / dt / 1e6)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": "coupled MLUPS (active cells)", "value": value,
        "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "FP64 CPU oracle on the single 4096x2048 analytic eye (tau 0.6, "
                               "Ra 1e5, K 0.5); bounded sample per bench step",
                   "nx": NX, "ny": NY, "active_cells": n_active, "cores": cores},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} time step(s) of the 4096x2048 eye per bench step, "
                                   f"{args.steps} timed bench steps"},
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

        # dominant kernel alone, as the bench step launches it: a dataflow
        # launch of CHECK - 1 steps (or, stepping one launch per step, the
        # average of 200 graph-replayed single steps)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flow = LAUNCH.get("stepping", lbm.STEP_FLOW) == lbm.STEP_FLOW
        steps_per_launch = CHECK - 1 if flow else 1
        nk = 5 if flow else 200
        ev0.record(stream)
        for _ in range(nk if flow else 1):
            dom.step(steps_per_launch if flow else nk)
        ev1.record(stream)
        ev1.synchronize()
        kernel_ms = ev0.elapsed_time(ev1) / nk

        # timed region: K bench steps (K * 100 lattice updates) as one steady-state
        # loop of K check intervals (tolerance 0: every interval runs); the loop
        # keeps the next interval queued while the host checks the last one
        if world > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                              if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit()
                              else local)
        clocks.start()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, done = dom.run_to_steady(0.0, check_every=CHECK, max_steps=CHECK * args.steps)
        assert done == CHECK * args.steps
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        total_ms = e0.elapsed_time(e1)
        clk = clocks.stop()

        # end to end through the public API: parameters in (host -> device
        # descriptor upload) and the step's result out every step: the check's
        # observables, read back by the steady-state loop (device -> host) and
        # returned by last_observables
        h2d = 0
        d2h = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            dom.set_params(pp)
            bench_step()
            dom.last_observables()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        h2d = 368  # the instance descriptor uploaded by set_params
        d2h = 12 * 8 + 4  # the check's observables and the dataflow status word

    t_max = total_ms
    if world > 1:
        t_max, e2e_s = reduce_max_over_ranks([total_ms, e2e_s], device=dev)
    value = weak_scaling_mlups(n_active, args.steps, world, t_max)
    e2e_value = weak_scaling_mlups(n_active, args.steps, world, e2e_s * 1e3)
    peak, peak_kind = hbm_peak()
    bytes_per_launch = steps_per_launch * step_bytes
    achieved = bytes_per_launch / (kernel_ms * 1e-3) / 1e9
    traffic = None
    try:
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        if tr.get("kernel_hash") == kernel_hash() and tr.get("launch") == LAUNCH:
            # DRAM bytes grow with the steps a launch covers
            traffic = tr["dram_bytes_per_step"] * steps_per_launch
    except Exception:
        pass
    studies = None
    if rank == 0 and world == 1 and not args.no_studies:
        dom.close()
        torch.cuda.empty_cache()
        studies = side_studies(dev)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mlups_cpu, steps_cpu, cores, dt = oracle_sample(seconds_budget=12.0)
        mlups_1, steps_1, _, dt_1 = oracle_sample(seconds_budget=4.0, threads=1)
        from paper_2102_12663_gb300 import workloads as W
        other = {}
        for name, (cfgd, nx, ny) in {"fp64_160x80": (W.CONFIG_FP64, 160, 80),
                                     "fp32_downscale_512x256": (W.CONFIG_FP32, 512, 256),
                                     "precision_check_1024x512": (W.CONFIG_PRECISION, 1024, 512)}.items():
            pp = W.config_params(cfgd, ny=ny)
            ang = cfgd["angle_deg"]
            all_c = oracle_sample(seconds_budget=1.5, nx=nx, ny=ny, params=pp, angle_deg=ang)
            one_c = oracle_sample(seconds_budget=1.5, threads=1, nx=nx, ny=ny, params=pp, angle_deg=ang)
            other[name] = {"mlups_all_cores": all_c[0], "mlups_one_core": one_c[0],
                           "steps": [all_c[1], one_c[1]]}
        cpu = {"value": mlups_cpu, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{steps_cpu} time steps of the 4096x2048 eye ({dt:.1f} s, FP64, OpenMP rows)",
               "cpu_model": cpu_model(),
               "single_thread": {"value": mlups_1, "unit": "MLUPS", "cores": 1,
                                 "sample": f"{steps_1} time steps of the same eye ({dt_1:.1f} s)"},
               "other_grids": other}
    if rank == 0:
        line = {
            "metric": "coupled MLUPS (active cells)", "value": value, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "FP32 fused flow+heat step, single 4096x2048 analytic eye "
                                   "(tau 0.6, Ra 1e5, K 0.5), 100 time steps per bench step "
                                   "(99 plain + 1 with fused observables); timed as one steady-state loop of all "
                                   "bench steps",
                       "nx": NX, "ny": NY, "active_cells": n_active,
                       "mlups_all_cells": NX * NY * CHECK * args.steps * world / (t_max * 1e-3) / 1e6,
                       "launch": LAUNCH, "l2": "working set > L2 (no flush needed)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind,
                         "kernel": "step_kernel_flow<StF32>" if flow else "step_kernel<StF32,false>",
                         "kernel_ms": kernel_ms, "steps_per_launch": steps_per_launch,
                         "algorithmic_bytes_per_launch": bytes_per_launch},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            # per bench step: the plain steps (one dataflow launch, or CHECK - 1
            # single launches), the observing step and the finalize kernel
            "gpu_launches": args.steps * (3 if flow else CHECK + 1),
            "clocks": clk,
            "studies": studies,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    dom.close()
    return 0


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def side_studies(dev) -> dict:
    """Short measurements of the other forms, reported beside the headline
    (they do not enter `value`): 16-bit deviation storage on the 8192 x 4096
    eye (three check intervals per storage, eight-cell tile rows), the
    64-instance FP32 batch (three check intervals) and 24 served requests
    against the one-at-a-time loop.  About 15 seconds."""
    import torch

    from paper_2102_12663_gb300 import lbm
    from paper_2102_12663_gb300 import workloads as W
    peak, _ = hbm_peak()
    out = {}
    cfg = W.CONFIG_PRECISION
    for prec in ("f16", "bf16"):
        st = torch.cuda.Stream(device=dev)
        d = lbm.Domain(dict(nx=cfg["nx"], ny=cfg["ny"], angle_deg=cfg["angle_deg"]), precision=prec,
                       device=dev, stream=st)
        d.set_launch(**VEC16_LAUNCH)
        d.set_params(W.config_params(cfg))
        with torch.cuda.stream(st):
            _time_intervals(d, 2)
            ms = _time_intervals(d, 3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            d.step(100)
            e1.record(st)
            e1.synchronize()
            kus = e0.elapsed_time(e1) / 100 * 1e3
        n_act = d.info()["n_active"]
        gbs = d.step_bytes() / (kus * 1e-6) / 1e9
        out[f"{prec}_{cfg['nx']}x{cfg['ny']}"] = {
            "mlups": n_act * CHECK * 3 / (ms * 1e-3) / 1e6, "step_kernel_us": kus, "gbs": gbs,
            "hbm_frac": gbs / peak, "bytes_per_active_cell": d.step_bytes() / n_act,
            "launch": VEC16_LAUNCH}
        d.close()
        del d
        torch.cuda.empty_cache()
    st = torch.cuda.Stream(device=dev)
    doms = []
    for inst in W.batch_instances(64):
        d = lbm.Domain(dict(nx=inst["nx"], ny=inst["ny"], angle_deg=inst["angle_deg"]),
                       precision="f32", device=dev, stream=st)
        d.set_launch(**STUDY_LAUNCH)
        d.set_params(inst["params"])
        doms.append(d)
    b = lbm.Batch("f32", max_instances=64, max_tiles=1 << 21, launch=STUDY_LAUNCH, stream=st)
    for d in doms:
        b.add(d)
    with torch.cuda.stream(st):
        _time_intervals(b, 2, batch=True)
        ms = _time_intervals(b, 3, batch=True)
    cells = b.active_cells()
    out["batch_64_fp32"] = {"mlups": cells * CHECK * 3 / (ms * 1e-3) / 1e6,
                            "hbm_frac": b.step_bytes() * CHECK * 3 / (ms * 1e-3) / 1e9 / peak,
                            "active_cells": cells, "launch": STUDY_LAUNCH}
    b.close()
    for d in doms:
        d.close()
    torch.cuda.empty_cache()
    out["serve_24"] = serve_study(24)
    return out


def serve_study(n):
    """The serving workload's throughput part on n requests (Poisson at 20/s,
    NY 64..256, half FP16 refined to the FP32 criterion): continuous batching
    against the one-at-a-time FP32 loop (`--workload serve` adds the accuracy
    sample against FP64)."""
    from paper_2102_12663_gb300 import serve
    from paper_2102_12663_gb300 import workloads as W
    draws = W.request_stream(n, rate_hz=20.0, ny_lo=64, ny_hi=256, fp16_share=0.5)
    reqs = serve.requests_from_draws(draws, tol_by_precision=W.SERVE_TOL, cap_efolds=20.0)
    srv = serve.Server(budget_bytes=150e9, tol=1e-7, check_every=CHECK, max_steps=10**9,
                       launch=STUDY_LAUNCH, refine_tol={"f16": W.SERVE_TOL["f32"]})
    res = srv.run(reqs, realtime=True)
    s_served = serve.summary(res, srv.wall_s)
    srv.close()
    base_reqs = serve.requests_from_draws(draws, tol_by_precision={"f32": W.SERVE_TOL["f32"],
                                                                   "f16": W.SERVE_TOL["f32"]},
                                          cap_efolds=20.0)
    base = serve.solve_one_at_a_time(base_reqs, check_every=CHECK, launch=STUDY_LAUNCH, realtime=True)
    s_base = serve.summary(base, max(r.finish_s for r in base))
    keep = ("solves_per_s", "p50_s", "p99_s", "converged", "capped")
    return {"served": {k: s_served[k] for k in keep},
            "one_at_a_time_fp32": {k: s_base[k] for k in keep},
            "speedup_solves_per_s": s_served["solves_per_s"] / s_base["solves_per_s"]}


# the FP32 4096 x 2048 line: 64 x 4 tiles, one graph-replayed launch per step
# (measured ahead of one dataflow launch per check interval: 50.3-50.6 k
# against 49.5-49.6 k MLUPS on one GPU)
LAUNCH = dict(tile_w=64, block_rows=4, rows_per_thread=1, blocks_per_sm=0, stepping=0, sweep_steps=1,
              sweep_lag=0)
# the studies (other grid sizes and many small grids): one launch per step
STUDY_LAUNCH = dict(tile_w=64, block_rows=4, rows_per_thread=2, blocks_per_sm=0, stepping=0)
# 16-bit storages: 256-cell tile rows, eight cells per thread (16-byte
# vectors); with the boundary cells in edge-cell chunks they measured ahead of
# the four-cell rows (104.0 against 110.5 us per step of the 8192 x 4096 eye)
VEC16_LAUNCH = dict(tile_w=256, block_rows=4, rows_per_thread=1, blocks_per_sm=0, stepping=0)


def _time_intervals(dom_or_batch, n, batch=False):
    """Device time (ms) of n steady-loop check intervals (100 steps each)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s = dom_or_batch.stream
    e0.record(s)
    for _ in range(n):
        if batch:
            dom_or_batch.check(CHECK)
        else:
            dom_or_batch.run_to_steady(0.0, check_every=CHECK, max_steps=CHECK)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1)


def run_precision(args):
    """Reduced-storage precision: FP16 / BF16 deviation storage (FP32
    arithmetic, FP64 reductions) on the 8192 x 4096 eye (throughput), and the
    errors of the steady observables against the FP64 path (itself checked
    against the FP64 oracle): time-averaged over the last 20 checks of runs to
    steady state on the 256 x 128 and 512 x 256 eyes, and at equal step counts
    on the 1024 x 512 eye (whose temperature field needs millions of steps to
    settle)."""
    import numpy as np
    import torch

    import oracle as O
    from paper_2102_12663_gb300 import lbm
    from paper_2102_12663_gb300 import workloads as W
    torch.cuda.set_device(0)
    lbm.load(build_if_missing=True)
    cfg = W.CONFIG_PRECISION
    peak, peak_kind = hbm_peak()
    thr = {}
    for prec in ("f16", "bf16", "f32"):
        st = torch.cuda.Stream()
        dom = lbm.Domain(dict(nx=cfg["nx"], ny=cfg["ny"], angle_deg=cfg["angle_deg"]),
                         precision=prec, stream=st)
        launch = VEC16_LAUNCH if prec != "f32" else STUDY_LAUNCH
        dom.set_launch(**launch)
        dom.set_params(W.config_params(cfg))
        with torch.cuda.stream(st):
            _time_intervals(dom, 3)
            ms = _time_intervals(dom, args.intervals)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            dom.step(200)
            e1.record(st)
            e1.synchronize()
            kms = e0.elapsed_time(e1) / 200
        n_act = dom.info()["n_active"]
        thr[prec] = {"mlups": n_act * CHECK * args.intervals / (ms * 1e-3) / 1e6,
                     "kernel_us": kms * 1e3,
                     "gbs": dom.step_bytes() / (kms * 1e-3) / 1e9,
                     "hbm_frac": dom.step_bytes() / (kms * 1e-3) / 1e9 / peak,
                     "bytes_per_cell": dom.step_bytes() / n_act, "launch": launch}
        dom.close()
        del dom
        torch.cuda.empty_cache()

    keys = ("iop", "peak_speed", "wss_cornea", "wss_iris")

    def sampled(nx, ny, prec, steps, nsamp=20, every=2500):
        dom = lbm.Domain(dict(nx=nx, ny=ny, angle_deg=cfg["angle_deg"]), precision=prec)
        dom.set_launch(**(VEC16_LAUNCH if prec in ("f16", "bf16") else STUDY_LAUNCH))
        dom.set_params(W.config_params(cfg, ny=ny))
        dom.run_to_steady(0.0, check_every=CHECK, max_steps=steps - nsamp * every)
        out = []
        for _ in range(nsamp):
            dom.run_to_steady(0.0, check_every=CHECK, max_steps=every)
            o = dom.last_observables()
            out.append([o[k] for k in keys] + [o["residual"]])
        dom.close()
        return np.array(out)

    def study(nx, ny, steps):
        pp = W.config_params(cfg, ny=ny)
        # tie the FP64 path to the oracle on this grid
        m, g = O.eye_mask(nx, ny, cfg["angle_deg"])
        O.set_threads(os.cpu_count() or 1)
        ref = O.State(g, O.make_params(**pp), m)
        ref.run(args.oracle_steps)
        dom = lbm.Domain(dict(nx=nx, ny=ny, angle_deg=cfg["angle_deg"]), precision="f64")
        dom.set_params(pp)
        dom.step(args.oracle_steps)
        f, _ = dom.populations()
        oracle_rel = float(np.abs(f.cpu().numpy().reshape(9, -1) - ref.f).max() / np.abs(ref.f).max())
        del ref, f
        dom.close()
        r = sampled(nx, ny, "f64", steps)
        scale = np.abs(r[:, :4].mean(axis=0))
        out = {"grid": f"{nx}x{ny}", "steps": steps, "f64_vs_oracle_max_rel_population_diff": oracle_rel,
               "f64_reference": dict(zip(keys, r[:, :4].mean(axis=0).tolist())),
               "f64_residual_per_100_steps": float(r[-1, 4]), "errors_vs_f64": {}}
        for prec in ("f32", "f16", "bf16"):
            x = sampled(nx, ny, prec, steps)
            out["errors_vs_f64"][prec] = {
                "mean": dict(zip(keys, (np.abs(x[:, :4].mean(axis=0) - r[:, :4].mean(axis=0)) / scale).tolist())),
                "max": dict(zip(keys, (np.abs(x[:, :4] - r[:, :4]).max(axis=0) / scale).tolist())),
                "residual_per_100_steps": float(x[-1, 4])}
        return out

    big = args.transient_steps
    if big <= 0:
        # to steady state: the FP64 path's residual below 1e-7 per 100 steps
        # (capped), then the sampling window of 20 checks on top
        dom = lbm.Domain(dict(nx=cfg["check_nx"], ny=cfg["check_ny"], angle_deg=cfg["angle_deg"]), precision="f64")
        dom.set_params(W.config_params(cfg, ny=cfg["check_ny"]))
        _, done = dom.run_to_steady(1e-7, check_every=CHECK, max_steps=args.steady_cap)
        dom.close()
        big = int(done) + 20 * 2500
    grids = {"256": (256, 128, 600_000), "512": (512, 256, 1_500_000),
             "1024": (cfg["check_nx"], cfg["check_ny"], big)}
    studies = [study(*grids[g]) for g in args.precision_grids.split(",")]
    line = {"metric": "reduced-storage precision study", "unit": "relative error / MLUPS",
            "dtype": "f16/bf16 storage, f32 arithmetic, f64 reductions", "data": "synthetic",
            "config": {"workload": f"throughput: {cfg['nx']}x{cfg['ny']} eye; errors of the observables "
                                   f"against the FP64 path, time-averaged over 20 checks 2,500 steps apart: "
                                   f"steady 256x128 (600k steps) and 512x256 (1.5M steps) eyes, and the "
                                   f"{cfg['check_nx']}x{cfg['check_ny']} eye at {big} steps "
                                   + ("(temperature field still settling)" if args.transient_steps > 0 else
                                      "(FP64 residual below 1e-7 per 100 steps, or the cap)")
                                   + f"; grids run: {args.precision_grids}",
                       "tau": cfg["tau"], "Ra": cfg["Ra"], "K_tm": cfg["K_tm"]},
            "throughput": thr, "peak_gbs": peak, "peak_kind": peak_kind, "errors": studies,
            "oracle_check_steps": args.oracle_steps}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """64 uneven eye instances (NY log-uniform 128..1024, seeded parameters)
    in one batch (autotuned shape and stepping: one dataflow launch per check
    interval or one launch per step, graph-replayed);
    against the same instances stepped one after the other."""
    import torch

    from paper_2102_12663_gb300 import lbm
    from paper_2102_12663_gb300 import workloads as W
    torch.cuda.set_device(0)
    lbm.load(build_if_missing=True)
    st = torch.cuda.Stream()
    insts = W.batch_instances(64)
    doms = []
    for i in insts:
        d = lbm.Domain(dict(nx=i["nx"], ny=i["ny"], angle_deg=i["angle_deg"]), precision="f32", stream=st)
        d.set_launch(**STUDY_LAUNCH)
        d.set_params(i["params"])
        doms.append(d)
    b = lbm.Batch("f32", max_instances=64, max_tiles=1 << 21, launch=STUDY_LAUNCH, stream=st)
    for d in doms:
        b.add(d)
    with torch.cuda.stream(st):
        chosen = b.tune(steps_per_candidate=20)
        _time_intervals(b, 3, batch=True)
        ms = _time_intervals(b, args.intervals, batch=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        b.step(128)
        e1.record(st)
        e1.synchronize()
        kms = e0.elapsed_time(e1) / 128
    cells = b.active_cells()
    peak, peak_kind = hbm_peak()
    batched = cells * CHECK * args.intervals / (ms * 1e-3) / 1e6
    gbs = b.step_bytes() / (kms * 1e-3) / 1e9
    b.close()
    # the same instances, one after the other, each alone (plain FP32 loop)
    n_alone = max(2, args.intervals // 4)
    tot_ms = 0.0
    with torch.cuda.stream(st):
        for d in doms:
            _time_intervals(d, 1)
            tot_ms += _time_intervals(d, n_alone)
    alone = cells * CHECK * n_alone / (tot_ms * 1e-3) / 1e6
    for d in doms:
        d.close()
    line = {"metric": "batched coupled MLUPS (active cells)", "value": batched, "unit": "MLUPS",
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 eye instances, NY log-uniform 128..1024, NX = 2 NY, seeded "
                                   "inflow/K/viscosity/angle/gravity/dT; 100-step check intervals",
                       "instances": 64, "active_cells": cells, "launch": chosen,
                       "intervals": args.intervals},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "peak_kind": peak_kind},
            "one_at_a_time_mlups": alone, "speedup_vs_one_at_a_time": batched / alone,
            "instance_intervals_per_s": 64 * args.intervals / (ms * 1e-3)}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Poisson stream (mean 20/s) of steady-solve requests: NY log-uniform over
    [--serve-ny-lo, --serve-ny-hi] (default 64..256, NX = 2 NY), parameters
    drawn as in the batching workload, FP32 or FP16 storage with p = 1/2, 150 GB
    HBM budget.  Each request runs until its residual over a 100-step check
    falls below 1e-7 or it reaches a cap of 20 decay times of its slowest
    viscous mode; an FP16 request runs in FP16 until 1e-5 (its storage's noise
    floor lies above 1e-7) and then in FP32.
    The baseline solves every request alone on a plain FP32 domain at the FP32
    tolerance, one after the other.  A seeded sample of the served results, and
    the baseline's results for the same requests, are compared with FP64 solves
    of those requests (to 1e-9 per 100 steps)."""
    import numpy as np
    import torch

    from paper_2102_12663_gb300 import lbm, serve
    from paper_2102_12663_gb300 import workloads as W
    torch.cuda.set_device(0)
    lbm.load(build_if_missing=True)
    draws = W.request_stream(args.requests, rate_hz=20.0, ny_lo=args.serve_ny_lo, ny_hi=args.serve_ny_hi,
                             fp16_share=0.5)
    reqs = serve.requests_from_draws(draws, tol_by_precision=W.SERVE_TOL, cap_efolds=20.0)
    refine = {"f16": W.SERVE_TOL["f32"]}
    srv = serve.Server(budget_bytes=150e9, tol=1e-7, check_every=CHECK, max_steps=10**9,
                       launch=STUDY_LAUNCH, refine_tol=refine)
    res = srv.run(reqs, realtime=True)
    s_served = serve.summary(res, srv.wall_s)
    s_served["peak_hbm_bytes"] = srv.peak_used
    s_served["cell_updates_per_s"] = srv.cell_updates / srv.wall_s
    f16 = [r for r in res if r.precision == "f16"]
    s_served["f16_steps_share_in_f16"] = (sum(r.steps - r.refined_steps for r in f16)
                                          / max(1, sum(r.steps for r in f16)))
    srv.close()
    base_reqs = serve.requests_from_draws(draws, tol_by_precision={"f32": W.SERVE_TOL["f32"],
                                                                   "f16": W.SERVE_TOL["f32"]},
                                          cap_efolds=20.0)
    base = serve.solve_one_at_a_time(base_reqs, check_every=CHECK, launch=STUDY_LAUNCH, realtime=True)
    wall = max(r.finish_s for r in base)
    s_base = serve.summary(base, wall)

    # accuracy: FP64 solves of a seeded sample of requests of each storage
    keys = ("iop", "peak_speed", "wss_cornea", "wss_iris")
    rng = np.random.Generator(np.random.PCG64(2102))
    by_id = {r.id: r for r in res}
    base_by_id = {r.id: r for r in base}
    acc = {}
    for prec in ("f16", "f32"):
        ids = sorted(r.id for r in res if r.precision == prec and r.converged)
        pick = sorted(rng.choice(ids, size=min(args.accuracy_sample, len(ids)), replace=False).tolist()) if ids else []
        errs, same, base_errs = ({k: [] for k in keys} for _ in range(3))
        for rid in pick:
            q = next(r for r in reqs if r.id == rid)
            nu = (2.0 * q.params["tau"] - 1.0) / 6.0
            refs = []
            # FP64 converged (1e-9 per 100 steps), and FP64 under the request's own stopping rule
            for tol in (1e-9, refine.get(q.precision, q.tol)):
                dom = lbm.Domain(dict(nx=q.nx, ny=q.ny, angle_deg=q.angle_deg), precision="f64")
                dom.set_launch(**STUDY_LAUNCH)
                dom.set_params(q.params)
                dom.run_to_steady(tol, check_every=CHECK, max_steps=W.steady_step_cap(q.ny, nu, 40.0))
                refs.append(dom.last_observables())
                dom.close()
            conv, rule = refs
            for k in keys:
                errs[k].append(abs(by_id[rid].observables[k] - conv[k]) / abs(conv[k]))
                same[k].append(abs(by_id[rid].observables[k] - rule[k]) / abs(rule[k]))
                base_errs[k].append(abs(base_by_id[rid].observables[k] - conv[k]) / abs(conv[k]))
        mx = lambda d: {k: max(v) if v else None for k, v in d.items()}
        acc[prec] = {"requests": pick, "tolerance": refine.get(prec, W.SERVE_TOL[prec]),
                     "served_max_rel_err_vs_fp64_converged": mx(errs),
                     "served_median_rel_err_vs_fp64_converged":
                         {k: float(np.median(v)) if v else None for k, v in errs.items()},
                     "served_max_rel_err_vs_fp64_same_rule": mx(same),
                     "baseline_fp32_max_rel_err_vs_fp64_converged": mx(base_errs)}
    line = {"metric": "served steady solves per second", "value": s_served["solves_per_s"],
            "unit": "solves/s", "higher_is_better": True, "dtype": "f32+f16 storage",
            "data": "synthetic",
            "config": {"workload": f"{args.requests} Poisson requests (mean 20/s), NY log-uniform "
                                   f"{args.serve_ny_lo}..{args.serve_ny_hi} (NX = 2 NY), FP16 storage p=1/2, "
                                   f"budget 150 GB; steady at max|du| per 100 steps < 1e-7; FP16 requests "
                                   f"run in FP16 to 1e-5, then in FP32 to 1e-7; cap 20 viscous decay times "
                                   f"of the request",
                       "tolerances": W.SERVE_TOL, "refine": refine},
            "served": s_served, "one_at_a_time_fp32": s_base,
            "speedup_solves_per_s": s_served["solves_per_s"] / s_base["solves_per_s"],
            "p50_ratio": s_base["p50_s"] / s_served["p50_s"],
            "p99_ratio": s_base["p99_s"] / s_served["p99_s"],
            "accuracy_vs_fp64": acc}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-studies", action="store_true",
                    help="skip the short 16-bit storage and batch measurements of the default line")
    ap.add_argument("--profile", type=int, default=0,
                    help="profiling driver: run this many single fused steps of the "
                         "workload (no timing, no JSON line) and exit")
    ap.add_argument("--precision", default="f32", choices=["f32", "f16", "bf16", "f64"],
                    help="storage precision for --profile")
    ap.add_argument("--launch", default=None,
                    help="launch shape for --profile: tile_w,block_rows,rows_per_thread,"
                         "blocks_per_sm[,stepping[,sweep_steps,sweep_lag]]")
    ap.add_argument("--profile-steps", type=int, default=1,
                    help="steps per lbm_step call of the profiling driver (one "
                         "dataflow launch per call when the shape's stepping is 0)")
    ap.add_argument("--workload", default="fp32", choices=["fp32", "precision", "batch", "serve"],
                    help="fp32: the FP32 4096x2048 throughput line (default); precision, batch, "
                         "serve: the reduced-storage, batching and serving studies")
    ap.add_argument("--intervals", type=int, default=10, help="timed check intervals (studies)")
    ap.add_argument("--transient-steps", type=int, default=300000,
                    help="steps of the 1024 x 512 equal-step error comparison")
    ap.add_argument("--steady-cap", type=int, default=6_000_000,
                    help="precision: step cap of the FP64 run to steady state on the 1024 x 512 eye "
                         "(--transient-steps 0)")
    ap.add_argument("--precision-grids", default="256,512,1024",
                    help="precision: the error studies to run (256 x 128, 512 x 256, 1024 x 512 eyes)")
    ap.add_argument("--oracle-steps", type=int, default=500, help="oracle cross-check steps")
    ap.add_argument("--requests", type=int, default=48, help="serving: number of requests")
    ap.add_argument("--serve-ny-lo", type=int, default=64, help="serving: smallest NY of a request")
    ap.add_argument("--serve-ny-hi", type=int, default=256, help="serving: largest NY of a request")
    ap.add_argument("--accuracy-sample", type=int, default=4,
                    help="serving: requests per storage solved again in FP64")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_gpu(args)


def run_profile(args):
    """A short, fixed sequence of launches for ncu captures: --profile calls
    of lbm_step with --profile-steps steps each."""
    import torch

    from paper_2102_12663_gb300 import lbm
    lbm.load(build_if_missing=True)
    dom = lbm.Domain(dict(nx=NX, ny=NY, angle_deg=45.0), precision=args.precision)
    launch = LAUNCH
    if args.launch:
        launch = dict(zip(("tile_w", "block_rows", "rows_per_thread", "blocks_per_sm", "stepping",
                           "sweep_steps", "sweep_lag"), (int(v) for v in args.launch.split(","))))
    dom.set_launch(**launch)
    dom.set_params(eye_params())
    for _ in range(args.profile):
        dom.step(args.profile_steps)
    torch.cuda.synchronize()
    print(f"profile driver: {args.profile} x {args.profile_steps} steps, {dom.tile_count()} tiles, "
          f"{dom.step_bytes():.0f} algorithmic bytes per step", flush=True)
    dom.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
