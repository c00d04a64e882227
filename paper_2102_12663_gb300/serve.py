"""Continuous-batching server of steady-state eye solves.

Requests (a grid size, a chamber angle, lattice parameters and a storage
precision) arrive over time.  Each one is admitted as soon as its device
memory fits the HBM budget and its precision's batch has a free slot.  Its
populations then stay resident, and it advances with every other admitted
request of that precision in one fused launch per time step (lbm_batch_*).
Every tick runs one check interval of the steady-state loop for all members.
A member whose residual max |du| over the interval falls below tol, that hits
the step cap, or whose pressure turned NaN is retired: its observables are
read, its memory is released, and waiting requests take its place.  Work of
requests that arrive while others run overlaps on the device inside the
shared launches.

``solve_one_at_a_time`` is the plain baseline: every request on its own FP32
domain, one after the other, through lbm_run_to_steady.

A request may carry its own steady tolerance (the 16-bit storages settle on
a residual noise floor above the FP32 criterion) and its own step cap
(workloads.steady_step_cap: a number of decay times of its slowest mode).
With refine_tol, a 16-bit request that meets its own tolerance moves to the
FP32 batch and finishes there to the FP32 criterion: the fast transient runs
in 16-bit storage, and the result has the FP32 loop's accuracy.

This module only orchestrates; every step of every solve runs in the CUDA
library.
"""
from __future__ import annotations

import dataclasses
import statistics
import time

from . import lbm


@dataclasses.dataclass
class Request:
    id: int
    nx: int
    ny: int
    angle_deg: float
    params: dict
    precision: str = "f32"
    arrival_s: float = 0.0
    tol: float | None = None      # steady tolerance (None: the server's)
    max_steps: int | None = None  # step cap (None: the server's)


@dataclasses.dataclass
class Result:
    id: int
    precision: str
    nx: int
    ny: int
    steps: int
    converged: bool
    unstable: bool
    observables: dict
    arrival_s: float
    admit_s: float
    finish_s: float
    refined_steps: int = 0  # steps taken in FP32 after the request's own storage met its tolerance

    @property
    def latency_s(self) -> float:
        return self.finish_s - self.arrival_s


def requests_from_draws(draws, tol_by_precision: dict | None = None, cap_efolds: float | None = None,
                        check_every: int = 100) -> list:
    """Requests from workloads.request_stream / batch_instances draws.
    tol_by_precision (e.g. workloads.SERVE_TOL) sets each request's steady
    tolerance by its storage; cap_efolds sets its step cap to that many decay
    times of its slowest viscous mode (workloads.steady_step_cap)."""
    from . import workloads as W
    out = []
    for d in draws:
        prec = "f16" if d.get("fp16") else "f32"
        nu = (2.0 * d["params"]["tau"] - 1.0) / 6.0
        out.append(Request(id=d["id"], nx=d["nx"], ny=d["ny"], angle_deg=d["angle_deg"],
                           params=d["params"], precision=prec, arrival_s=d.get("arrival_s", 0.0),
                           tol=(tol_by_precision or {}).get(prec),
                           max_steps=(W.steady_step_cap(d["ny"], nu, cap_efolds, check_every)
                                      if cap_efolds else None)))
    return out


def domain_bytes(req: Request) -> int:
    import ctypes
    L = lbm.load()
    g, _ = lbm.geometry_desc(dict(nx=req.nx, ny=req.ny, angle_deg=req.angle_deg))
    return int(L.lbm_domain_bytes(ctypes.byref(g), lbm.PRECISIONS[req.precision]))


class Server:
    def __init__(self, budget_bytes: float = 150e9, tol: float = 1e-7, check_every: int = 100,
                 max_steps: int = 20000, max_instances: int = 64, max_tiles: int = 1 << 21,
                 launch: dict | None = None, autotune: bool = False, device=None, stream=None,
                 refine_tol: dict | None = None):
        """refine_tol: {storage: tol}.  A request of such a storage that meets
        its own tolerance is not retired: its state moves (on the device) to an
        FP32 domain, which runs on to `tol` of the storage (the 16-bit
        storages' residual settles above the FP32 criterion, so the fast
        transient runs in 16-bit and the end of the approach in FP32)."""
        import torch
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.budget = float(budget_bytes)
        self.tol, self.check_every, self.max_steps = tol, int(check_every), int(max_steps)
        self.max_instances, self.max_tiles = int(max_instances), int(max_tiles)
        self.launch = launch or dict(tile_w=64, block_rows=1, rows_per_thread=4, blocks_per_sm=0)
        self.autotune = autotune
        self.batches = {}
        self.active = {}  # id -> (request, domain, bytes, admit time)
        self.used = 0
        self.peak_used = 0
        self.results = []
        self.ticks = 0
        self.cell_updates = 0
        self.refine_tol = dict(refine_tol or {})
        self.refined = {}  # id -> steps taken before refinement

    def _batch(self, precision: str):
        if precision not in self.batches:
            self.batches[precision] = lbm.Batch(precision, self.max_instances, self.max_tiles,
                                                launch=self.launch, device=self.device,
                                                stream=self.stream)
        return self.batches[precision]

    def fits(self, req: Request) -> bool:
        b = self.batches.get(req.precision)
        room = b is None or len(b) < self.max_instances
        return room and self.used + domain_bytes(req) <= self.budget

    def admit(self, req: Request, now: float):
        nbytes = domain_bytes(req)
        with self.torch.cuda.stream(self.stream):
            dom = lbm.Domain(dict(nx=req.nx, ny=req.ny, angle_deg=req.angle_deg),
                             precision=req.precision, device=self.device, stream=self.stream)
            dom.set_launch(**self.launch)
            dom.set_params(req.params)
        self._batch(req.precision).add(dom)
        self.active[req.id] = (req, dom, nbytes, now)
        self.used += nbytes
        self.peak_used = max(self.peak_used, self.used)

    def tick(self, now_fn):
        """One check interval for every batch; retire finished members."""
        for prec, b in self.batches.items():
            if len(b) == 0:
                continue
            if self.autotune and not getattr(b, "_tuned", False) and len(b) >= 4:
                b.tune(steps_per_candidate=8)
                self.launch = b.get_launch()
                b._tuned = True
            self.cell_updates += b.active_cells() * self.check_every
            b.check(self.check_every)
        self.ticks += 1
        t = now_fn()
        for rid in list(self.active):
            req, dom, nbytes, t_admit = self.active[rid]
            o = dom.last_observables()
            refining = rid in self.refined
            prec = "f32" if refining else req.precision
            done_before = self.refined.get(rid, 0)
            if refining:
                tol = self.refine_tol[req.precision]
            else:
                tol = self.tol if req.tol is None else req.tol
            cap = self.max_steps if req.max_steps is None else req.max_steps
            converged = 0.0 <= o["residual"] < tol
            unstable = bool(o["nan_flag"])
            steps = done_before + dom.step_count
            if converged and not refining and req.precision in self.refine_tol and steps < cap:
                # (without room in the FP32 batch or the budget it keeps going
                # in its own storage and tries again at the next check)
                if self._refine(rid, req, dom, nbytes, t_admit, steps):
                    continue
                converged = False
            if converged or unstable or steps >= cap:
                self.batches[prec].remove(dom)
                self.results.append(Result(req.id, req.precision, req.nx, req.ny, steps,
                                           converged, unstable, o, req.arrival_s, t_admit, t,
                                           refined_steps=dom.step_count if refining else 0))
                dom.close()
                del self.active[rid]
                self.refined.pop(rid, None)
                self.used -= nbytes

    def _refine(self, rid, req, dom, nbytes, t_admit, steps) -> bool:
        """Moves a request's state to an FP32 domain of the FP32 batch (device
        copies through FP64 tensors: populations read back and written again).
        False, and nothing done, while that batch or the budget has no room."""
        nb = domain_bytes(dataclasses.replace(req, precision="f32"))
        b32 = self.batches.get("f32")
        if (b32 is not None and len(b32) >= self.max_instances) or self.used + nb - nbytes > self.budget:
            return False
        with self.torch.cuda.stream(self.stream):
            f, g = dom.populations()
            nd = lbm.Domain(dict(nx=req.nx, ny=req.ny, angle_deg=req.angle_deg), precision="f32",
                            device=self.device, stream=self.stream)
            nd.set_launch(**self.launch)
            nd.set_params(req.params)
            nd.write_populations(f, g)
            del f, g
        self.batches[req.precision].remove(dom)
        dom.close()
        self.used += nb - nbytes
        self.peak_used = max(self.peak_used, self.used)
        self._batch("f32").add(nd)
        self.active[rid] = (req, nd, nb, t_admit)
        self.refined[rid] = steps
        return True

    def run(self, requests, realtime: bool = True) -> list:
        """Serve `requests`; arrival times are honoured against the wall clock
        when realtime is set (else every request is present at t = 0)."""
        pending = sorted(requests, key=lambda r: r.arrival_s)
        t0 = time.perf_counter()
        now = (lambda: time.perf_counter() - t0) if realtime else (lambda: time.perf_counter() - t0)
        arrivals = {r.id: (r.arrival_s if realtime else 0.0) for r in pending}
        for r in pending:
            r.arrival_s = arrivals[r.id]
        while pending or self.active:
            t = now()
            while pending and pending[0].arrival_s <= t and self.fits(pending[0]):
                self.admit(pending.pop(0), t)
            if not self.active:
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival_s - now(), 0.05)))
                continue
            self.tick(now)
        self.wall_s = now()
        return self.results

    def close(self):
        for _, dom, _, _ in self.active.values():
            dom.close()
        self.active.clear()
        for b in self.batches.values():
            b.close()
        self.batches.clear()


def solve_one_at_a_time(requests, tol: float = 1e-7, check_every: int = 100,
                        max_steps: int = 20000, launch: dict | None = None, device=None,
                        realtime: bool = True, precision: str = "f32") -> list:
    """Baseline: each request alone on a plain FP32 domain, in arrival order."""
    import torch
    dev = torch.device(device if device is not None else "cuda")
    stream = torch.cuda.Stream(device=dev)
    launch = launch or dict(tile_w=64, block_rows=1, rows_per_thread=4, blocks_per_sm=0)
    t0 = time.perf_counter()
    out = []
    for r in sorted(requests, key=lambda q: q.arrival_s):
        arrival = r.arrival_s if realtime else 0.0
        wait = arrival - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        t_start = time.perf_counter() - t0
        with torch.cuda.stream(stream):
            dom = lbm.Domain(dict(nx=r.nx, ny=r.ny, angle_deg=r.angle_deg), precision=precision,
                             device=dev, stream=stream)
            dom.set_launch(**launch)
            dom.set_params(r.params)
            try:
                st, steps = dom.run_to_steady(tol if r.tol is None else r.tol, check_every=check_every,
                                              max_steps=max_steps if r.max_steps is None else r.max_steps)
                unstable = False
            except lbm.LBMError as e:
                if e.status != lbm.EUNSTABLE:
                    raise
                st, steps, unstable = e.status, dom.step_count, True
            o = dom.observables()
            dom.close()
        out.append(Result(r.id, precision, r.nx, r.ny, steps, st == lbm.OK, unstable, o, arrival,
                          t_start, time.perf_counter() - t0))
    return out


def summary(results, wall_s: float) -> dict:
    lat = sorted(r.latency_s for r in results)
    def pct(q):
        if not lat:
            return None
        k = min(len(lat) - 1, max(0, int(round(q * (len(lat) - 1)))))
        return lat[k]
    return {"solves": len(results), "wall_s": wall_s,
            "solves_per_s": len(results) / wall_s if wall_s > 0 else None,
            "p50_s": pct(0.50), "p99_s": pct(0.99),
            "converged": sum(r.converged for r in results),
            "capped": sum((not r.converged) and (not r.unstable) for r in results),
            "unstable": sum(r.unstable for r in results),
            "mean_steps": statistics.mean(r.steps for r in results) if results else None}
