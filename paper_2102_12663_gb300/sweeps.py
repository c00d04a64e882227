"""Steady-state parameter sweeps as batched workloads.

The paper's Sec. 3.2-3.6 vary one parameter at a time around a base eye and
report steady observables: IOP against the secretion rate (Tab. 4), the TM
permeability (Tab. 5), the viscosity (Tab. 6) and the chamber angle (Tab. 7),
and the cornea / iris wall shear stress against the temperature difference
and the eye orientation (Tab. 8).  Here every variant of a sweep is one member
of a single batch (one fused launch per time step for all of them), and each
member leaves the batch once it is steady.  Only the orchestration lives
here; every step runs in the CUDA library.
"""
from __future__ import annotations

from . import lbm


def steady_sweep(geometry: dict, params: dict, variants: list, precision: str = "f64",
                 tol: float = 1e-10, check_every: int = 100, max_steps: int = 2_000_000,
                 launch: dict | None = None, device=None, vortex: bool = False) -> list:
    """Steady observables for each variant.

    geometry, params: the base eye (lbm.Domain geometry dict, lbm_params dict).
    variants: list of dicts; key "geometry" overrides geometry entries, every
    other key overrides a parameter.  Returns, per variant, the observables of
    its last check plus "steps" and "converged", and with vortex=True the
    vortex measures of its final state (Eq. 18, Tab. 3) under "vortex"."""
    import torch
    dev = torch.device(device if device is not None else "cuda")
    stream = torch.cuda.Stream(device=dev)
    launch = launch or dict(tile_w=128, block_rows=2, rows_per_thread=2, blocks_per_sm=0)
    doms, out = [], [None] * len(variants)
    with torch.cuda.stream(stream):
        batch = lbm.Batch(precision, max_instances=len(variants), max_tiles=1 << 20,
                          launch=launch, device=dev, stream=stream)
        try:
            for v in variants:
                geo = dict(geometry, **v.get("geometry", {}))
                p = dict(params, **{k: val for k, val in v.items() if k != "geometry"})
                d = lbm.Domain(geo, precision=precision, device=dev, stream=stream)
                d.set_launch(**launch)
                d.set_params(p)
                batch.add(d)
                doms.append(d)
            active = dict(enumerate(doms))
            while active:
                batch.check(check_every)
                for k in list(active):
                    d = active[k]
                    o = d.last_observables()
                    converged = 0.0 <= o["residual"] < tol
                    if converged or o["nan_flag"] or d.step_count >= max_steps:
                        out[k] = dict(o, steps=d.step_count, converged=converged)
                        if vortex:
                            out[k]["vortex"] = d.vortex()
                        batch.remove(d)
                        del active[k]
        finally:
            batch.close()
            for d in doms:
                d.close()
    return out
