"""Calibration of the effective trabecular-meshwork thickness.

The paper (Sec. 3.1) keeps every geometric and physical parameter at its
normal value except the TM thickness of the lumped meshwork model (Sec. 2.3),
which it adjusts until the steady IOP is the normal 1950 Pa.  This module does
that adjustment as a chain of steady solves on one resident domain: each solve
starts from the previous steady state, and a secant step on h_tm moves the
steady IOP towards the target (IOP - p_SC is close to linear in h_tm, exactly
so where the meshwork dominates the resistance).  Every solve runs in the
CUDA library through lbm_run_to_steady.
"""
from __future__ import annotations

from . import lbm

# Porosity labels of the meshwork permeability.  Tab. 5 pairs each
# permeability K of the TM with a porosity e; the pairs follow the
# Kozeny-Carman form K = C e^3 / (1 - e)^2 with one constant, C = 4.27e-13 m^2
# (every row within 0.5 %).  The model's Darcy law (Eq. 4) has no porosity:
# these functions only translate between the two labels.
KOZENY_CARMAN_C = 4.27e-13  # m^2


def permeability_from_porosity(eps: float, c: float = KOZENY_CARMAN_C) -> float:
    """K(e) = c e^3 / (1 - e)^2 in m^2, for 0 <= e < 1."""
    if not 0.0 <= eps < 1.0:
        raise ValueError("porosity must lie in [0, 1)")
    return c * eps ** 3 / (1.0 - eps) ** 2


def porosity_from_permeability(k: float, c: float = KOZENY_CARMAN_C) -> float:
    """The porosity e in [0, 1) with K(e) = k (K is increasing in e), by
    bisection to double precision."""
    if not k >= 0.0:
        raise ValueError("permeability must be non-negative")
    lo, hi = 0.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if c * mid ** 3 / (1.0 - mid) ** 2 < k:
            lo = mid
        else:
            hi = mid
    return lo


def calibrate_tm_thickness(geometry: dict, params: dict, target_iop_pa: float, h0: float,
                           h1: float, precision: str = "f32", tol_pa: float = 0.5,
                           steady_tol: float = 1e-7, check_every: int = 100,
                           max_steps: int = 500000, max_iters: int = 12, device=None,
                           launch: dict | None = None) -> dict:
    """Secant iteration on h_tm until |IOP_pa - target| <= tol_pa at steady state.

    Returns {"h_tm", "iop_pa", "iterations", "history": [(h, iop_pa, steps)]}.
    Raises lbm.LBMError if a solve turns unstable."""
    dom = lbm.Domain(geometry, precision=precision, device=device)
    if launch:
        dom.set_launch(**launch)
    p = dict(params, tm_model=1, h_tm=float(h0))
    dom.set_params(p)
    history = []

    def solve(h: float) -> float:
        p["h_tm"] = float(h)
        dom.set_params(p)  # keeps the state: the solve starts from the last steady state
        _, steps = dom.run_to_steady(steady_tol, check_every=check_every, max_steps=max_steps)
        iop = dom.observables()["iop_pa"]
        history.append((float(h), iop, steps))
        return iop - target_iop_pa

    try:
        ha, fa = float(h0), solve(h0)
        hb, fb = float(h1), solve(h1)
        for it in range(max_iters):
            if abs(fb) <= tol_pa:
                break
            if fb == fa:
                break
            hn = hb - fb * (hb - ha) / (fb - fa)
            if not hn > 0.0:
                hn = 0.5 * hb
            ha, fa = hb, fb
            hb, fb = hn, solve(hn)
        return {"h_tm": hb, "iop_pa": fb + target_iop_pa, "iterations": len(history),
                "history": history}
    finally:
        dom.close()
