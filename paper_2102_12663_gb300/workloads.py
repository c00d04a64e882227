"""Seeded synthetic inputs: test-flow masks, parameter recipes and request
streams.

This module holds none of the method's arithmetic (no equilibria, moments,
collision or streaming).  It only builds inputs: cell-type masks of simple
test geometries, lattice parameter sets derived from dimensionless numbers,
and seeded parameter draws for batched and served workloads.  Both the CUDA
path and the FP64 oracle consume what it returns; neither is imported here.

Cell-type codes (an interface convention of the mask format):
0 fluid, 1 porous (trabecular meshwork), 2 cold wall (cornea), 3 hot wall
(iris/lens), 4 adiabatic wall, 5 inlet, 6 outlet.
"""
from __future__ import annotations

import math

import numpy as np

FLUID, POROUS, COLD, HOT, ADIABATIC, INLET, OUTLET = range(7)


def _desc(nx, ny, periodic_x=0, periodic_y=0, inlet_dir=(0, 1), inlet_profile=0,
          inlet_lo=0, inlet_width=1):
    return dict(nx=nx, ny=ny, periodic_x=periodic_x, periodic_y=periodic_y,
                inlet_dir=tuple(inlet_dir), inlet_profile=inlet_profile,
                inlet_lo=inlet_lo, inlet_width=inlet_width)


def channel(nx: int, H: int, porous: bool = False):
    """Plane channel, periodic in x; hot wall row y = 0, cold wall row
    y = H + 1, H fluid (or porous) rows between.  Walls sit halfway, at
    y = 1/2 and y = H + 1/2."""
    ny = H + 2
    m = np.full((ny, nx), POROUS if porous else FLUID, dtype=np.uint8)
    m[0, :] = HOT
    m[-1, :] = COLD
    return m, _desc(nx, ny, periodic_x=1)


def porous_box(nx: int, ny: int):
    """Porous cells everywhere, periodic in both directions."""
    m = np.full((ny, nx), POROUS, dtype=np.uint8)
    return m, _desc(nx, ny, periodic_x=1, periodic_y=1)


def darcy_column(n_in: int, n_por: int, n_out: int, ny: int):
    """Inlet column (plug inflow along +x) -> n_in fluid columns -> n_por
    porous columns -> n_out fluid columns -> outlet column; periodic in y."""
    nx = 1 + n_in + n_por + n_out + 1
    m = np.full((ny, nx), FLUID, dtype=np.uint8)
    m[:, 0] = INLET
    m[:, 1 + n_in:1 + n_in + n_por] = POROUS
    m[:, -1] = OUTLET
    return m, _desc(nx, ny, periodic_y=1, inlet_dir=(1, 0), inlet_profile=0)


def ra_to_gbeta(Ra: float, tau: float, tau_T: float, dT: float, L: float) -> float:
    """g*beta from the Rayleigh number Ra = g beta dT L^3 / (nu theta), with the
    lattice viscosity and diffusivity of the chosen relaxation times."""
    nu = (2.0 * tau - 1.0) / 6.0
    theta = (2.0 * tau_T - 1.0) / 4.0
    return Ra * nu * theta / (dT * L ** 3)


def tau_T_for_Pr(tau: float, Pr: float) -> float:
    """Thermal relaxation time that gives Prandtl number Pr = nu / theta."""
    nu = (2.0 * tau - 1.0) / 6.0
    return 0.5 * (4.0 * nu / Pr + 1.0)


UPRIGHT = (-1.0, 0.0)   # gravity across the chamber (standing patient)
SUPINE = (0.0, -1.0)    # gravity along the optical axis, cornea up


def eye_params(ny: int, tau: float, Ra: float, K_tm: float, Pr: float = 5.0,
               u_in_max: float = 0.005, g_dir=UPRIGHT, dT: float = 1.0,
               noise_amp: float = 1e-6, seed: int = 1234, porosity: float = 0.3):
    """Lattice parameters of the analytic eye: cornea T = 0, iris/lens and
    inflow T = dT, reference T0 = dT / 2, Ra on the domain height."""
    tau_T = tau_T_for_Pr(tau, Pr)
    gb = ra_to_gbeta(Ra, tau, tau_T, 1.0, float(ny)) if Ra > 0 else 0.0
    return dict(tau=tau, tau_T=tau_T, g_beta=gb, g_dir=tuple(g_dir),
                T_cold=0.0, T_hot=dT, T0=0.5 * dT, T_in=dT, u_in_max=u_in_max,
                K_tm=K_tm, porosity=porosity, p_out=0.0, drive=(0.0, 0.0),
                noise_amp=noise_amp, seed=seed,
                dx_m=12.8e-3 / 1921.0, dt_s=1e-4, rho0=990.0, p_sc_pa=1200.0)


def eye_geometry(nx: int, ny: int, angle_deg: float = 45.0):
    return dict(nx=nx, ny=ny, angle_deg=angle_deg)


# Plain FP64 model: 160x80 eye, 5,000 steps, tau 0.8, Pr 5, Ra 1e4, K 0.05.
CONFIG_FP64 = dict(nx=160, ny=80, steps=5000, tau=0.8, Ra=1e4, K_tm=0.05,
                   angle_deg=45.0, g_dir=UPRIGHT)
# FP32 throughput: 4096x2048 eye, 20,000 steps, tau 0.6, Ra 1e5, K 0.5.
CONFIG_FP32 = dict(nx=4096, ny=2048, steps=20000, tau=0.6, Ra=1e5, K_tm=0.5,
                   angle_deg=45.0, g_dir=UPRIGHT, check_nx=512, check_ny=256)
# Reduced storage: 8192x4096, error grid 1024x512.
CONFIG_PRECISION = dict(nx=8192, ny=4096, tau=0.6, Ra=1e5, K_tm=0.5, angle_deg=45.0,
                        g_dir=UPRIGHT, check_nx=1024, check_ny=512, tol=1e-7,
                        check_every=100)


def config_params(cfg: dict, nx: int | None = None, ny: int | None = None, **over):
    ny = ny or cfg["ny"]
    kw = dict(tau=cfg["tau"], Ra=cfg["Ra"], K_tm=cfg["K_tm"], g_dir=cfg["g_dir"])
    kw.update(over)
    return eye_params(ny, **kw)


def batch_instances(n: int = 64, seed: int = 2102, ny_lo: int = 128, ny_hi: int = 1024,
                    fp16_share: float = 0.0):
    """Seeded uneven eye instances: NY log-uniform in [ny_lo, ny_hi], NX = 2 NY
    (multiples of 8); inflow x U[0.5, 2] of 0.005; TM permeability
    log-uniform over [0.05, 5]; viscosity x U[0.7, 1.3] of 0.1; chamber angle
    U[20, 45] deg; gravity upright or supine with p = 1/2; temperature
    difference U[0, 3] with g*beta fixed by Ra = 1e4 per unit difference."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n):
        ny = int(round(math.exp(rng.uniform(math.log(ny_lo), math.log(ny_hi))) / 8.0)) * 8
        ny = max(ny, 64)
        nx = 2 * ny
        nu = 0.1 * rng.uniform(0.7, 1.3)
        tau = 3.0 * nu + 0.5
        u_in = 0.005 * rng.uniform(0.5, 2.0)
        K = math.exp(rng.uniform(math.log(0.05), math.log(5.0)))
        angle = rng.uniform(20.0, 45.0)
        g_dir = UPRIGHT if rng.uniform() < 0.5 else SUPINE
        dT = rng.uniform(0.0, 3.0)
        fp16 = bool(rng.uniform() < fp16_share)
        tau_T = tau_T_for_Pr(tau, 5.0)
        gb = ra_to_gbeta(1e4, tau, tau_T, 1.0, float(ny))
        p = dict(tau=tau, tau_T=tau_T, g_beta=gb, g_dir=g_dir, T_cold=0.0, T_hot=dT,
                 T0=0.5 * dT, T_in=dT, u_in_max=u_in, K_tm=K, porosity=0.3, p_out=0.0,
                 drive=(0.0, 0.0), noise_amp=1e-6, seed=1234 + k,
                 dx_m=12.8e-3 / 1921.0, dt_s=1e-4, rho0=990.0, p_sc_pa=1200.0)
        out.append(dict(id=k, nx=nx, ny=ny, angle_deg=angle, params=p, fp16=fp16))
    return out


def request_stream(n: int, rate_hz: float = 20.0, seed: int = 2102, ny_lo: int = 128,
                   ny_hi: int = 2048, fp16_share: float = 0.5):
    """Poisson arrivals (mean rate_hz) of steady-solve requests with sizes and
    parameters drawn as in batch_instances; returns a list sorted by arrival."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    inst = batch_instances(n, seed=seed, ny_lo=ny_lo, ny_hi=ny_hi, fp16_share=fp16_share)
    t = 0.0
    for r in inst:
        t += rng.exponential(1.0 / rate_hz)
        r["arrival_s"] = t
    return inst


# Steady-state tolerance of served solves per storage: max |du| over a
# 100-step check interval.  FP32 and FP64 reach the 1e-7 criterion; the 16-bit
# storages re-round every population each step, and their residual settles on
# a noise floor (about 3e-6 per 100 steps for FP16, 4e-5 for BF16 on the
# 256 x 128 eye), so they take the lowest tolerance above it.
SERVE_TOL = {"f64": 1e-7, "f32": 1e-7, "f16": 1e-5, "bf16": 1e-4}


def steady_step_cap(ny: int, nu: float, efolds: float = 20.0, check_every: int = 100) -> int:
    """Step cap of a steady solve: `efolds` decay times 1/(nu k^2) of the
    slowest viscous mode across the chamber (k = pi / ny), rounded up to whole
    check intervals."""
    steps = efolds * ny * ny / (math.pi ** 2 * nu)
    return int(math.ceil(steps / check_every) * check_every)
