"""Steady-state accuracy of the reduced-precision paths against the FP64 path
(which is bit-identical to the FP64 oracle; checked here on the same grid).

FP32: the 512 x 256 downscale of the FP32 throughput workload (tau 0.6, Ra 1e5
on the domain height, TM permeability 0.5 cells^2), run until FP64's residual
is far below the steady criterion; IOP, peak speed and both wall shear
stresses must agree to 1e-5 relative.  The bound holds because the FP32
collision takes the mean of its rounded non-equilibrium parts out (no
rounding bias of the conserved mass or heat): what is left of its rounding is
unbiased, and the steady state moves by the unbiased rounding of about
10^5 cells, about 1e-7 of it per step relative to the inflow.
"""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2102_12663_gb300 import lbm
from paper_2102_12663_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("iop", "peak_speed", "wss_cornea", "wss_iris")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm.load(build_if_missing=True)


def _eye(nx, ny, prec, **over):
    cfg = W.CONFIG_FP32
    pp = W.config_params(cfg, ny=ny, **over)
    dom = lbm.Domain(dict(nx=nx, ny=ny, angle_deg=cfg["angle_deg"]), precision=prec)
    dom.set_launch(tile_w=64, block_rows=4, rows_per_thread=1)
    dom.set_params(pp)
    return dom, pp


def _final(dom):
    """Observables after one more check interval (residual over its 100 steps)."""
    dom.run_to_steady(0.0, check_every=100, max_steps=100)
    dom.step(99)
    return dom.observables()


def test_fp64_path_matches_oracle_on_the_512x256_eye():
    nx, ny = 512, 256
    dom, pp = _eye(nx, ny, "f64")
    m, g = O.eye_mask(nx, ny, W.CONFIG_FP32["angle_deg"])
    O.set_threads(os.cpu_count() or 1)
    ref = O.State(g, O.make_params(**pp), m)
    dom.step(400)
    ref.run(400)
    f, gg = dom.populations()
    torch.cuda.synchronize()
    f = f.cpu().numpy().reshape(9, -1)
    gg = gg.cpu().numpy().reshape(4, -1)
    assert np.abs(f - ref.f).max() <= 1e-12 * np.abs(ref.f).max()
    assert np.abs(gg - ref.T).max() <= 1e-12 * np.abs(ref.T).max()


def test_fp32_steady_observables_within_1e5_of_fp64():
    nx, ny, steps = 512, 256, 1_200_000
    out = {}
    for prec in ("f64", "f32"):
        dom, _ = _eye(nx, ny, prec)
        dom.step(steps - 100)
        out[prec] = _final(dom)
        dom.close()
    ref, got = out["f64"], out["f32"]
    assert 0.0 <= ref["residual"] < 1e-9  # FP64 is steady
    for k in KEYS:
        assert abs(got[k] - ref[k]) <= 1e-5 * abs(ref[k]), (k, got[k], ref[k])
    # the fluxes balance to the same order at steady state
    assert abs(got["q_out"] - got["q_in"]) <= 1e-5 * got["q_in"]
