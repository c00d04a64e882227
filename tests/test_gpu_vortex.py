"""Vortex intensity and centres (Eq. 18, Tab. 3) through the C ABI against
the FP64 oracle on the same velocity fields: analytic fields on periodic and
walled grids, and the velocity of a stepped eye.  The per-cell vorticity is
evaluated without contraction on both sides, so only the summation order of
the intensities differs (1e-12 relative); the stream function is the same
running sum on both sides, so its extrema and their cells must match
exactly."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2102_12663_gb300 import lbm
from paper_2102_12663_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm.load(build_if_missing=True)


def mask_domain(mask, desc):
    geo = dict(mask=mask, **{k: v for k, v in desc.items() if k not in ("nx", "ny")})
    return lbm.Domain(geo, precision="f64")


def compare(dom, geom, mask, u_np):
    u = torch.tensor(u_np, dtype=torch.float64, device="cuda").contiguous()
    got = dom.vortex(u)
    ref = O.vortex(geom, mask, u_np)
    scale = max(ref["intensity_abs"], 1e-300)
    assert got["n_fluid"] == ref["n_fluid"]
    assert abs(got["intensity"] - ref["intensity"]) <= 1e-12 * scale
    assert got["intensity_abs"] == pytest.approx(ref["intensity_abs"], rel=1e-12)
    for k in ("psi_max", "psi_min", "max_x", "max_y", "min_x", "min_y"):
        assert got[k] == ref[k], k
    return got, ref


def test_taylor_green_periodic_box():
    n = 160  # more than one 128-column block
    k = 2 * math.pi / 32
    X, Y = np.meshgrid(np.arange(n), np.arange(64))
    u = np.stack([1e-3 * np.sin(k * X) * np.cos(k * Y), -1e-3 * np.cos(k * X) * np.sin(k * Y)])
    m, d = W.porous_box(n, 64)
    m[:] = W.FLUID
    g = O.mask_geom(n, 64, 1, 1)
    got, _ = compare(mask_domain(m, d), g, m, u)
    assert abs(got["intensity"]) <= 1e-12 * got["intensity_abs"]


@pytest.mark.parametrize("nx, ny", [(300, 150), (160, 80)])
def test_random_field_on_eye_mask(nx, ny):
    """A seeded random field on the eye's mask (ragged column blocks): every
    wall, inlet, outlet and porous neighbour case of the stencil."""
    rng = np.random.default_rng(2102)
    u = rng.standard_normal((2, ny, nx)) * 1e-3
    m, g = O.eye_mask(nx, ny, 40.0)
    dom = lbm.Domain(dict(nx=nx, ny=ny, angle_deg=40.0), precision="f64")
    compare(dom, g, m, u)


def test_stepped_eye_velocity():
    nx, ny = 160, 80
    pp = W.eye_params(ny, tau=0.8, Ra=1e4, K_tm=0.05)
    dom = lbm.Domain(dict(nx=nx, ny=ny, angle_deg=45.0), precision="f64")
    dom.set_params(pp)
    dom.step(1500)
    u = dom.fields()[0]
    torch.cuda.synchronize()
    m, g = O.eye_mask(nx, ny, 45.0)
    got, ref = compare(dom, g, m, u.cpu().numpy())
    assert got["intensity_abs"] > 0.0
    assert got["intensity_abs_phys"] == pytest.approx(
        got["intensity_abs"] * pp["dx_m"] ** 2 / pp["dt_s"], rel=1e-12)
    assert got["max_mm"][0] == pytest.approx((got["max_x"] + 0.5) * pp["dx_m"] * 1e3, rel=1e-12)


def test_small_grid_and_one_row_rejection():
    """An 8 x 4 channel still fits the reduction scratch; a one-row grid (the
    only shape whose domain buffer cannot hold it) is rejected."""
    m, d = W.channel(8, 2)
    rng = np.random.default_rng(7)
    compare(mask_domain(m, d), O.mask_geom(8, 4, 1, 0), m, rng.standard_normal((2, 4, 8)))
    m, d = W.porous_box(8, 1)
    dom = mask_domain(m, d)
    u = torch.zeros((2, 1, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError):
        dom.vortex(u)
