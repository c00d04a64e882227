"""Trends of the paper's parameter studies (Sec. 3.2-3.6), reproduced as
batched steady sweeps on the analytic eye.  The geometry is not the paper's
(its Fig. 1 is not in the text), so the tests check the shape of each result,
not its value:
  Tab. 4  IOP - p_SC grows linearly with the secretion rate;
  Tab. 5  (IOP - p_SC) K stays nearly constant when the meshwork dominates;
  Tab. 6  IOP rises with the viscosity;
  Tab. 7  IOP rises as the chamber angle narrows;
  Tab. 8  wall shear grows with the temperature difference, and a standing eye
          has higher cornea wall shear than an up-facing one;
  Tab. 3  the vortex intensity (Eq. 18) grows with the temperature difference,
          and an up-facing eye carries two mirror-image vortices."""
import numpy as np
import pytest

from paper_2102_12663_gb300 import lbm, sweeps
from paper_2102_12663_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GEO = dict(nx=160, ny=80, angle_deg=45.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm.load(build_if_missing=True)


def base(**over):
    p = W.eye_params(80, tau=0.8, Ra=0.0, K_tm=0.05, noise_amp=0.0)
    p.update(g_beta=0.0, T_hot=0.0, T_in=0.0, T0=0.0, tm_model=1, h_tm=6.0)
    p.update(over)
    return p


def dp(results):
    return np.array([r["iop"] for r in results])  # p_out = 0


def test_iop_linear_in_secretion_rate():
    scale = [0.5, 1.0, 1.5, 2.0]
    res = sweeps.steady_sweep(GEO, base(), [dict(u_in_max=0.005 * s) for s in scale])
    assert all(r["converged"] for r in res)
    ratio = dp(res) / np.array(scale)
    assert np.ptp(ratio) <= 1e-3 * ratio.mean()


def test_iop_times_permeability_nearly_constant():
    Ks = [0.01, 0.02, 0.05]
    res = sweeps.steady_sweep(GEO, base(h_tm=20.0), [dict(K_tm=k) for k in Ks])
    assert all(r["converged"] for r in res)
    prod = dp(res) * np.array(Ks)
    assert np.ptp(prod) <= 0.05 * prod.mean()
    assert np.all(np.diff(dp(res)) < 0)  # IOP falls as the meshwork opens


def test_iop_rises_with_viscosity_and_narrowing_angle():
    taus = [0.7, 0.8, 0.9]
    res = sweeps.steady_sweep(GEO, base(), [dict(tau=t, tau_T=W.tau_T_for_Pr(t, 5.0)) for t in taus])
    assert all(r["converged"] for r in res)
    assert np.all(np.diff(dp(res)) > 0)
    angles = [45.0, 35.0, 25.0]
    res = sweeps.steady_sweep(GEO, base(), [dict(geometry=dict(angle_deg=a)) for a in angles])
    assert all(r["converged"] for r in res)
    assert np.all(np.diff(dp(res)) > 0)


def test_wall_shear_grows_with_temperature_difference_and_orientation():
    gb = W.ra_to_gbeta(1e3, 0.8, W.tau_T_for_Pr(0.8, 5.0), 1.0, 80.0)
    dts = [0.5, 1.0, 2.0]
    variants = [dict(g_beta=gb, g_dir=W.UPRIGHT, T_hot=dt, T_in=dt, T0=0.5 * dt) for dt in dts]
    variants.append(dict(g_beta=gb, g_dir=W.SUPINE, T_hot=2.0, T_in=2.0, T0=1.0))
    res = sweeps.steady_sweep(GEO, base(), variants, tol=1e-9, vortex=True)
    assert all(r["converged"] for r in res)
    wc = np.array([r["wss_cornea"] for r in res[:3]])
    wi = np.array([r["wss_iris"] for r in res[:3]])
    assert np.all(np.diff(wc) > 0) and np.all(np.diff(wi) > 0)
    assert res[2]["wss_cornea"] > res[3]["wss_cornea"]  # standing above up-facing
    # Tab. 3: intensity grows with the temperature difference
    vi = np.array([r["vortex"]["intensity_abs"] for r in res[:3]])
    assert np.all(np.diff(vi) > 0)
    # up-facing (Sec. 3.4): two vortices, mirror images about the mid-plane
    v = res[3]["vortex"]
    assert v["max_x"] + v["min_x"] == GEO["nx"] - 1 and v["max_y"] == v["min_y"]
    assert v["psi_max"] > 0 > v["psi_min"]
    assert v["psi_max"] == pytest.approx(-v["psi_min"], rel=1e-6)
