"""TM-thickness calibration (Sec. 3.1): a chain of steady solves of the lumped
meshwork model converges on the thickness that gives the target IOP."""
import pytest

from paper_2102_12663_gb300 import calibrate, lbm
from paper_2102_12663_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_calibration_hits_target_iop():
    lbm.load(build_if_missing=True)
    geo = dict(nx=96, ny=48, angle_deg=45.0)
    pp = W.eye_params(48, tau=0.8, Ra=0.0, K_tm=0.05, noise_amp=0.0)
    pp.update(g_beta=0.0, dx_m=1.0, dt_s=1.0, rho0=1.0, p_sc_pa=0.0)
    # IOP in these units is the lattice pressure above p_out
    probe = calibrate.calibrate_tm_thickness(geo, pp, target_iop_pa=0.0, h0=2.0, h1=2.0,
                                             precision="f64", max_iters=0, steady_tol=1e-10)
    iop_at_2 = probe["history"][0][1]
    target = 2.5 * iop_at_2
    res = calibrate.calibrate_tm_thickness(geo, pp, target_iop_pa=target, h0=2.0, h1=4.0,
                                           precision="f64", tol_pa=1e-4 * target,
                                           steady_tol=1e-10)
    assert abs(res["iop_pa"] - target) <= 1e-4 * target
    assert res["iterations"] <= 8
    assert res["h_tm"] > 2.0
