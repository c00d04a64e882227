"""Bouzidi's interpolated bounce-back on the curved cornea (the no-slip
scheme the paper names, Sec. 2.3 ref. 36) through the C ABI against the FP64
oracle with the same rule.  The library completes the q < 1/2 links when a
cell next reads its populations, so the checks cover every reader: the step
kernels (per-step, dataflow, staged, batched), the observables, the field and
population read-back, and the population write-back."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2102_12663_gb300 import lbm
from paper_2102_12663_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NX, NY, ANGLE = 160, 80, 45.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm.load(build_if_missing=True)


def params(**over):
    p = W.eye_params(NY, tau=0.8, Ra=1e4, K_tm=0.05)
    p.update(bouzidi=1)
    p.update(over)
    return p


def pair(prec, launch=None, **over):
    pp = params(**over)
    dom = lbm.Domain(dict(nx=NX, ny=NY, angle_deg=ANGLE), precision=prec)
    if launch:
        dom.set_launch(**launch)
    dom.set_params(pp)
    m, g = O.eye_mask(NX, NY, ANGLE)
    return dom, O.State(g, O.make_params(**pp), m)


def pops(dom):
    f, g = dom.populations()
    torch.cuda.synchronize()
    return f.cpu().numpy().reshape(9, -1), g.cpu().numpy().reshape(4, -1)


def rel(dom, ref):
    f, g = pops(dom)
    return max(np.abs(f - ref.f).max() / np.abs(ref.f).max(),
               np.abs(g - ref.T).max() / np.abs(ref.T).max())


def test_link_fractions_match_the_oracle_geometry():
    """The library's arc is the oracle's: same centre and radius."""
    m, g = O.eye_mask(NX, NY, ANGLE)
    info = lbm.Domain(dict(nx=NX, ny=NY, angle_deg=ANGLE), precision="f64").info()
    assert (info["arc_xc"], info["arc_yc"], info["arc_r"]) == (g.arc_xc, g.arc_yc, g.arc_r)


@pytest.mark.parametrize("stepping", [lbm.STEP_PER_LAUNCH, lbm.STEP_FLOW])
def test_fp64_parity_and_effect(stepping):
    launch = dict(tile_w=64, block_rows=4, rows_per_thread=2, blocks_per_sm=0, stepping=stepping)
    dom, ref = pair("f64", launch)
    dom.step(700)
    ref.run(700)
    assert rel(dom, ref) <= 1e-12
    # the rule changes the flow (against halfway bounce-back)
    off = lbm.Domain(dict(nx=NX, ny=NY, angle_deg=ANGLE), precision="f64")
    off.set_params(params(bouzidi=0))
    off.step(700)
    assert np.abs(pops(off)[0] - ref.f).max() > 1e-6 * np.abs(ref.f).max()


def test_fields_and_observables_read_the_completed_links():
    dom, ref = pair("f64")
    dom.step(401)  # odd parity
    ref.run(401)
    u, p, T = dom.fields()
    uo, po, To = ref.fields()
    assert np.abs(u.cpu().numpy().reshape(2, -1) - uo).max() <= 1e-12 * np.abs(uo).max()
    assert np.abs(p.cpu().numpy().reshape(-1) - po).max() <= 1e-12 * np.abs(po).max()
    o, oo = dom.observables(), ref.observe()
    for k, kr in [("iop", "iop"), ("mass", "mass"), ("peak_speed", "peak"),
                  ("wss_cornea", "wss_cornea"), ("wss_iris", "wss_iris")]:
        assert o[k] == pytest.approx(oo[kr], rel=1e-12), k


def test_population_write_back_round_trip():
    """Writing the oracle's state and reading it back gives it again; then
    both sides step on from it."""
    dom, ref = pair("f64")
    ref.run(233)
    dom.write_populations(ref.f.reshape(9, NY, NX), ref.T.reshape(4, NY, NX))
    f, g = pops(dom)
    assert np.abs(f - ref.f).max() <= 1e-15 * np.abs(ref.f).max()
    dom.step(64)
    ref.run(64)
    assert rel(dom, ref) <= 1e-12


@pytest.mark.parametrize("launch", [
    dict(tile_w=64, block_rows=4, rows_per_thread=1, blocks_per_sm=0),
    dict(tile_w=128, block_rows=1, rows_per_thread=4, blocks_per_sm=0),  # staged kernel
])
def test_fp32_parity(launch):
    dom, ref = pair("f32", launch)
    dom.step(300)
    ref.run(300)
    assert rel(dom, ref) <= 1.5e-5


def test_batched_member():
    dom, ref = pair("f64")
    other = lbm.Domain(dict(nx=96, ny=48, angle_deg=40.0), precision="f64")
    other.set_params(W.eye_params(48, tau=0.7, Ra=1e4, K_tm=0.5))
    b = lbm.Batch("f64", max_instances=2, max_tiles=1 << 14,
                  launch=dict(tile_w=64, block_rows=2, rows_per_thread=2, blocks_per_sm=0))
    b.add(dom)
    b.add(other)
    b.step(120)
    b.check(30)
    ref.run(150)
    assert rel(dom, ref) <= 1e-12
    b.close()
