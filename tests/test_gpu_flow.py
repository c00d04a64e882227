"""Dataflow stepping (one cooperative launch for many steps, tiles released
by their 3 x 3 tile neighbourhood) against one launch per step.

The two schedules run the same per-cell arithmetic on the same slots, so the
populations must be bit-identical for every storage, launch shape and step
split, including domains far smaller than the grid (where most blocks wait
several steps ahead of the tiles they depend on) and periodic domains (where
the neighbourhood wraps around).  FP64 dataflow stepping is also checked
against the oracle directly.
"""
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


def pops(dom):
    f, g = dom.populations()
    torch.cuda.synchronize()
    return f.cpu().numpy(), g.cpu().numpy()


def eye_domain(nx, ny, prec, launch, stepping, sweep=(1, 0)):
    pp = W.eye_params(ny, tau=0.8, Ra=1e4, K_tm=0.05)
    dom = lbm.Domain(dict(nx=nx, ny=ny, angle_deg=40.0), precision=prec)
    dom.set_launch(**launch, stepping=stepping, sweep_steps=sweep[0], sweep_lag=sweep[1])
    dom.set_params(pp)
    return dom


def mask_domain(mask, desc, params, prec, launch, stepping, sweep=(1, 0)):
    geo = dict(mask=mask, **{k: v for k, v in desc.items() if k not in ("nx", "ny")})
    dom = lbm.Domain(geo, precision=prec)
    dom.set_launch(**launch, stepping=stepping, sweep_steps=sweep[0], sweep_lag=sweep[1])
    dom.set_params(params)
    return dom


SHAPES = [
    dict(tile_w=64, block_rows=4, rows_per_thread=1, blocks_per_sm=0),
    dict(tile_w=32, block_rows=1, rows_per_thread=4, blocks_per_sm=0),
    dict(tile_w=128, block_rows=2, rows_per_thread=2, blocks_per_sm=1),
    dict(tile_w=256, block_rows=1, rows_per_thread=1, blocks_per_sm=2),
]
SPLITS = [(2,), (37,), (5, 32, 1, 9)]
# (steps per wavefront sweep, tile rows of lag): step by step, the tightest
# lag, and deep sweeps
SWEEPS = [(1, 0), (2, 2), (4, 3), (8, 0)]


def run(dom, split):
    for n in split:
        dom.step(n)


def direct_twin(prec, launch):
    """Per-launch shape that runs the same per-cell code as the dataflow
    kernel with `launch`.  The dataflow kernel always takes the direct path;
    one launch per step of a one-row FP32-arithmetic shape takes the staged
    kernel instead, whose interior collision rounds differently.  The direct
    path's results depend only on whether warps hold whole 64-cell row
    segments (pair path) or not (tile_w 32), not on the rest of the shape."""
    if prec == "f64" or launch["block_rows"] > 1:
        return launch
    return dict(tile_w=64 if launch["tile_w"] >= 64 else 32, block_rows=4, rows_per_thread=1,
                blocks_per_sm=0)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_flow_matches_per_launch_eye(prec, shape):
    launch = SHAPES[shape]
    for split in SPLITS:
        a = eye_domain(200, 100, prec, launch, lbm.STEP_FLOW)
        b = eye_domain(200, 100, prec, direct_twin(prec, launch), lbm.STEP_PER_LAUNCH)
        run(a, split)
        run(b, split)
        assert a.step_count == b.step_count == sum(split)
        fa, ga = pops(a)
        fb, gb = pops(b)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), (prec, launch, split)
        a.close()
        b.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("sweep", SWEEPS[1:])
def test_flow_sweeps_match_per_launch_eye(prec, sweep):
    """Wavefront sweeps of several steps (the issue order is all that
    changes) against one launch per step, over step counts that end inside a
    sweep."""
    launch = dict(tile_w=64, block_rows=2, rows_per_thread=2, blocks_per_sm=0)
    for split in SPLITS + [(sweep[0] * 3 + 1,)]:
        a = eye_domain(256, 128, prec, launch, lbm.STEP_FLOW, sweep)
        b = eye_domain(256, 128, prec, launch, lbm.STEP_PER_LAUNCH)
        run(a, split)
        run(b, split)
        fa, ga = pops(a)
        fb, gb = pops(b)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), (prec, sweep, split)
        a.close()
        b.close()


PERIODIC = {
    "channel": (W.channel(96, 20), dict(tau=0.8, tau_T=0.7, drive=(1e-5, 0.0), T_hot=1.0,
                                        T_cold=0.0, T0=0.5, g_beta=1e-4, g_dir=(0.0, -1.0),
                                        noise_amp=1e-3, seed=5)),
    "porous_box": (W.porous_box(80, 8), dict(tau=0.7, drive=(1e-5, -3e-6), K_tm=0.2,
                                              noise_amp=1e-3, T0=0.3, g_beta=1e-4,
                                              g_dir=(0.6, -0.8), seed=9)),
}


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", sorted(PERIODIC))
@pytest.mark.parametrize("sweep", [(1, 0), (4, 2)])
def test_flow_matches_per_launch_periodic(prec, case, sweep):
    """Wrap-around neighbourhoods: in x (channel, which also sweeps) and in
    both directions (porous box, whose 3 x 1 tile grid makes a tile its own
    neighbour; periodic in y, so it steps one sweep step at a time)."""
    (mask, desc), params = PERIODIC[case]
    launch = dict(tile_w=32, block_rows=2, rows_per_thread=4, blocks_per_sm=0)
    a = mask_domain(mask, desc, params, prec, launch, lbm.STEP_FLOW, sweep)
    b = mask_domain(mask, desc, params, prec, launch, lbm.STEP_PER_LAUNCH)
    a.step(401)
    b.step(401)
    fa, ga = pops(a)
    fb, gb = pops(b)
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_flow_tiny_domain_long_run():
    """A 64 x 32 eye has a handful of tiles and the grid has hundreds of
    blocks, so nearly every block waits for earlier steps: 3,001 steps in
    one launch (sweeps of 8 steps, 2 tile rows apart) against 3,001 single
    launches."""
    launch = dict(tile_w=32, block_rows=2, rows_per_thread=2, blocks_per_sm=0)
    a = eye_domain(64, 32, "f32", launch, lbm.STEP_FLOW, (8, 2))
    b = eye_domain(64, 32, "f32", launch, lbm.STEP_PER_LAUNCH)
    a.step(3001)
    b.step(3001)
    fa, ga = pops(a)
    fb, gb = pops(b)
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    # the steady check reads the dataflow status word: no wait expired
    status, _ = a.run_to_steady(0.0, check_every=10, max_steps=10)
    assert status == lbm.ENOTCONVERGED


def test_flow_fp64_matches_oracle():
    nx, ny = 192, 96
    pp = W.eye_params(ny, tau=0.8, Ra=1e4, K_tm=0.05)
    dom = lbm.Domain(dict(nx=nx, ny=ny, angle_deg=45.0), precision="f64")
    dom.set_launch(tile_w=64, block_rows=4, rows_per_thread=1, blocks_per_sm=0,
                   stepping=lbm.STEP_FLOW)
    dom.set_params(pp)
    m, g = O.eye_mask(nx, ny, 45.0)
    ref = O.State(g, O.make_params(**pp), m)
    dom.step(333)
    ref.run(333)
    f, t = pops(dom)
    assert np.array_equal(f.reshape(9, -1), ref.f) and np.array_equal(t.reshape(4, -1), ref.T)


def test_expired_wait_is_reported_and_the_context_survives():
    """The failure path of the bounded waits, made on the host: a tile that
    never reports progress makes its neighbours' waits run out; the launch
    aborts and completes, the next observable read reports the invalid
    results, and the domain steps correctly again once the hook is off."""
    launch = dict(tile_w=64, block_rows=4, rows_per_thread=1, blocks_per_sm=0)
    dom = eye_domain(192, 96, "f32", launch, lbm.STEP_FLOW)
    dom.debug_stall_tile(dom.tile_count() // 2)
    dom.step(3)
    with pytest.raises(lbm.LBMError) as e:
        dom.observables()
    assert e.value.status == lbm.ECUDA and "too long" in str(e.value)
    dom.debug_stall_tile(-1)
    dom.reset()
    ref = eye_domain(192, 96, "f32", launch, lbm.STEP_PER_LAUNCH)
    dom.step(20)
    ref.step(20)
    fa, ga = pops(dom)
    fb, gb = pops(ref)
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert dom.observables()["nan_flag"] == 0


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_large_domain_launch_order(prec):
    """A domain of more than 4096 tiles, whose per-step launches run the
    tiles that hold boundary cells first, against the dataflow kernel (which
    follows its own wavefront order), bit for bit, with the observables of the
    check step agreeing as well."""
    launch = dict(tile_w=32, block_rows=4, rows_per_thread=1, blocks_per_sm=0)
    a = eye_domain(2304, 1152, prec, launch, lbm.STEP_PER_LAUNCH)
    b = eye_domain(2304, 1152, prec, launch, lbm.STEP_FLOW)
    assert a.tile_count() > 4096
    for n in (1, 36):
        a.step(n)
        b.step(n)
    fa, ga = pops(a)
    fb, gb = pops(b)
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    oa, ob = a.observables(), b.observables()
    for k in ("iop", "mass", "peak_speed", "wss_cornea", "wss_iris", "q_in", "q_out"):
        assert oa[k] == ob[k], k
    a.close()
    b.close()
