"""Batched stepping: many uneven eye instances advanced by one launch per
step over a merged tile list.  A member's results must not depend on the
batch it runs in (bitwise), must match the FP64 oracle, and the autotuner's
pick must not change them."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2102_12663_gb300 import lbm
from paper_2102_12663_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPE = dict(tile_w=64, block_rows=1, rows_per_thread=4, blocks_per_sm=0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm.load(build_if_missing=True)


def make(inst, prec):
    dom = lbm.Domain(dict(nx=inst["nx"], ny=inst["ny"], angle_deg=inst["angle_deg"]), precision=prec)
    dom.set_launch(**SHAPE)
    dom.set_params(inst["params"])
    return dom


def small_instances(n, seed=7):
    return W.batch_instances(n, seed=seed, ny_lo=48, ny_hi=112)


def pops(dom):
    f, g = dom.populations()
    torch.cuda.synchronize()
    return f.cpu().numpy().reshape(9, -1), g.cpu().numpy().reshape(4, -1)


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_alone_equals_in_mix_bitwise(prec):
    inst = small_instances(5)
    alone = make(inst[0], prec)
    b1 = lbm.Batch(prec, max_instances=1, max_tiles=1 << 14, launch=SHAPE)
    b1.add(alone)
    mixed = [make(i, prec) for i in inst]
    b5 = lbm.Batch(prec, max_instances=8, max_tiles=1 << 16, launch=SHAPE)
    for d in mixed:
        b5.add(d)
    for _ in range(3):
        b1.check(100)
        b5.check(100)
    fa, ga = pops(alone)
    fm, gm = pops(mixed[0])
    assert np.array_equal(fa, fm) and np.array_equal(ga, gm)
    oa, om = alone.last_observables(), mixed[0].last_observables()
    assert oa == om
    assert oa["step"] == 299 and oa["residual"] >= 0.0
    b1.close()
    b5.close()


def test_batch_matches_oracle_with_mixed_parity():
    """Members of different sizes, parameters and step parities (one was
    stepped alone an odd number of times before joining) against the oracle."""
    inst = small_instances(3, seed=11)
    doms = [make(i, "f64") for i in inst]
    refs = []
    for i in inst:
        m, g = O.eye_mask(i["nx"], i["ny"], i["angle_deg"])
        refs.append(O.State(g, O.make_params(**i["params"]), m))
    doms[1].step(3)
    refs[1].run(3)
    b = lbm.Batch("f64", max_instances=4, max_tiles=1 << 16, launch=SHAPE)
    for d in doms:
        b.add(d)
    b.step(45)
    b.check(20)
    for d, r in zip(doms, refs):
        r.run(65)
        assert d.step_count == r.step_count
        f, g = pops(d)
        assert np.abs(f - r.f).max() <= 1e-12 * np.abs(r.f).max()
        assert np.abs(g - r.T).max() <= 1e-12 * np.abs(r.T).max()
    # the observables of the check step (step 64 for the even members)
    o = doms[0].last_observables()
    r0 = O.State(O.eye_mask(inst[0]["nx"], inst[0]["ny"], inst[0]["angle_deg"])[1],
                 O.make_params(**inst[0]["params"]),
                 O.eye_mask(inst[0]["nx"], inst[0]["ny"], inst[0]["angle_deg"])[0])
    r0.run(64)
    oo = r0.observe()
    assert o["step"] == 64
    assert o["iop"] == pytest.approx(oo["iop"], rel=1e-12)
    assert o["wss_cornea"] == pytest.approx(oo["wss_cornea"], rel=1e-12)
    assert o["mass"] == pytest.approx(oo["mass"], rel=1e-12)
    # a second check: its residual against the first check's velocity (S9)
    snap = r0.fields()[0].copy()
    b.check(20)
    r0.run(20)
    oo = r0.observe(snap)
    o = doms[0].last_observables()
    assert o["step"] == 84 and oo["residual"] > 0.0
    assert o["residual"] == pytest.approx(oo["residual"], rel=1e-12)
    for r in refs:
        r.run(20)
    # removal hands the domain back; it keeps stepping alone
    b.remove(doms[2])
    doms[2].step(5)
    refs[2].run(5)
    f, g = pops(doms[2])
    assert np.abs(f - refs[2].f).max() <= 1e-12 * np.abs(refs[2].f).max()
    b.close()


def test_autotuner_keeps_results():
    inst = small_instances(4, seed=3)
    doms = [make(i, "f64") for i in inst]
    refs = []
    for i in inst:
        m, g = O.eye_mask(i["nx"], i["ny"], i["angle_deg"])
        refs.append(O.State(g, O.make_params(**i["params"]), m))
    b = lbm.Batch("f64", max_instances=4, max_tiles=1 << 16, launch=SHAPE)
    for d in doms:
        b.add(d)
    chosen = b.tune(steps_per_candidate=4)
    assert chosen == b.get_launch()
    n = doms[0].step_count
    b.step(33)
    for d, r in zip(doms, refs):
        r.run(n + 33)
        f, g = pops(d)
        assert np.abs(f - r.f).max() <= 1e-12 * np.abs(r.f).max()
    b.close()


def test_batch_capacity_errors():
    inst = small_instances(2, seed=5)
    doms = [make(i, "f32") for i in inst]
    b = lbm.Batch("f32", max_instances=1, max_tiles=1 << 14, launch=SHAPE)
    b.add(doms[0])
    with pytest.raises(lbm.LBMError) as e:
        b.add(doms[1])
    assert e.value.status == lbm.EBUSY
    d64 = make(inst[1], "f64")
    b2 = lbm.Batch("f32", max_instances=2, max_tiles=1 << 14, launch=SHAPE)
    with pytest.raises(lbm.LBMError) as e:
        b2.add(d64)
    assert e.value.status == lbm.EINVAL
    b.close()
    b2.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_dataflow_matches_per_launch_bitwise(prec):
    """One dataflow launch over all members (each member's own parity, mixed
    by a lone odd step before joining) against one launch per step, member
    by member, bit for bit."""
    inst = small_instances(4, seed=13)
    out = []
    for stepping in (lbm.STEP_FLOW, lbm.STEP_PER_LAUNCH):
        shape = dict(tile_w=64, block_rows=4, rows_per_thread=2, blocks_per_sm=0, stepping=stepping)
        doms = [make(i, prec) for i in inst]
        doms[2].step(1)
        b = lbm.Batch(prec, max_instances=4, max_tiles=1 << 16, launch=shape)
        for d in doms:
            b.add(d)
        b.step(37)
        b.check(20)
        out.append([pops(d) for d in doms])
        b.close()
    for (fa, ga), (fb, gb) in zip(*out):
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_fp32_check_step_observables_match_the_oracle():
    """The check step of an FP32 batch computes the observables of interior
    cell pairs on the fast pair path and of boundary cells on the per-cell
    path; both against the FP64 oracle within the FP32 tolerance."""
    inst = small_instances(2, seed=17)
    doms = [make(i, "f32") for i in inst]
    b = lbm.Batch("f32", max_instances=2, max_tiles=1 << 16,
                  launch=dict(tile_w=64, block_rows=4, rows_per_thread=2, blocks_per_sm=0))
    for d in doms:
        b.add(d)
    b.step(45)
    b.check(20)
    for d, i in zip(doms, inst):
        m, g = O.eye_mask(i["nx"], i["ny"], i["angle_deg"])
        r = O.State(g, O.make_params(**i["params"]), m)
        r.run(64)
        oo = r.observe()
        o = d.last_observables()
        assert o["step"] == 64
        for k, kr in [("iop", "iop"), ("mass", "mass"), ("peak_speed", "peak"),
                      ("wss_cornea", "wss_cornea"), ("wss_iris", "wss_iris")]:
            assert o[k] == pytest.approx(oo[kr], rel=2e-5), k
        assert (o["n_fluid"], o["n_cornea"], o["n_iris"]) == (oo["n_fluid"], oo["n_cornea"], oo["n_iris"])
    b.close()


def channel_with_wall(nx=256, ny=128):
    """Periodic fluid channel with a two-row adiabatic wall across it: only
    the rows beside the wall hold boundary cells, 2 of 128 rows, below the
    8 % share from which an FP32 grid takes edge-cell chunks."""
    m, desc = W.porous_box(nx, ny)
    m[:, :] = W.FLUID
    m[ny // 2:ny // 2 + 2, :] = W.ADIABATIC
    params = dict(tau=0.7, tau_T=0.8, drive=(2e-6, 0.0), K_tm=0.5, noise_amp=1e-3, T0=0.3, T_cold=0.2,
                  T_hot=0.4, g_beta=1e-4, g_dir=(0.0, -1.0), seed=5)
    return m, desc, params


def test_split_and_unsplit_members_bitwise_and_against_the_oracle():
    """FP32 members choose edge-cell chunks per grid: a small eye takes them,
    the walled channel does not.  A batch holding both runs the chunked
    kernel, where the channel's rows update every cell as they do alone; so
    each member computes the same bits alone and in the batch, and the
    channel matches the oracle."""
    m, desc, params = channel_with_wall()
    geo = dict(mask=m, **{k: v for k, v in desc.items() if k not in ("nx", "ny")})

    def channel():
        d = lbm.Domain(geo, precision="f32")
        d.set_launch(**SHAPE)
        d.set_params(params)
        return d

    eye = small_instances(1, seed=3)[0]
    ch_alone, eye_alone = channel(), make(eye, "f32")
    assert ch_alone.edge_cell_count() == 0
    assert eye_alone.edge_cell_count() > 0
    ch_mix, eye_mix = channel(), make(eye, "f32")
    b = lbm.Batch("f32", max_instances=2, max_tiles=1 << 16, launch=SHAPE)
    b.add(ch_mix)
    b.add(eye_mix)
    for d in (ch_alone, eye_alone):
        d.step(57)
    b.step(57)
    for a, x in ((ch_alone, ch_mix), (eye_alone, eye_mix)):
        fa, ga = pops(a)
        fx, gx = pops(x)
        assert np.array_equal(fa, fx) and np.array_equal(ga, gx)
    g = O.mask_geom(desc["nx"], desc["ny"], desc["periodic_x"], desc["periodic_y"], desc["inlet_dir"],
                    desc["inlet_profile"], desc["inlet_lo"], desc["inlet_width"])
    ref = O.State(g, O.make_params(**params), m)
    ref.run(57)
    f, gg = pops(ch_mix)
    # the FP32 parity bound of the other tests, max(1e-5, 5e-8 n) of the largest value
    assert np.abs(f - ref.f).max() <= 1e-5 * np.abs(ref.f).max()
    assert np.abs(gg - ref.T).max() <= 1e-5 * np.abs(ref.T).max()
    b.close()
    for d in (ch_alone, eye_alone):
        d.close()
