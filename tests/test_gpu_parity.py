"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs.

FP64 storage and arithmetic must match to 1e-12 relative (the kernel follows
the oracle's evaluation order without FMA contraction, so in practice it is
bit-exact).  FP32 populations must match to max(1e-5, 5e-8 n) relative to the
population scale after n steps: each step rounds every stored population once
(unit roundoff 6e-8), and in the worst case these errors add up linearly.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2102_12663_gb300 import lbm
from paper_2102_12663_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def tol(prec, steps):
    return TOL["f64"] if prec == "f64" else max(TOL["f32"], 5e-8 * steps)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm.load(build_if_missing=True)


def eye_pair(nx, ny, prec, angle=45.0, launch=None, **over):
    pp = W.eye_params(ny, tau=0.8, Ra=1e4, K_tm=0.05)
    pp.update(over)
    dom = lbm.Domain(dict(nx=nx, ny=ny, angle_deg=angle), precision=prec)
    if launch:
        dom.set_launch(**launch)
    dom.set_params(pp)
    m, g = O.eye_mask(nx, ny, angle)
    ref = O.State(g, O.make_params(**pp), m)
    return dom, ref, pp


def mask_pair(mask, desc, prec, params, launch=None):
    geo = dict(mask=mask, **{k: v for k, v in desc.items() if k not in ("nx", "ny")})
    dom = lbm.Domain(geo, precision=prec)
    if launch:
        dom.set_launch(**launch)
    dom.set_params(params)
    g = O.mask_geom(desc["nx"], desc["ny"], desc["periodic_x"], desc["periodic_y"],
                    desc["inlet_dir"], desc["inlet_profile"], desc["inlet_lo"], desc["inlet_width"])
    ref = O.State(g, O.make_params(**params), mask)
    return dom, ref


def pops(dom):
    f, g = dom.populations()
    torch.cuda.synchronize()
    return f.cpu().numpy().reshape(9, -1), g.cpu().numpy().reshape(4, -1)


def rel_err(dom, ref):
    f, g = pops(dom)
    ef = np.abs(f - ref.f).max() / max(np.abs(ref.f).max(), 1e-300)
    eg = np.abs(g - ref.T).max() / max(np.abs(ref.T).max(), 1e-300)
    return max(ef, eg)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_initial_state(prec):
    dom, ref, _ = eye_pair(160, 80, prec)
    assert rel_err(dom, ref) <= (0.0 if prec == "f64" else 1e-7)


@pytest.mark.parametrize("steps", [1, 2, 3, 10, 257])
def test_eye_fp64_stepwise(steps):
    dom, ref, _ = eye_pair(160, 80, "f64")
    dom.step(steps)
    ref.run(steps)
    assert dom.step_count == steps
    assert rel_err(dom, ref) <= TOL["f64"]


def test_eye_fp64_full_config_5000_steps():
    """Plain FP64 model, 160 x 80 eye, 5,000 steps: populations, fields and
    observables against the oracle."""
    dom, ref, pp = eye_pair(160, 80, "f64")
    dom.step(5000)
    ref.run(5000)
    assert rel_err(dom, ref) <= TOL["f64"]
    u, p, T = dom.fields()
    uo, po, To = ref.fields()
    assert np.abs(u.cpu().numpy().reshape(2, -1) - uo).max() <= 1e-12 * np.abs(uo).max()
    assert np.abs(p.cpu().numpy().reshape(-1) - po).max() <= 1e-12 * np.abs(po).max()
    assert np.abs(T.cpu().numpy().reshape(-1) - To).max() <= 1e-12 * np.abs(To).max()
    o = dom.observables()
    oo = ref.observe()
    qi, qo = ref.step()
    for k_gpu, k_ref in [("iop", "iop"), ("mass", "mass"), ("peak_speed", "peak"),
                         ("wss_cornea", "wss_cornea"), ("wss_iris", "wss_iris")]:
        assert o[k_gpu] == pytest.approx(oo[k_ref], rel=1e-12), k_gpu
    assert o["q_in"] == pytest.approx(qi, rel=1e-12)
    assert o["q_out"] == pytest.approx(qo, rel=1e-12)
    assert (o["n_fluid"], o["n_cornea"], o["n_iris"]) == (oo["n_fluid"], oo["n_cornea"], oo["n_iris"])
    assert o["nan_flag"] == 0 and o["residual"] == -1.0


@pytest.mark.parametrize("launch", [
    dict(tile_w=32, block_rows=4, rows_per_thread=1, blocks_per_sm=0),
    dict(tile_w=64, block_rows=1, rows_per_thread=3, blocks_per_sm=0),
    dict(tile_w=256, block_rows=1, rows_per_thread=1, blocks_per_sm=2),
    dict(tile_w=128, block_rows=2, rows_per_thread=4, blocks_per_sm=1),
])
@pytest.mark.parametrize("stepping", [lbm.STEP_FLOW, lbm.STEP_PER_LAUNCH])
def test_ragged_grid_and_launch_shapes(launch, stepping):
    """A grid that is no multiple of any tile (150 x 75, 33 degrees) under
    several tile shapes and grid sizes, with dataflow and per-step launches."""
    dom, ref, _ = eye_pair(150, 75, "f64", angle=33.0, launch=dict(launch, stepping=stepping))
    dom.step(37)
    ref.run(37)
    assert rel_err(dom, ref) <= TOL["f64"]


@pytest.mark.parametrize("gdir", [W.UPRIGHT, W.SUPINE])
def test_eye_fp32(gdir):
    dom, ref, _ = eye_pair(160, 80, "f32", g_dir=gdir)
    dom.step(300)
    ref.run(300)
    assert rel_err(dom, ref) <= tol("f32", 300)


def test_periodic_channel_and_porous_box():
    """Wrap-around in x (channel) and in both directions (porous box)."""
    m, d = W.channel(24, 12)
    P = dict(tau=0.8, tau_T=0.7, drive=(1e-5, 0.0), T_hot=1.0, T_cold=0.0, T0=0.5,
             g_beta=1e-4, g_dir=(0.0, -1.0), noise_amp=1e-3, seed=5)
    dom, ref = mask_pair(m, d, "f64", P)
    dom.step(200)
    ref.run(200)
    assert rel_err(dom, ref) <= TOL["f64"]
    m, d = W.porous_box(40, 20)
    P = dict(tau=0.7, drive=(1e-5, -3e-6), K_tm=0.2, noise_amp=1e-3, T0=0.3, g_beta=1e-4,
             g_dir=(0.6, -0.8), seed=9)
    dom, ref = mask_pair(m, d, "f64", P)
    dom.step(111)
    ref.run(111)
    assert rel_err(dom, ref) <= TOL["f64"]


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("launch", [
    dict(tile_w=64, block_rows=1, rows_per_thread=16, blocks_per_sm=0),
    dict(tile_w=128, block_rows=1, rows_per_thread=5, blocks_per_sm=1),
])
@pytest.mark.parametrize("stepping", [lbm.STEP_FLOW, lbm.STEP_PER_LAUNCH])
def test_periodic_wrap_low_precision(prec, launch, stepping):
    """Wrap-around columns and rows on the FP32-arithmetic paths (pairs at a
    periodic edge, strips that wrap in y; one launch per step takes the
    staged kernel for these one-row shapes), against the FP64 oracle."""
    launch = dict(launch, stepping=stepping)
    m, d = W.porous_box(64, 24)
    m[5:9, 20:30] = 1
    m[12:14, :] = 0  # a fluid lane across the periodic box
    P = dict(tau=0.7, tau_T=0.8, drive=(1e-5, -3e-6), K_tm=0.2, noise_amp=1e-3, T0=0.3,
             g_beta=1e-4, g_dir=(0.6, -0.8), seed=9)
    dom, ref = mask_pair(m, d, prec, P, launch=launch)
    dom.step(60)
    ref.run(60)
    assert rel_err(dom, ref) <= (tol("f32", 60) if prec == "f32" else 3e-3)


def test_darcy_column_plug_inlet_outlet():
    m, d = W.darcy_column(8, 32, 8, 6)
    P = dict(tau=0.8, u_in_max=1e-4, K_tm=0.5, T_in=1.0, T0=0.5)
    for prec in ("f64", "f32"):
        dom, ref = mask_pair(m, d, prec, P)
        dom.step(500)
        ref.run(500)
        assert rel_err(dom, ref) <= tol(prec, 500)


def test_mass_balance_every_step_on_gpu():
    """M(n+1) - M(n) = q_in(n) - q_out(n) (Guo's conserved mass) on the GPU."""
    dom, ref, _ = eye_pair(160, 80, "f64")
    dom.step(100)
    o0 = dom.observables()
    for _ in range(5):
        dom.step(1)
        o1 = dom.observables()
        scale = abs(o0["mass"]) + 1.0
        assert abs((o1["mass"] - o0["mass"]) - (o0["q_in"] - o0["q_out"])) <= 1e-13 * scale
        o0 = o1


def test_write_read_populations_and_checkpoint():
    dom, ref, pp = eye_pair(96, 48, "f64")
    dom.step(5)
    f, g = dom.populations()
    blob = dom.save_state()
    dom.step(7)
    after = pops(dom)
    dom.load_state(blob)
    assert dom.step_count == 5
    f2, g2 = dom.populations()
    assert torch.equal(f, f2) and torch.equal(g, g2)
    # write_populations at odd parity round-trips exactly
    dom.write_populations(f, g)
    f3, g3 = dom.populations()
    assert torch.equal(f, f3) and torch.equal(g, g3)
    dom.step(7)
    again = pops(dom)
    assert np.array_equal(after[0], again[0]) and np.array_equal(after[1], again[1])


def test_run_to_steady_and_errors():
    m, d = W.darcy_column(4, 8, 4, 2)
    P = dict(tau=0.8, u_in_max=1e-4, K_tm=0.5)
    dom, ref = mask_pair(m, d, "f64", P)
    st, steps = dom.run_to_steady(1e-12, check_every=100, max_steps=200000)
    assert st == lbm.OK and steps % 100 == 0 and steps > 100
    o = dom.observables()
    assert 0.0 <= o["residual"] < 1e-12
    assert o["q_out"] == pytest.approx(o["q_in"], rel=1e-9)
    st, steps = dom.run_to_steady(0.0, check_every=50, max_steps=100)
    assert st == lbm.ENOTCONVERGED and steps == 100
    with pytest.raises(lbm.LBMError) as e:
        dom.set_params(dict(P, tau=0.5))
    assert e.value.status == lbm.EINVAL
    with pytest.raises(lbm.LBMError):
        dom.set_params(dict(P, K_tm=0.0))
    with pytest.raises(lbm.LBMError):
        dom.set_params(dict(P, g_beta=1e-3, g_dir=(1.0, 1.0)))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_steady_check_residual_matches_oracle(prec):
    """S9, the steady-state check: the residual of a check is the maximum over
    active cells of |u(n) - u(n - 100)|, u of Eq. 9, against the oracle's
    residual with the velocity of the previous check as its snapshot.  Each
    check observes the last step of its interval, so the second check of a
    run from step s0 compares the states after s0 + 199 and s0 + 99 steps.
    FP32: u sums six populations, so each velocity is off by at most 6 times
    the population tolerance, and the residual by twice that."""
    dom, ref, pp = eye_pair(160, 80, prec)
    s0 = 300
    dom.step(s0)
    st, steps = dom.run_to_steady(0.0, check_every=100, max_steps=200)
    assert st == lbm.ENOTCONVERGED and steps == 200
    o = dom.last_observables()
    assert o["step"] == s0 + 199
    ref.run(s0 + 99)
    snap = ref.fields()[0].copy()
    ref.run(100)
    oo = ref.observe(snap)
    assert oo["residual"] > 1e-7  # the flow is still developing
    if prec == "f64":
        assert o["residual"] == pytest.approx(oo["residual"], rel=1e-12)
        assert o["iop"] == pytest.approx(oo["iop"], rel=1e-12)
        assert o["peak_speed"] == pytest.approx(oo["peak"], rel=1e-12)
    else:
        bound = 12 * tol("f32", s0 + 200) * np.abs(ref.f).max()
        assert abs(o["residual"] - oo["residual"]) <= bound


def test_unstable_parameters_report_nan():
    """A deliberately unstable run (huge inflow at tau close to 1/2) is caught
    by the NaN flag and reported as EUNSTABLE, not as a fault."""
    dom, ref, pp = eye_pair(96, 48, "f32", tau=0.5001, u_in_max=0.9, g_beta=0.05)
    with pytest.raises(lbm.LBMError) as e:
        dom.run_to_steady(1e-9, check_every=100, max_steps=20000)
    assert e.value.status == lbm.EUNSTABLE


def _patch_step_check(dom, x0, y0, w, h, info, pp):
    """Sampled parity at full size: step the oracle on a w x h window of the
    GPU state and compare the window's interior after one GPU step."""
    f, g = dom.populations()
    fw = f[:, y0:y0 + h, x0:x0 + w].cpu().numpy().reshape(9, -1).copy()
    gw = g[:, y0:y0 + h, x0:x0 + w].cpu().numpy().reshape(4, -1).copy()
    del f, g
    mask, _ = lbm.build_mask(dict(nx=dom.nx, ny=dom.ny, angle_deg=45.0))
    mw = np.ascontiguousarray(mask[y0:y0 + h, x0:x0 + w])
    geo = O.mask_geom(w, h, 0, 0, (info["inlet_dir_x"], info["inlet_dir_y"]),
                      info["inlet_profile"], info["inlet_lo"] - (x0 if info["inlet_dir_x"] == 0 else y0),
                      info["inlet_width"])
    st = O.State(geo, O.make_params(**pp), mw)
    st.f[:] = fw
    st.T[:] = gw
    st.step()
    dom.step(1)
    f, g = dom.populations()
    fn = f[:, y0 + 1:y0 + h - 1, x0 + 1:x0 + w - 1].cpu().numpy()
    gn = g[:, y0 + 1:y0 + h - 1, x0 + 1:x0 + w - 1].cpu().numpy()
    fo = st.f.reshape(9, h, w)[:, 1:-1, 1:-1]
    go = st.T.reshape(4, h, w)[:, 1:-1, 1:-1]
    scale = max(np.abs(fo).max(), 1e-30)
    return np.abs(fn - fo).max() / scale, np.abs(gn - go).max() / np.abs(go).max()


@pytest.mark.parametrize("bench_launch", [True, False])
def test_full_size_fp32_sampled_windows(bench_launch):
    """4096 x 2048 FP32 eye in the benchmark's launch configuration (64 x 8
    tiles, dataflow launches) and in the default one: after 2,000 steps,
    windows at the inlet, the trabecular meshwork, the cornea apex and the
    chamber interior match one oracle step computed from the same state."""
    import bench
    nx, ny = 4096, 2048
    pp = W.config_params(W.CONFIG_FP32)
    dom = lbm.Domain(dict(nx=nx, ny=ny, angle_deg=45.0), precision="f32")
    if bench_launch:
        dom.set_launch(**bench.LAUNCH)
    dom.set_params(pp)
    dom.step(2000)
    info = dom.info()
    windows = [(info["inlet_lo"] - 8, 200, 48, 24),   # ciliary inlet
               (150, 200, 48, 48),                    # TM block / angle
               (2020, 960, 48, 48),                   # cornea near the apex
               (1500, 500, 48, 48)]                   # chamber interior
    for (x0, y0, w, h) in windows:
        ef, eg = _patch_step_check(dom, x0, y0, w, h, info, pp)
        assert ef <= 1e-5 and eg <= 1e-5, (x0, y0, ef, eg)
    o = dom.observables()
    assert o["nan_flag"] == 0 and o["n_fluid"] == info["n_fluid"]


def _lumped_oracle_checks(ref, params, h_tm, checks, every):
    """The host side of the lumped meshwork (Sec. 2.3) in the oracle, in the
    cadence of lbm_run_to_steady: every-1 plain steps, one observed step, then
    the seepage speed for the observed IOP."""
    for _ in range(checks):
        ref.run(every - 1)
        o = ref.observe()
        ref.step()
        params.u_seep = O.seepage_velocity(params, o["iop"], h_tm)


def test_lumped_tm_eye_fp64_parity():
    """Paper's lumped meshwork on the eye (no drag in the TM cells, seepage
    velocity at the outlets fed back from the IOP every 50 steps)."""
    h_tm = 3.0
    dom, ref, pp = eye_pair(160, 80, "f64", tm_model=1, h_tm=h_tm)
    P = O.make_params(**pp)
    ref.params = P
    st, steps = dom.run_to_steady(0.0, check_every=50, max_steps=400)
    assert steps == 400
    _lumped_oracle_checks(ref, P, h_tm, 8, 50)
    assert rel_err(dom, ref) <= 1e-12
    o = dom.observables()
    assert o["u_seep"] == pytest.approx(P.u_seep, rel=1e-12) and o["u_seep"] > 0


def test_lumped_tm_column_reaches_darcy_iop_on_gpu():
    m, d = W.darcy_column(12, 0, 12, 2)
    u, K, h, tau = 1e-4, 0.5, 4.0, 0.8
    geo = dict(mask=m, **{k: v for k, v in d.items() if k not in ("nx", "ny")})
    for prec, tol_rel in (("f64", 1e-8), ("f32", 1e-4)):
        dom = lbm.Domain(geo, precision=prec)
        dom.set_params(dict(tau=tau, u_in_max=u, K_tm=K, tm_model=1, h_tm=h))
        st, steps = dom.run_to_steady(1e-13 if prec == "f64" else 1e-9, check_every=50,
                                      max_steps=40000)
        o = dom.observables()
        nu = (2 * tau - 1) / 6
        assert o["iop"] == pytest.approx(nu * h * u / K, rel=tol_rel)
        assert o["q_out"] == pytest.approx(o["q_in"], rel=tol_rel)


@pytest.mark.parametrize("prec,unit_roundoff", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_eye_sixteen_bit_storage(prec, unit_roundoff):
    """16-bit deviation storage against the FP64 oracle after n = 100 steps:
    every step re-rounds each stored population once (relative unit roundoff u
    of the format), so the deviation stays within a few u sqrt(n) of the
    population scale; a wrong slot or scale would be off by O(1)."""
    n = 100
    dom, ref, _ = eye_pair(160, 80, prec)
    dom.step(n)
    ref.run(n)
    assert rel_err(dom, ref) <= 4.0 * unit_roundoff * n ** 0.5


STAGED_SHAPES = [
    dict(tile_w=64, block_rows=1, rows_per_thread=4, blocks_per_sm=0),
    dict(tile_w=256, block_rows=1, rows_per_thread=2, blocks_per_sm=1),
]


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("nx,ny", [(160, 80), (200, 100), (150, 75)])
@pytest.mark.parametrize("launch", range(len(STAGED_SHAPES)))
def test_staged_kernel_eye(prec, nx, ny, launch):
    """The warp-specialised staged kernel (one launch per step of a one-row
    shape with tiles of whole 64-cell segments) on grids whose mask rows are
    staged (nx a multiple of 16), read from global memory (nx = 200), or
    whose rows are not staged at all (nx = 150: population rows off the
    16-byte grid), after an odd and an even number of steps, against the FP64
    oracle (16-bit storages: a few unit roundoffs times sqrt(n), as above)."""
    dom, ref, _ = eye_pair(nx, ny, prec, launch=STAGED_SHAPES[launch])
    u = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}.get(prec)
    done = 0
    for n in (1, 40):
        dom.step(n)
        ref.run(n)
        done += n
        bound = tol("f32", done) if u is None else 4.0 * u * done ** 0.5
        assert rel_err(dom, ref) <= bound, done


@pytest.mark.parametrize("stepping", [lbm.STEP_FLOW, lbm.STEP_PER_LAUNCH])
def test_last_observables_after_steady_loop(stepping):
    """lbm_last_observables after lbm_run_to_steady returns the last check's
    observables: those of the state after 99 steps (the check observes before
    its own update), as a separate domain stepped 99 times reads them, to the
    FP32 partials' precision; the residual of the second check is defined."""
    launch = dict(tile_w=64, block_rows=4, rows_per_thread=2, blocks_per_sm=0, stepping=stepping)
    dom, _, pp = eye_pair(160, 80, "f32", launch=launch)
    with pytest.raises(lbm.LBMError):
        dom.last_observables()
    st, steps = dom.run_to_steady(0.0, check_every=50, max_steps=100)
    assert steps == 100 and dom.step_count == 100
    got = dom.last_observables()
    twin, _, _ = eye_pair(160, 80, "f32", launch=launch)
    twin.step(99)
    ref = twin.observables()
    assert got["step"] == 99 and ref["step"] == 99
    for k in ("iop", "mass", "peak_speed", "wss_cornea", "wss_iris", "q_in", "q_out"):
        assert got[k] == pytest.approx(ref[k], rel=1e-5), k
    for k in ("n_fluid", "n_cornea", "n_iris", "nan_flag"):
        assert got[k] == ref[k], k
    assert got["residual"] > 0.0


def test_supine_eye_mirror_symmetry_fp32():
    """The supine eye without noise stays mirror-symmetric on the FP32 path
    (cell pairs, shuffled x-shifted links in both directions)."""
    dom, ref, _ = eye_pair(160, 80, "f32", g_dir=W.SUPINE, noise_amp=0.0)
    dom.step(600)
    u, p, T = (t.cpu().numpy() for t in dom.fields())
    ux, uy = u[0], u[1]
    assert np.abs(ux + ux[:, ::-1]).max() <= 1e-5 * np.abs(ux).max()
    assert np.abs(uy - uy[:, ::-1]).max() <= 1e-5 * np.abs(uy).max()
    assert np.abs(T - T[:, ::-1]).max() <= 1e-5


@pytest.mark.parametrize("launch", [
    dict(tile_w=32, block_rows=1, rows_per_thread=4, blocks_per_sm=0),   # 16-thread blocks
    dict(tile_w=64, block_rows=4, rows_per_thread=2, blocks_per_sm=0),
])
def test_fp32_observables_any_block_width(launch):
    """Observables of the FP32 eye through the check step (which also
    writes) and through an observe-only read, for blocks narrower than a
    warp and for full warps, against the oracle."""
    dom, ref, _ = eye_pair(160, 80, "f32", launch=launch)
    st, steps = dom.run_to_steady(0.0, check_every=60, max_steps=120)
    assert steps == 120
    ref.run(120)
    o, oo = dom.observables(), ref.observe()
    for k, kr in [("iop", "iop"), ("mass", "mass"), ("peak_speed", "peak"),
                  ("wss_cornea", "wss_cornea"), ("wss_iris", "wss_iris")]:
        assert o[k] == pytest.approx(oo[kr], rel=2e-5), k
    assert o["residual"] > 0.0


VEC16_SHAPES = [
    dict(tile_w=256, block_rows=2, rows_per_thread=2, blocks_per_sm=0, stepping=lbm.STEP_PER_LAUNCH),
    dict(tile_w=256, block_rows=4, rows_per_thread=1, blocks_per_sm=0, stepping=lbm.STEP_FLOW),
    dict(tile_w=128, block_rows=4, rows_per_thread=1, blocks_per_sm=0, stepping=lbm.STEP_PER_LAUNCH),
]


@pytest.mark.parametrize("prec,unit_roundoff", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
@pytest.mark.parametrize("nx,ny", [(512, 256), (520, 130), (516, 130)])
@pytest.mark.parametrize("launch", range(len(VEC16_SHAPES)))
def test_vector16_path_eye(prec, unit_roundoff, nx, ny, launch):
    """The vector paths of the 16-bit storages (eight cells and one 16-byte
    vector per plane and lane on 256-cell tile rows, four cells and 8-byte
    vectors on 128-cell rows) against the FP64 oracle after an
    odd and an even number of steps (a few unit roundoffs times sqrt(n), as
    for the pair path), and against the pair-path shape within the same
    bound.  512 x 256 has whole interior rows; 520 x 130 ends in a partial
    tile (the last segment falls back to cell pairs); 516 x 130 is no multiple
    of eight columns (every eight-cell row falls back; four-cell rows do not)."""
    dom, ref, _ = eye_pair(nx, ny, prec, launch=VEC16_SHAPES[launch])
    pair, _, _ = eye_pair(nx, ny, prec, launch=dict(tile_w=64, block_rows=4, rows_per_thread=1))
    done = 0
    for n in (1, 40):
        dom.step(n)
        pair.step(n)
        ref.run(n)
        done += n
        bound = 4.0 * unit_roundoff * done ** 0.5
        assert rel_err(dom, ref) <= bound, done
        fv, gv = pops(dom)
        fp, gp = pops(pair)
        assert np.abs(fv - fp).max() <= bound * np.abs(ref.f).max()
        assert np.abs(gv - gp).max() <= bound * np.abs(ref.T).max()


@pytest.mark.parametrize("prec,unit_roundoff", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_vector16_path_periodic_wrap(prec, unit_roundoff):
    """Vector rows that wrap around periodic edges: the lanes at column 0 and
    at the last column fetch and store the code across the edge."""
    m, d = W.porous_box(256, 24)
    m[5:9, 20:60] = 1
    m[12:14, :] = 0
    P = dict(tau=0.7, tau_T=0.8, drive=(1e-5, -3e-6), K_tm=0.2, noise_amp=1e-3, T0=0.3,
             g_beta=1e-4, g_dir=(0.6, -0.8), seed=9)
    dom, ref = mask_pair(m, d, prec, P, launch=VEC16_SHAPES[0])
    dom.step(61)
    ref.run(61)
    assert rel_err(dom, ref) <= 4.0 * unit_roundoff * 61 ** 0.5
