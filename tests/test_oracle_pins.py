"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: algebraic
identities of Guo's incompressible equilibrium (Sec. 2.3, Eqs. 7-9), the
transport coefficients of Eqs. 10 and 14 measured from decaying waves,
closed-form flows (plane Poiseuille, uniform Darcy flow, Brinkman channel,
Darcy pressure drop, pure conduction, Poiseuille flow against a wall at a
fractional link position), the Rayleigh-Benard onset, the exact per-step mass
balance, mirror symmetry, and published test vectors.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2102_12663_gb300 import workloads as W

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector():
    """Counter-based noise generator: SplitMix64 against its published outputs."""
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    gamma = 0x9E3779B97F4A7C15
    for k, v in enumerate(vals):
        assert O.splitmix64((k * gamma) % 2**64) == v


def test_equilibrium_values_at_rest():
    """Eq. 7 at u = 0 with the reading sigma = 5/12, lambda = 1/3, gamma = 1/12."""
    f = O.feq(1.0, 0.0, 0.0)
    assert f[0] == pytest.approx(-4 * 5 / 12, rel=1e-15)
    assert np.allclose(f[1:5], 1 / 3, rtol=1e-15)
    assert np.allclose(f[5:9], 1 / 12, rtol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(seed):
    """Eqs. 7-9: sum feq = 0, sum e feq = u, sum e e feq = p I + u u, and
    the moments of Eq. 9 recover (p, u) from feq."""
    rng = np.random.default_rng(seed)
    p, ux, uy = rng.normal(0, 1e-2), rng.normal(0, 3e-2), rng.normal(0, 3e-2)
    f = O.feq(p, ux, uy)
    assert abs(f.sum()) < 1e-16
    assert f @ EX == pytest.approx(ux, abs=1e-17)
    assert f @ EY == pytest.approx(uy, abs=1e-17)
    assert f @ (EX * EX) == pytest.approx(p + ux * ux, abs=1e-16)
    assert f @ (EY * EY) == pytest.approx(p + uy * uy, abs=1e-16)
    assert f @ (EX * EY) == pytest.approx(ux * uy, abs=1e-17)
    p2, ux2, uy2 = O.moments(f)
    assert (p2, ux2, uy2) == pytest.approx((p, ux, uy), abs=1e-16)


def _rand_cell(rng):
    f = O.feq(rng.normal(0, 1e-2), rng.normal(0, 1e-2), rng.normal(0, 1e-2))
    f = f + rng.normal(0, 1e-4, 9)
    g = 0.25 * (0.5 + rng.normal(0, 0.1)) + rng.normal(0, 1e-3, 4)
    return f, g


@pytest.mark.parametrize("porous", [False, True])
def test_collision_invariants(porous):
    """Collision conserves sum_{i>=1} f (the mass of Guo's model, Eq. 9) and
    T (Eq. 13); the flow momentum changes by exactly the applied force
    (Eq. 17) in fluid cells."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        f, g = _rand_cell(rng)
        drive = rng.normal(0, 1e-5, 2)
        P = O.make_params(tau=rng.uniform(0.55, 1.5), tau_T=rng.uniform(0.55, 1.5),
                          drive=tuple(drive), K=rng.uniform(0.05, 5.0))
        fs, gs = O.collide(P, porous, f, g)
        assert fs[1:].sum() == pytest.approx(f[1:].sum(), abs=1e-16)
        assert gs.sum() == pytest.approx(g.sum(), abs=1e-15)
        _, ux, uy = O.moments(f)
        jx, jy = fs @ EX, fs @ EY
        if not porous:
            assert jx == pytest.approx(ux + drive[0], abs=1e-16)
            assert jy == pytest.approx(uy + drive[1], abs=1e-16)
        else:
            # Darcy drag of Eq. 4 taken at the mid-step momentum
            nu = (2 * P.tau - 1) / 6
            umx = (ux + 0.5 * drive[0]) / (1 + nu / (2 * P.K))
            assert jx == pytest.approx(ux + drive[0] - nu / P.K * umx, abs=1e-16)


def test_buoyancy_force_direction_and_size():
    """Eq. 17 (generalised to every axis link): the force adds
    -g beta (T - T0) g_hat of momentum and no mass; it lives on i = 1..4."""
    f, g = _rand_cell(np.random.default_rng(9))
    T = g.sum()
    for gdir in [(0.0, -1.0), (-1.0, 0.0), (0.6, -0.8)]:
        P0 = O.make_params(tau=0.9, tau_T=0.7, T0=0.3)
        P1 = O.make_params(tau=0.9, tau_T=0.7, T0=0.3, g_beta=1e-3, g_dir=gdir)
        d = O.collide(P1, False, f, g)[0] - O.collide(P0, False, f, g)[0]
        assert abs(d.sum()) < 1e-18
        assert np.all(d[5:] == 0) and d[0] == 0
        assert d @ EX == pytest.approx(-1e-3 * (T - 0.3) * gdir[0], rel=1e-12, abs=1e-20)
        assert d @ EY == pytest.approx(-1e-3 * (T - 0.3) * gdir[1], rel=1e-12, abs=1e-20)
        # hot fluid (T > T0) is pushed against gravity
        assert (d @ EX) * gdir[0] + (d @ EY) * gdir[1] < 0


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.3])
def test_shear_wave_viscosity(tau):
    """Eq. 10: a decaying shear wave in a periodic box gives nu = (2 tau - 1)/6."""
    n = 64
    k = 2 * math.pi / n
    m = np.zeros((n, 1), np.uint8)
    s = O.State(O.mask_geom(1, n, 1, 1), O.make_params(tau=tau), m)
    for c in range(n):
        s.f[:, c] = O.feq(0.0, 1e-4 * math.sin(k * c), 0.0)
    s.run(100)
    a1 = np.abs(s.fields()[0][0]).max()
    s.run(400)
    a2 = np.abs(s.fields()[0][0]).max()
    nu = -math.log(a2 / a1) / (400 * k * k)
    assert nu == pytest.approx((2 * tau - 1) / 6, rel=5e-3)


@pytest.mark.parametrize("tau_T", [0.55, 0.8, 1.2])
def test_diffusion_wave_diffusivity(tau_T):
    """Eq. 14: a decaying temperature wave at rest gives theta = (2 tau_T - 1)/4."""
    n = 64
    k = 2 * math.pi / n
    m = np.zeros((1, n), np.uint8)
    s = O.State(O.mask_geom(n, 1, 1, 1), O.make_params(tau=0.8, tau_T=tau_T), m)
    s.T[:] = 0.25 * (1.0 + 0.1 * np.sin(k * np.arange(n)))[None, :]
    s.run(100)
    a1 = np.abs(s.fields()[2] - 1).max()
    s.run(400)
    a2 = np.abs(s.fields()[2] - 1).max()
    theta = -math.log(a2 / a1) / (400 * k * k)
    assert theta == pytest.approx((2 * tau_T - 1) / 4, rel=5e-3)


def _channel_profile(H, tau, G, porous=False, K=1.0):
    m, d = W.channel(2, H, porous=porous)
    s = O.State(O.mask_geom(d["nx"], d["ny"], 1, 0),
                O.make_params(tau=tau, drive=(G, 0.0), K=K), m)
    nu = (2 * tau - 1) / 6
    s.run(int(8 * H * H / nu) if not porous else int(40 * K / nu + 8 * min(H * H, 50 * K) / nu))
    u = s.fields()[0][0].reshape(d["ny"], d["nx"])[1:-1, 0]
    return s, u, nu


def test_plane_poiseuille_second_order():
    """Halfway bounce-back + BGK + forcing: steady plane Poiseuille flow
    u = G/(2 nu) (y - 1/2)(H + 1/2 - y) with second-order convergence."""
    errs = []
    for H in (8, 16, 32):
        _, u, nu = _channel_profile(H, 0.8, 1e-6)
        y = np.arange(1, H + 1)
        ex = 1e-6 / (2 * nu) * (y - 0.5) * (H + 0.5 - y)
        errs.append(np.abs(u - ex).max() / ex.max())
    assert errs[-1] < 1e-3
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.5


def test_wall_shear_stress_channel():
    """Sec. 3.6 WSS from the non-equilibrium stress: in Poiseuille flow the
    shear stress half a cell from the wall is G (H - 1) / 2 exactly."""
    H, G = 32, 1e-6
    s, _, _ = _channel_profile(H, 0.8, G)
    o = s.observe()
    assert o["wss_iris"] == pytest.approx(G * (H - 1) / 2, rel=1e-9)
    assert o["wss_cornea"] == pytest.approx(G * (H - 1) / 2, rel=1e-9)
    assert o["n_iris"] == 2 and o["n_cornea"] == 2


def test_uniform_porous_box_darcy_velocity():
    """Eq. 4 in a uniform periodic porous box driven by G: u = K G / nu to
    round-off."""
    m, d = W.porous_box(4, 4)
    for K in (0.05, 0.5, 5.0):
        P = O.make_params(tau=0.8, drive=(1e-5, -2e-6), K=K)
        s = O.State(O.mask_geom(4, 4, 1, 1), P, m)
        s.run(400 + int(40 * K / 0.1))
        u = s.fields()[0]
        assert np.allclose(u[0], K * 1e-5 / 0.1, rtol=1e-12)
        assert np.allclose(u[1], -K * 2e-6 / 0.1, rtol=1e-12)


def test_brinkman_channel_second_order():
    """Porous channel (Brinkman with effective viscosity nu):
    u = (G K / nu)[1 - cosh((y - y_c)/sqrt K) / cosh(H / (2 sqrt K))],
    converging as the lattice resolves sqrt K (H / sqrt K fixed)."""
    errs = []
    for H in (16, 32):
        K = (H / 8.0) ** 2
        _, u, nu = _channel_profile(H, 0.8, 1e-6, porous=True, K=K)
        y = np.arange(1, H + 1)
        yc, sk = (H + 1) / 2, math.sqrt(K)
        ex = 1e-6 * K / nu * (1 - np.cosh((y - yc) / sk) / np.cosh(H / (2 * sk)))
        errs.append(np.abs(u - ex).max() / ex.max())
    assert errs[0] < 6e-3 and errs[1] < errs[0] / 2.5


@pytest.mark.parametrize("K", [0.05, 0.5, 2.0])
def test_darcy_pressure_drop_and_iop(K):
    """Inlet -> fluid -> porous block (length L) -> fluid -> outlet, periodic
    across: the drop over the block is nu Q L / K (mu Q L / (K A) per unit
    width), the interior slope is -(nu/K) Q, outflow equals inflow, and IOP
    (mean p over fluid cells) equals the upstream share of the drop."""
    n_in, L, n_out, ny, u, tau = 8, 32, 8, 2, 1e-4, 0.8
    nu = (2 * tau - 1) / 6
    m, d = W.darcy_column(n_in, L, n_out, ny)
    g = O.mask_geom(d["nx"], d["ny"], 0, 1, d["inlet_dir"], d["inlet_profile"])
    s = O.State(g, O.make_params(tau=tau, u_in_max=u, K=K), m)
    s.run(4000 + int(3000 / K))
    p = s.fields()[1].reshape(ny, -1)[0]
    x0, x1 = 1 + n_in, 1 + n_in + L
    dp = nu * u * L / K
    assert p[x0 - 1] - p[x1] == pytest.approx(dp, rel=1e-9)
    slope = np.diff(p[x0 + 2:x1 - 2])
    assert np.allclose(slope, -nu / K * u, rtol=1e-9)
    o = s.observe()
    assert o["iop"] == pytest.approx(dp * n_in / (n_in + n_out), rel=1e-9)
    qi, qo = s.step()
    assert qi == pytest.approx(u * ny, rel=1e-12)
    assert qo == pytest.approx(qi, rel=1e-9)


def test_pure_conduction_linear_profile():
    """Eqs. 11-14 with anti-bounce-back Dirichlet walls at rest: the steady
    temperature is linear between the halfway walls, to round-off."""
    H = 16
    m, d = W.channel(2, H)
    P = O.make_params(tau=0.8, tau_T=0.7, T_hot=1.0, T_cold=0.0, T0=0.5)
    s = O.State(O.mask_geom(2, H + 2, 1, 0), P, m)
    s.run(30000)
    u, _, T = s.fields()
    Ty = T.reshape(H + 2, 2)[1:-1, 0]
    y = np.arange(1, H + 1)
    assert np.abs(Ty - (1.0 - (y - 0.5) / H)).max() < 1e-12
    assert np.abs(u).max() == 0.0


def _rb_growth(Ra, H=16, nx=32, tau=0.8):
    m, d = W.channel(nx, H)
    tT = W.tau_T_for_Pr(tau, 1.0)
    gb = W.ra_to_gbeta(Ra, tau, tT, 1.0, H)
    P = O.make_params(tau=tau, tau_T=tT, g_beta=gb, g_dir=(0, -1), T_hot=1.0,
                      T_cold=0.0, T0=0.5, noise_amp=1e-3, seed=7)
    s = O.State(O.mask_geom(nx, H + 2, 1, 0), P, m)
    s.run(4000)
    e1 = float((s.fields()[0][0] ** 2).sum())
    s.run(8000)
    e2 = float((s.fields()[0][0] ** 2).sum())
    return e2 / e1


def test_rayleigh_benard_onset():
    """Boussinesq coupling (Eqs. 5, 15-17): a fluid layer heated from below
    between rigid walls stays conductive below the textbook critical
    Rayleigh number 1708 and convects above it."""
    assert _rb_growth(1500.0) < 1e-3
    assert _rb_growth(2000.0) > 10.0


def _eye(nx=160, ny=80, **kw):
    m, g = O.eye_mask(nx, ny, kw.pop("angle_deg", 45.0))
    pp = W.eye_params(ny, tau=0.8, Ra=1e4, K_tm=0.05)
    pp.update(kw)
    return m, g, O.make_params(**pp)


def test_mass_balance_every_step():
    """Guo's model conserves M = sum_{i>=1} f in collision, so each step
    M(n+1) - M(n) = q_in(n) - q_out(n) up to round-off."""
    m, g, P = _eye()
    s = O.State(g, P, m)
    s.run(300)
    for _ in range(10):
        m0 = s.observe()["mass"]
        qi, qo = s.step()
        m1 = s.observe()["mass"]
        assert abs((m1 - m0) - (qi - qo)) <= 1e-13 * np.abs(s.f[1:]).sum()
    assert qi == pytest.approx(0.005 * 4 * (0.4375 * 2 + 0.9375 * 2) / 4, rel=1e-12)


def test_rest_state_stays_at_rest():
    """No inflow, no temperature difference, no noise: u = 0 and p = p_out
    exactly, whatever the gravity direction."""
    for gdir in (W.UPRIGHT, W.SUPINE):
        m, g, P = _eye(u_in_max=0.0, T_hot=0.5, T_cold=0.5, T_in=0.5, T0=0.5,
                       noise_amp=0.0, g_dir=gdir)
        s = O.State(g, P, m)
        s.run(300)
        u, p, _ = s.fields()
        assert np.abs(u).max() == 0.0 and np.abs(p).max() == 0.0


def test_supine_eye_mirror_symmetry():
    """Mirror-symmetric eye, gravity along the optical axis, no noise: u_x is
    odd and u_y, p, T are even about the mid-line (the two mirror vortices of
    the up-facing eye)."""
    m, g, P = _eye(g_dir=W.SUPINE, noise_amp=0.0)
    s = O.State(g, P, m)
    s.run(1500)
    u, p, T = s.fields()
    ux, uy = u[0].reshape(80, 160), u[1].reshape(80, 160)
    p, T = p.reshape(80, 160), T.reshape(80, 160)
    assert np.abs(ux + ux[:, ::-1]).max() < 1e-12 * np.abs(ux).max()
    assert np.abs(uy - uy[:, ::-1]).max() < 1e-12 * np.abs(uy).max()
    assert np.abs(p - p[:, ::-1]).max() < 1e-12 * np.abs(p).max()
    assert np.abs(T - T[:, ::-1]).max() < 1e-12


@pytest.mark.parametrize("angle", [20.0, 30.0, 45.0])
def test_eye_geometry(angle):
    """The analytic eye: mirror-symmetric, one inlet gap, two TM blocks with
    outlets behind, and a cornea arc whose sagitta a tan(alpha/2) sets the
    chamber angle alpha."""
    nx, ny = 320, 160
    m, g = O.eye_mask(nx, ny, angle)
    assert np.array_equal(m, m[:, ::-1])
    assert (m == O.INLET).sum() == g.inlet_width == 8
    assert (m == O.OUTLET).sum() == 2 * 20
    band = 16
    xa = 12 + 2
    a = nx / 2 - xa
    h = a * math.tan(math.radians(angle) / 2)
    fluid_rows = np.where((m == O.FLUID).any(axis=1))[0]
    assert fluid_rows.min() == band
    assert abs((fluid_rows.max() + 0.5) - (band - 0.5 + h)) <= 1.0
    cols = np.where((m == O.FLUID).any(axis=0))[0]
    assert cols.min() >= xa and cols.max() <= nx - 1 - xa
    assert abs((cols.max() - cols.min() + 1) - 2 * a) <= 2.0


def test_lumped_tm_steady_state_obeys_darcy_law():
    """Lumped meshwork of Sec. 2.3: with the seepage velocity fed back from the
    IOP, the steady state balances inflow and outflow and the IOP satisfies
    Darcy's law (Eq. 4) across the meshwork, IOP - p_0 = mu h Q / (K A)."""
    m, d = W.darcy_column(12, 0, 12, 2)
    g = O.mask_geom(d["nx"], d["ny"], 0, 1, d["inlet_dir"], d["inlet_profile"])
    u, K, h, tau = 1e-4, 0.5, 4.0, 0.8
    P = O.make_params(tau=tau, u_in_max=u, K_tm=K, tm_model=1)
    s = O.State(g, P, m)
    nu = (2 * tau - 1) / 6
    for _ in range(300):
        s.run(49)
        o = s.observe()
        s.step()
        P.u_seep = O.seepage_velocity(P, o["iop"], h)
    o = s.observe()
    qi, qo = s.step()
    assert o["iop"] == pytest.approx(nu * h * u / K, rel=1e-8)
    assert P.u_seep == pytest.approx(u, rel=1e-8)
    assert qo == pytest.approx(qi, rel=1e-8)


# ---- vortex measures (Eq. 18, Tab. 3) ----------------------------------------

def test_vortex_taylor_green_closed_forms():
    """Taylor-Green field u_x = U sin(kx) cos(ky), u_y = -U cos(kx) sin(ky) on a
    fully periodic box.  The centred differences of the trigonometric field are
    exact multiples of it: 2 omega_z = 2 U sin(k) sin(kx) sin(ky), so the
    signed sum over whole periods is zero and the sum of |2 omega_z| factors
    into (sum_x |sin kx|)^2.  The midpoint sum of u_x along y is
    U sin(kx) (cot(k/2) sin(ky) + 1) / 2, largest at (n/4, n/4) and smallest
    at (3n/4, n/4)."""
    n, U = 32, 1e-3
    k = 2 * math.pi / n
    x = np.arange(n)
    X, Y = np.meshgrid(x, x)  # [y, x]
    u = np.stack([U * np.sin(k * X) * np.cos(k * Y), -U * np.cos(k * X) * np.sin(k * Y)])
    m, d = W.porous_box(n, n)
    m[:] = O.FLUID
    g = O.mask_geom(n, n, 1, 1)
    v = O.vortex(g, m, u)
    s1 = np.abs(np.sin(k * x)).sum()
    assert v["n_fluid"] == n * n
    assert abs(v["intensity"]) <= 1e-15 * n * n * U
    assert v["intensity_abs"] == pytest.approx(2 * U * math.sin(k) * s1 * s1, rel=1e-12)
    peak = U * (1 / math.tan(k / 2) + 1) / 2
    assert v["psi_max"] == pytest.approx(peak, rel=1e-12)
    assert (v["max_x"], v["max_y"]) == (n // 4, n // 4)
    assert v["psi_min"] == pytest.approx(-peak, rel=1e-12)
    assert (v["min_x"], v["min_y"]) == (3 * n // 4, n // 4)


def test_vortex_poiseuille_wall_stencil_and_ties():
    """Plane Poiseuille u_x = G Y (H - Y), Y = y - 1/2, between halfway walls
    (fluid rows 1..H, periodic in x).  Interior rows see the exact slope
    G (H - 2Y); a wall row sees the wall value 0 at distance 1/2, which gives
    the one-sided slope +-G (H - 3/2).  The signed sum vanishes by symmetry.
    psi grows with y in every column, so its extrema are ties across x that go
    to x = 0."""
    H, nx, G = 20, 6, 1e-5
    m, d = W.channel(nx, H)
    g = O.mask_geom(nx, H + 2, 1, 0)
    y = np.arange(H + 2, dtype=float)
    Yc = y - 0.5
    prof = np.where((y >= 1) & (y <= H), G * Yc * (H - Yc), 0.0)
    u = np.zeros((2, H + 2, nx))
    u[0] = prof[:, None]
    v = O.vortex(g, m, u)
    slope = [G * (H - 1.5)] + [G * (H - 2 * (j - 0.5)) for j in range(2, H)] + [-G * (H - 1.5)]
    assert v["intensity"] == pytest.approx(0.0, abs=1e-15 * nx * H * G * H)
    assert v["intensity_abs"] == pytest.approx(nx * sum(abs(s) for s in slope), rel=1e-12)
    top = sum(prof[1:H]) + 0.5 * prof[H]
    assert v["psi_max"] == pytest.approx(top, rel=1e-14)
    assert (v["max_x"], v["max_y"]) == (0, H)
    assert v["psi_min"] == pytest.approx(0.5 * prof[1], rel=1e-14)
    assert (v["min_x"], v["min_y"]) == (0, 1)


# ---- interpolated bounce-back on a curved wall (Bouzidi, [36] of the paper) ---

def test_link_q_closed_forms():
    """Link fractions to a circle: an axis link from (10, 0) to the circle of
    radius 10.3 about the origin meets it at 0.3; a diagonal link from (7, 7)
    to the circle of radius 10 at t = sqrt(50) - 7."""
    g = O.mask_geom(32, 32, arc=(0.0, 0.0, 10.3))
    assert O.link_q(g, 10, 0, 1) == pytest.approx(0.3, abs=1e-14)
    assert O.link_q(g, 0, 10, 2) == pytest.approx(0.3, abs=1e-14)
    g = O.mask_geom(32, 32, arc=(0.0, 0.0, 10.0))
    assert O.link_q(g, 7, 7, 5) == pytest.approx(math.sqrt(50.0) - 7.0, abs=1e-14)
    assert O.link_q(g, -7, -7, 7) == pytest.approx(math.sqrt(50.0) - 7.0, abs=1e-14)


def _fractional_wall_profile(H, q0, bouzidi, tau=0.8, G=1e-6):
    """Channel with the halfway bottom wall at y = 1/2 and a flat top wall at
    y = H + q0 (a circle of radius 1e5: its sag over the two columns is
    1e-6 cells), fluid rows 1..H."""
    m, d = W.channel(2, H)
    R = 1e5
    g = O.mask_geom(d["nx"], d["ny"], 1, 0, arc=(0.5, H + q0 - R, R))
    s = O.State(g, O.make_params(tau=tau, drive=(G, 0.0), bouzidi=bouzidi), m)
    nu = (2 * tau - 1) / 6
    s.run(int(8 * H * H / nu))
    u = s.fields()[0][0].reshape(d["ny"], d["nx"])[1:-1, 0]
    y = np.arange(1, H + 1)
    ex = G / (2 * nu) * (y - 0.5) * (H + q0 - y)
    return np.abs(u - ex).max() / ex.max()


@pytest.mark.parametrize("q0", [0.25, 0.75])
def test_bouzidi_places_the_wall_second_order(q0):
    """Plane Poiseuille between a halfway wall and a wall at fraction q0 of
    the last link (both branches of the rule): the interpolated bounce-back
    converges at second order to u = G/(2 nu)(y - 1/2)(H + q0 - y), while
    halfway bounce-back, which puts the wall at H + 1/2, keeps a first-order
    error."""
    errs = [_fractional_wall_profile(H, q0, 1) for H in (8, 16, 32)]
    for a, b in zip(errs, errs[1:]):
        assert 3.0 < a / b < 5.0
    halfway = _fractional_wall_profile(32, q0, 0)
    assert errs[-1] < halfway / 10


def test_residual_of_decaying_shear_waves():
    """Steady-state residual (max over cells of |u(t) - u(t - D)|): two
    crossed shear waves u_x = U sin(k y), u_y = V sin(k x) in a periodic box
    each decay as exp(-nu k^2 t) with nu from Eq. 10, so at the cell where
    both sines are 1 the residual over an interval of D steps ending at t is
    sqrt(U^2 + V^2) e^{-nu k^2 (t - D)} (1 - e^{-nu k^2 D}).  Different
    amplitudes make a dropped component, a squared norm or max |u| fail."""
    n, tau, U, V = 64, 0.8, 1e-5, 2e-5
    k = 2 * math.pi / n
    nu = (2 * tau - 1) / 6
    m = np.zeros((n, n), np.uint8)
    s = O.State(O.mask_geom(n, n, 1, 1), O.make_params(tau=tau), m)
    for y in range(n):
        for x in range(n):
            s.f[:, y * n + x] = O.feq(0.0, U * math.sin(k * y), V * math.sin(k * x))
    assert s.observe()["residual"] == -1.0  # no snapshot yet
    t0, D = 300, 200
    s.run(t0)
    snap = s.fields()[0].copy()
    assert s.observe(snap)["residual"] == 0.0
    s.run(D)
    r = s.observe(snap)["residual"]
    expect = math.hypot(U, V) * math.exp(-nu * k * k * t0) * (1 - math.exp(-nu * k * k * D))
    assert r == pytest.approx(expect, rel=2e-2)


def test_advected_temperature_wave():
    """The advective term of Eq. 12, T_i^eq = (T/4)(1 + 2 e_i.u): its first
    moment is T u, so in a uniform flow u0 a temperature wave translates at
    u0 and decays at theta k^2 (theta from Eq. 14).  The phase shift over the
    run is a quarter wave, so a sign error, a dropped factor 2 or a missing
    term each move it by at least pi/4."""
    n, tau_T, u0, A = 64, 0.8, 0.04, 0.1
    k = 2 * math.pi / n
    theta = (2 * tau_T - 1) / 4
    m = np.zeros((1, n), np.uint8)
    s = O.State(O.mask_geom(n, 1, 1, 1), O.make_params(tau=0.8, tau_T=tau_T), m)
    x = np.arange(n)
    T = 1.0 + A * np.sin(k * x)
    for c in range(n):
        s.f[:, c] = O.feq(0.0, u0, 0.0)
    EXT, EYT = np.array([1, 0, -1, 0]), np.array([0, 1, 0, -1])
    s.T[:] = 0.25 * T[None, :] * (1 + 2 * (EXT[:, None] * u0 + EYT[:, None] * 0.0))

    def amp():
        _, _, Tf = s.fields()
        return np.sum((Tf - 1.0) * np.exp(-1j * k * x))

    s.run(100)
    a1 = amp()
    t = 400  # u0 t = 16 cells: a quarter wave
    s.run(t)
    a2 = amp()
    shift = -np.angle(a2 / a1)
    assert shift == pytest.approx(k * u0 * t, rel=1e-2)
    rate = -math.log(abs(a2 / a1)) / (t * k * k)
    assert rate == pytest.approx(theta, rel=2e-2)
    u, _, _ = s.fields()
    assert np.abs(u[0] - u0).max() < 1e-15 and np.abs(u[1]).max() < 1e-15


def test_thermal_inlet_and_outlet_rules_still_column():
    """Thermal boundary rules with no flow: the inlet holds T_in at its
    half link (anti-bounce-back, -T* + T_in/2) and the outlet has zero
    gradient (-T* + T(x)/2, the cell's own T).  From T = 0 the deficit
    T_in - T of a column of L cells then decays in the slowest mode of a
    Dirichlet-Neumann slab, sin(pi xi / 2L) e^{-theta (pi/2L)^2 t} with xi the
    distance from the inlet's half link.  An outlet that held a fixed
    temperature would decay four times faster in sin(pi xi / L)."""
    L, tau_T = 32, 1.0
    theta = (2 * tau_T - 1) / 4
    m, d = W.darcy_column(L, 0, 0, 1)
    g = O.mask_geom(d["nx"], d["ny"], d["periodic_x"], d["periodic_y"], d["inlet_dir"],
                    d["inlet_profile"], d["inlet_lo"], d["inlet_width"])
    P = O.make_params(tau=0.8, tau_T=tau_T, T_in=1.0, T_hot=0.3, T_cold=0.6, T0=0.0)
    s = O.State(g, P, m)
    xi = np.arange(1, L + 1) - 0.5

    def deficit():
        return 1.0 - s.fields()[2][1:L + 1]

    s.run(3000)
    w1 = deficit()
    s.run(2000)
    w2 = deficit()
    lam = -math.log(w2.max() / w1.max()) / 2000
    assert lam == pytest.approx(theta * (math.pi / (2 * L)) ** 2, rel=2e-2)
    shape = np.sin(math.pi * xi / (2 * L))
    assert np.abs(w2 / w2.max() - shape).max() < 1e-2
    assert np.argmax(w2) == L - 1  # the deficit peaks at the outlet end


def test_thermal_inlet_and_outlet_rules_through_flow():
    """Plug inflow at T_in through a column to the pressure outlet: the
    uniform state f = feq(p_out, u_in), T_i = (T_in/4)(1 + 2 e_i.u_in) is a
    fixed point of the inlet rule (moving-wall bounce-back and -T* + T_in/2),
    the bulk and the outlet rules (pressure anti-bounce-back and the
    zero-gradient -T* + T(x)/2), so the column settles at T = T_in exactly.
    An outlet that bounced heat back, or an inlet that imposed another
    temperature, would not."""
    m, d = W.darcy_column(24, 0, 8, 1)
    g = O.mask_geom(d["nx"], d["ny"], d["periodic_x"], d["periodic_y"], d["inlet_dir"],
                    d["inlet_profile"], d["inlet_lo"], d["inlet_width"])
    P = O.make_params(tau=0.8, tau_T=0.9, T_in=0.7, T_hot=1.0, T_cold=0.0, T0=0.2,
                      u_in_max=0.02)
    s = O.State(g, P, m)
    s.run(40000)
    u, p, T = s.fields()
    act = m.reshape(-1) <= O.POROUS
    assert np.abs(T[act] - 0.7).max() < 1e-12
    assert np.abs(u[0][act] - 0.02).max() < 1e-12
    assert np.abs(p[act]).max() < 1e-12


def _sector_mask(nx, ny, xc, yc, r, deg_lo, deg_hi):
    """Fluid box with cold cells beyond radius r of (xc, yc) inside the
    angular sector [deg_lo, deg_hi]: a curved wall whose angles have no
    symmetry axis; the cold wall's normal is radial from (xc, yc)."""
    m = np.full((ny, nx), W.FLUID, dtype=np.uint8)
    for y in range(ny):
        for x in range(nx):
            th = math.degrees(math.atan2(y - yc, x - xc))
            if math.hypot(x - xc, y - yc) > r and deg_lo <= th <= deg_hi:
                m[y, x] = W.COLD
    g = O.mask_geom(nx, ny, arc=(xc, yc, r))
    g.eye_normals = 1
    return m, g


@pytest.mark.parametrize("geometry", ["eye", "sector"])
def test_curved_wall_shear_normal_closed_form(geometry):
    """Wall shear on the analytic eye's curved cornea and on the iris.  Every
    active cell holds f = feq(0, 0) + w_i 4.5 (e_i e_i - I/3) : Pi with a
    uniform traceless Pi = [[-q, s], [s, q]]: then sum_i e_i e_i (f_i - feq_i)
    = Pi, and p = 0, u = 0.  For a wall of unit normal n at angle theta the
    shear t.sigma.n with sigma = -(1 - 1/(2 tau)) Pi is, by the double-angle
    identities, (1 - 1/(2 tau)) |q sin 2 theta + s cos 2 theta|.  The cornea's
    normal points from the arc's centre to the cell, so each adjacent fluid
    cell contributes at its own angle; the iris's normal is +y (theta = 90
    deg), so every iris cell contributes (1 - 1/(2 tau)) |s|.  q and s both
    non-zero tell a normal from its mirror image (components swapped) on the
    sector, whose angles (10 to 50 deg) have no symmetry axis; on the eye the
    cornea is symmetric about its axis, which hides that mirror but not a
    wrong centre or length."""
    tau = 0.8
    if geometry == "eye":
        nx, ny = 160, 80
        m, g = O.eye_mask(nx, ny, 45.0)
    else:
        nx, ny = 96, 96
        m, g = _sector_mask(nx, ny, 20.5, 15.5, 40.0, 10.0, 50.0)
    st = O.State(g, O.make_params(tau=tau), m)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    q, s = 3e-4, 5e-4
    pxx, pxy, pyy = -q, s, q
    fneq = 4.5 * w * ((EX * EX - 1 / 3) * pxx + 2 * EX * EY * pxy + (EY * EY - 1 / 3) * pyy)
    f9 = O.feq(0.0, 0.0, 0.0) + fneq
    mask = m.reshape(-1)
    act = mask <= W.POROUS
    st.f[:, act] = f9[:, None]
    obs = st.observe()

    k = 1.0 - 1.0 / (2.0 * tau)
    grid = m.reshape(ny, nx)
    cornea, iris = [], []
    for y in range(ny):
        for x in range(nx):
            if grid[y, x] != W.FLUID:
                continue
            nb = [grid[y + dy, x + dx] for dx in (-1, 0, 1) for dy in (-1, 0, 1)
                  if (dx or dy) and 0 <= x + dx < nx and 0 <= y + dy < ny]
            if W.COLD in nb:
                th = math.atan2(y - g.arc_yc, x - g.arc_xc)
                cornea.append(k * abs(q * math.sin(2 * th) + s * math.cos(2 * th)))
            if W.HOT in nb:
                iris.append(k * abs(s))
    assert len(cornea) > 20 and (len(iris) > 20 or geometry == "sector")
    assert obs["n_cornea"] == len(cornea) and obs["n_iris"] == len(iris)
    assert obs["wss_cornea"] == pytest.approx(np.mean(cornea), rel=1e-12)
    if iris:
        assert obs["wss_iris"] == pytest.approx(np.mean(iris), rel=1e-12)
    # the state is at rest: the other observables see no flow
    assert obs["peak"] == pytest.approx(0.0, abs=1e-15)
