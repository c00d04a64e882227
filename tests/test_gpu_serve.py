"""Continuous-batching server: each request's result is the same alone and
in the mix (bitwise: members are independent and folded per member), memory
stays within the HBM budget, and the one-at-a-time baseline completes."""
import pytest

from paper_2102_12663_gb300 import lbm, serve
from paper_2102_12663_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm.load(build_if_missing=True)


def small_requests(n=6, seed=21):
    draws = W.request_stream(n, seed=seed, ny_lo=64, ny_hi=128, fp16_share=0.5)
    return serve.requests_from_draws(draws)


def test_each_result_same_alone_and_in_mix():
    reqs = small_requests()
    assert {r.precision for r in reqs} == {"f32", "f16"}
    srv = serve.Server(budget_bytes=4e9, tol=1e-14, check_every=100, max_steps=600)
    mixed = {r.id: r for r in srv.run(reqs, realtime=False)}
    srv.close()
    assert len(mixed) == len(reqs)
    for q in small_requests():
        one = serve.Server(budget_bytes=4e9, tol=1e-14, check_every=100, max_steps=600)
        (res,) = one.run([q], realtime=False)
        one.close()
        m = mixed[q.id]
        assert res.steps == m.steps == 600
        assert res.observables == m.observables, q.id


def test_admission_respects_budget_and_finishes_all():
    reqs = small_requests(8, seed=4)
    sizes = [serve.domain_bytes(r) for r in reqs]
    budget = max(sizes) * 2.5
    srv = serve.Server(budget_bytes=budget, tol=1e-14, check_every=50, max_steps=200)
    res = srv.run(reqs, realtime=False)
    srv.close()
    assert len(res) == len(reqs)
    assert srv.peak_used <= budget
    assert all(r.steps == 200 and not r.unstable for r in res)
    s = serve.summary(res, srv.wall_s)
    assert s["solves"] == 8 and s["p99_s"] >= s["p50_s"] > 0


def test_steady_requests_retire_on_convergence():
    """Flowing requests (inflow on, buoyancy on, small grids) retire when their
    residual falls below their storage's tolerance (FP32 1e-7, FP16 1e-5 per
    100 steps), well before the cap of 20 decay times of their slowest viscous
    mode.  Each served result is compared with an FP64 solve of its request
    under the same stopping rule, which separates the storage's effect from
    the criterion's own truncation (the velocity residual falls below the
    tolerance while the temperature field still relaxes): FP32 within 1e-4
    (one interval of drift at 1e-7 plus FP32 rounding), FP16 within 1e-2 (its
    1e-5 stop lies in the transient, where one interval moves the wall shear by
    about 1e-3)."""
    draws = W.request_stream(4, seed=7, ny_lo=48, ny_hi=64, fp16_share=0.5)
    reqs = serve.requests_from_draws(draws, tol_by_precision=W.SERVE_TOL, cap_efolds=20.0)
    assert {r.precision for r in reqs} == {"f32", "f16"}
    assert all(r.params["u_in_max"] > 0.0 for r in reqs)
    srv = serve.Server(budget_bytes=4e9, check_every=100, max_steps=10**9)
    res = {r.id: r for r in srv.run(reqs, realtime=False)}
    srv.close()
    for q in reqs:
        r = res[q.id]
        assert r.converged and not r.unstable and r.steps < q.max_steps, (q.id, r.steps, q.max_steps)
        dom = lbm.Domain(dict(nx=q.nx, ny=q.ny, angle_deg=q.angle_deg), precision="f64")
        dom.set_params(q.params)
        st, _ = dom.run_to_steady(q.tol, check_every=100, max_steps=q.max_steps)
        assert st == lbm.OK
        ref = dom.last_observables()
        dom.close()
        bound = 1e-4 if q.precision == "f32" else 1e-2
        for k in ("iop", "wss_cornea", "wss_iris"):
            assert abs(r.observables[k] - ref[k]) <= bound * abs(ref[k]), (q.id, q.precision, k)


def test_one_at_a_time_baseline():
    reqs = [r for r in small_requests(4, seed=2)]
    res = serve.solve_one_at_a_time(reqs, tol=1e-14, check_every=100, max_steps=300,
                                    realtime=False)
    assert len(res) == 4 and all(r.steps == 300 for r in res)


def test_refined_fp16_requests_reach_the_fp32_criterion():
    """With refinement, an FP16 request that meets its own tolerance moves to
    the FP32 batch and retires at the FP32 criterion: its result then agrees
    with an FP64 solve of the request under that criterion as closely as a
    plain FP32 request's does (1e-4), and the FP16 phase took part of its
    steps."""
    draws = W.request_stream(4, seed=7, ny_lo=48, ny_hi=64, fp16_share=0.5)
    reqs = serve.requests_from_draws(draws, tol_by_precision=W.SERVE_TOL, cap_efolds=20.0)
    srv = serve.Server(budget_bytes=4e9, check_every=100, max_steps=10**9,
                       refine_tol={"f16": W.SERVE_TOL["f32"]})
    res = {r.id: r for r in srv.run(reqs, realtime=False)}
    srv.close()
    for q in reqs:
        r = res[q.id]
        assert r.converged and not r.unstable and r.steps < q.max_steps
        if q.precision == "f16":
            assert 0 < r.refined_steps < r.steps
        dom = lbm.Domain(dict(nx=q.nx, ny=q.ny, angle_deg=q.angle_deg), precision="f64")
        dom.set_params(q.params)
        st, _ = dom.run_to_steady(W.SERVE_TOL["f32"], check_every=100, max_steps=q.max_steps)
        assert st == lbm.OK
        ref = dom.last_observables()
        dom.close()
        for k in ("iop", "wss_cornea", "wss_iris"):
            assert abs(r.observables[k] - ref[k]) <= 1e-4 * abs(ref[k]), (q.id, q.precision, k)
