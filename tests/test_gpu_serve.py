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
    """A request that reaches the residual tolerance leaves before the cap."""
    reqs = small_requests(2, seed=9)
    for r in reqs:
        r.params = dict(r.params, g_beta=0.0, T_hot=0.0, T_in=0.0, T0=0.0, noise_amp=0.0,
                        u_in_max=0.0)
    srv = serve.Server(budget_bytes=4e9, tol=1e-9, check_every=100, max_steps=5000)
    res = srv.run(reqs, realtime=False)
    srv.close()
    assert all(r.converged and r.steps < 5000 for r in res)


def test_one_at_a_time_baseline():
    reqs = [r for r in small_requests(4, seed=2)]
    res = serve.solve_one_at_a_time(reqs, tol=1e-14, check_every=100, max_steps=300,
                                    realtime=False)
    assert len(res) == 4 and all(r.steps == 300 for r in res)
