"""Serving several simulations at once (continuous batching): each result is the same alone
and in the mix; admission follows the HBM budget; latency percentiles are reported."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2311_05170_gb300 import build
    build.build()
    from paper_2311_05170_gb300 import native as N
    return N


def _alone(native, w, nsteps):
    s = native.Solver(w, precision="fp32")
    s.step(nsteps)
    f = s.fields()
    s.close()
    return f


def test_results_equal_alone_and_in_the_mix(native):
    from paper_2311_05170_gb300.serve import run_serving
    reqs = W.serving_requests_small(n=6, nsteps=4)
    stats, done = run_serving(reqs, hbm_budget_bytes=8 << 30, keep_fields=True, background=False)
    assert stats["requests"] == 6 and stats["max_concurrency"] >= 2
    assert stats["step_latency_ms_p50"] is not None and stats["step_latency_ms_p99"] >= stats["step_latency_ms_p50"]
    # a request's own step time is positive and within the tick that carried it
    assert all(x > 0 for r in done for x in r.latencies_ms)
    assert stats["step_latency_ms_p99"] <= stats["tick_ms_p99"] + 1.0
    for r in done:
        ref = _alone(native, r.w, r.nsteps)
        for k in ref:
            rel = np.linalg.norm(r.fields[k] - ref[k]) / np.linalg.norm(ref[k])
            assert rel <= 1e-12, (r.rid, k, rel)


def test_admission_by_hbm_budget(native):
    """With a budget smaller than the three simulations together some of them wait (they are
    refused with TPNS_EBUDGET until memory is released) and still finish with the same results."""
    from paper_2311_05170_gb300.serve import run_serving
    reqs = W.serving_requests_small(n=3, nsteps=2)
    sizes = []
    for _, w, _ in reqs:
        s = native.Solver(w, precision="fp32")
        sizes.append(s.stats()["device_bytes"])
        s.close()
    # all arrive at once; the budget holds the largest one, never all three
    budget = max(sizes) + 1
    assert sum(sizes) > budget
    stats, done = run_serving(reqs, hbm_budget_bytes=budget, keep_fields=True, time_scale=0.0)
    assert stats["requests"] == 3
    assert stats["refused_for_budget"] > 0
    for r in done:
        ref = _alone(native, r.w, r.nsteps)
        for k in ref:
            assert np.linalg.norm(r.fields[k] - ref[k]) <= 1e-12 * np.linalg.norm(ref[k])


def test_batch_step_matches_individual_steps(native):
    ws = [w for _, w, _ in W.serving_requests_small(n=3, nsteps=3)]
    batch = [native.Solver(w, precision="fp32") for w in ws]
    for _ in range(3):
        native.batch_step(batch)
    for s, w in zip(batch, ws):
        ref = _alone(native, w, 3)
        f = s.fields()
        for k in ref:
            assert np.array_equal(f[k], ref[k]), k
        s.close()


def test_served_results_match_the_oracle(native):
    """A seeded sample of served requests (different mesh sizes and parameters, run in the mix)
    meets the mixed-precision tolerance against the CPU oracle run alone."""
    from oracle.scheme import TwoGridOracle
    from paper_2311_05170_gb300.serve import run_serving
    reqs = W.serving_requests_small(n=4, nsteps=3)
    stats, done = run_serving(reqs, hbm_budget_bytes=8 << 30, keep_fields=True)
    assert stats["requests"] == 4
    for r in done[:2]:
        o = TwoGridOracle(r.w)
        o.run(r.nsteps)
        for k in o.fine:
            rel = np.linalg.norm(r.fields[k] - o.fine[k]) / np.linalg.norm(o.fine[k])
            assert rel <= 1e-8, (r.rid, k, rel)
    # the observed latency (from the step's readiness to the end of its tick) is at least the
    # device time of the step
    assert stats["observed_step_latency_ms_p50"] >= stats["step_latency_ms_p50"] * 0.5
    assert all(len(r.observed_ms) == r.nsteps for r in done)


def test_background_admission_results_equal_alone(native):
    """Contexts created by the background thread while others step (all requests arrive at
    once) give the same results as the same simulations run alone."""
    from paper_2311_05170_gb300.serve import run_serving
    reqs = W.serving_requests_small(n=4, nsteps=3)
    stats, done = run_serving(reqs, hbm_budget_bytes=8 << 30, keep_fields=True, time_scale=0.0)
    assert stats["requests"] == 4
    for r in done:
        ref = _alone(native, r.w, r.nsteps)
        for k in ref:
            rel = np.linalg.norm(r.fields[k] - ref[k]) / np.linalg.norm(ref[k])
            assert rel <= 1e-12, (r.rid, k, rel)
