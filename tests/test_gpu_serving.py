"""Serving: continuous admission by HBM footprint, concurrent slots (GPU)."""
import numpy as np
import pytest

from paper_2502_17217_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def test_served_results_equal_alone_results_and_requests_overlap():
    from paper_2502_17217_gb300 import jfnk, serving
    reqs_def = I.serving_requests(8, lo=500, hi=4000, seed=9, frac_nh=0.4)
    opts = dict(pc=jfnk.PC_MG, precision=jfnk.PREC_MIXED, mg_coarse_max=50)
    cases = [c for c, _ in reqs_def]
    steps = [s for _, s in reqs_def]
    reqs, wall, srv = serving.serve_stream(cases, rate_per_s=500.0, seed=3, load_steps=steps, max_slots=4, **opts)
    bad = [(k, r.status, r.error, r.cells) for k, r in enumerate(reqs) if r.status != 0]
    assert not bad, bad
    assert srv.max_concurrent > 1  # requests ran concurrently
    for r, (c, st) in zip(reqs, reqs_def):
        ua, _, rc = jfnk.Solver.from_case(c, **opts).solve(load_steps=st)
        assert rc == 0
        assert np.array_equal(r.u, ua)  # the same alone and in the mix
    summ = serving.summarize(reqs, wall)
    assert summ["p99_latency_s"] >= summ["p50_latency_s"] > 0


def test_admission_respects_the_memory_budget():
    """Requests share the device only while their estimated footprints fit the budget; a
    request larger than the whole budget still runs, alone."""
    from paper_2502_17217_gb300 import jfnk, serving
    reqs_def = I.serving_requests(6, lo=1000, hi=3000, seed=10, frac_nh=0.0)
    budget = 2.5 * serving.DEFAULT_BYTES_PER_CELL[0] * 3000
    reqs, wall, srv = serving.serve_stream([c for c, _ in reqs_def], rate_per_s=1000.0, seed=4, max_slots=6,
                                           hbm_budget_bytes=budget, pc=jfnk.PC_BJACOBI)
    assert all(r.status == 0 for r in reqs)
    assert srv.max_shared_footprint <= budget
    # a budget smaller than any request: every request runs, one at a time
    reqs, wall, srv = serving.serve_stream([c for c, _ in reqs_def[:3]], rate_per_s=1000.0, seed=5, max_slots=6,
                                           hbm_budget_bytes=1.0, pc=jfnk.PC_BJACOBI)
    assert all(r.status == 0 for r in reqs) and srv.max_concurrent == 1


def test_served_results_under_contention_with_load_steps():
    """Many large requests in a burst (copy engines and SMs shared by 8 contexts), half of
    them neo-Hookean with two load steps: every result equals the request solved alone.  A
    load factor uploaded outside the request's stream order showed up here as requests
    converging to the wrong load step."""
    from paper_2502_17217_gb300 import jfnk, serving
    reqs_def = I.serving_requests(16, lo=20000, hi=200000, seed=11, frac_nh=0.5)
    opts = dict(pc=jfnk.PC_MG, precision=jfnk.PREC_MIXED)
    cases = [c for c, _ in reqs_def]
    steps = [s for _, s in reqs_def]
    reqs, wall, srv = serving.serve_stream(cases, rate_per_s=5000.0, seed=6, load_steps=steps, max_slots=8, **opts)
    assert srv.max_concurrent >= 4
    bad = [(k, r.status, r.error, r.cells) for k, r in enumerate(reqs) if r.status != 0]
    assert not bad, bad
    for r, (c, st) in zip(reqs, reqs_def):
        ua, sta, rc = jfnk.Solver.from_case(c, **opts).solve(load_steps=st)
        assert rc == 0 and sta.load_steps_done == st
        assert np.array_equal(r.u, ua)


@pytest.mark.parametrize("mode", ["contexts", "contexts_ahead", "lockstep"])
def test_served_results_match_the_oracle(mode):
    """Every served request (Poisson arrivals, Hooke and neo-Hookean with two load steps,
    mixed precision, multigrid) against the oracle's FP64 solve of that request, both to
    |R| <= 1e-10 |R0| per load step: relative difference <= 1e-8.  In lockstep mode the
    requests run as concatenated batches; in contexts mode each in its own context, with
    (contexts_ahead) or without queued requests set up while the slots solve."""
    import oracle as O
    from paper_2502_17217_gb300 import jfnk, serving
    reqs_def = I.serving_requests(8, lo=500, hi=4000, seed=9, frac_nh=0.4)
    opts = dict(pc=jfnk.PC_MG, precision=jfnk.PREC_MIXED, mg_coarse_max=50, newton_rtol=1e-10)
    cases = [c for c, _ in reqs_def]
    steps = [s for _, s in reqs_def]
    ahead = 4 if mode == "contexts_ahead" else 0
    reqs, wall, srv = serving.serve_stream(cases, rate_per_s=500.0, seed=3, load_steps=steps, max_slots=4,
                                           mode="lockstep" if mode == "lockstep" else "contexts", setup_ahead=ahead, **opts)
    bad = [(k, r.status, r.error, r.cells) for k, r in enumerate(reqs) if r.status != 0]
    assert not bad, bad
    if mode == "lockstep":
        assert srv.max_concurrent > 1  # some requests shared a batch
    for k, (r, (c, st)) in enumerate(zip(reqs, reqs_def)):
        o = O.Oracle.from_case(c)
        o.mg_setup(theta=0.4, coarse_max=50, smoothed=True, sweeps=2)
        uo, rco, _ = o.newton(load_steps=st, rtol=1e-10, pc=O.PC_MG, m=30, aug=2)
        assert rco == 0
        err = np.linalg.norm(r.u - uo) / np.linalg.norm(uo)
        assert err <= 1e-8, (k, mode, c.name, err)
