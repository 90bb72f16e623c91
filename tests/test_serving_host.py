"""Host-side logic of the solve server (no GPU): admission in arrival order by estimated HBM
footprint, the slot limit, an oversized request running alone, refinement of the
bytes-per-cell estimate from measured footprints, a failing request reported on the request
while the others are served, and the Poisson-arrival driver with its latency summary.  The
per-request solver is replaced by a fake that sleeps and records how many requests were
live at once and in which order they were set up."""
import threading
import time
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2502_17217_gb300 import serving


class _Live:
    def __init__(self):
        self.lock = threading.Lock()
        self.n = 0
        self.max_n = 0
        self.solving = 0
        self.max_solving = 0
        self.order = []
        self.events = []  # (time, "setup-start" | "setup-end" | "solve-start" | "solve-end", tag)
        self.closed = 0


def _case(cells, law=0, hold=0.05, fail=False, true_bpc=None, setup_hold=0.0, tag=None):
    return SimpleNamespace(mesh=SimpleNamespace(n_cells=cells), material=SimpleNamespace(law=law),
                           hold=hold, fail=fail, true_bpc=true_bpc, setup_hold=setup_hold, tag=tag)


@pytest.fixture
def live(monkeypatch):
    rec = _Live()

    class FakeSolver:
        def __init__(self, case):
            self.case = case

        @classmethod
        def from_case(cls, case, **kw):
            return cls(case)

        def setup(self):
            with rec.lock:
                rec.n += 1
                rec.max_n = max(rec.max_n, rec.n)
                rec.order.append(id(self.case))
                rec.events.append((time.perf_counter(), "setup-start", self.case.tag))
            time.sleep(self.case.setup_hold)
            with rec.lock:
                rec.events.append((time.perf_counter(), "setup-end", self.case.tag))

        def solve(self, load_steps=1, raise_on_fail=True):
            with rec.lock:
                rec.solving += 1
                rec.max_solving = max(rec.max_solving, rec.solving)
                rec.events.append((time.perf_counter(), "solve-start", self.case.tag))
            try:
                time.sleep(self.case.hold)
                if self.case.fail:
                    raise RuntimeError("planted solve failure")
                st = SimpleNamespace(load_steps=load_steps)
                return np.zeros((self.case.mesh.n_cells, 3)), st, 0
            finally:
                with rec.lock:
                    rec.n -= 1
                    rec.solving -= 1
                    rec.events.append((time.perf_counter(), "solve-end", self.case.tag))

        def device_bytes(self):
            bpc = self.case.true_bpc
            return int(bpc * self.case.mesh.n_cells) if bpc else 0

        def close(self):
            with rec.lock:
                rec.closed += 1

    monkeypatch.setattr(serving.jfnk, "Solver", FakeSolver)
    import torch
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    return rec


def _run(cases, **kw):
    srv = serving.Server(**kw)
    reqs = [srv.submit(c, tag=k) for k, c in enumerate(cases)]
    srv.drain()
    srv.close()
    return srv, reqs


def test_admission_keeps_the_footprint_within_the_budget(live):
    one = serving.DEFAULT_BYTES_PER_CELL[0] * 1000
    srv, reqs = _run([_case(1000) for _ in range(8)], hbm_budget_bytes=2.5 * one, max_slots=8)
    assert all(r.status == 0 and r.error is None for r in reqs)
    assert srv.max_concurrent == 2 and live.max_n == 2
    assert srv.max_shared_footprint <= 2.5 * one
    assert srv._in_use == 0 and srv._running == 0


def test_slot_limit_caps_concurrency(live):
    srv, reqs = _run([_case(100, hold=0.1) for _ in range(10)], hbm_budget_bytes=1e15, max_slots=3)
    assert len(srv.completed) == 10
    assert srv.max_concurrent == 3 and live.max_n == 3


def test_oversized_request_runs_alone(live):
    srv, reqs = _run([_case(5000), _case(5000), _case(5000)], hbm_budget_bytes=1000.0, max_slots=8)
    assert all(r.status == 0 for r in reqs)
    assert srv.max_concurrent == 1 and live.max_n == 1


def test_admission_is_in_arrival_order(live):
    # A (small, long) runs; B needs the whole budget, so it waits for A; C (small) would fit
    # beside A but must not overtake B.
    bpc = serving.DEFAULT_BYTES_PER_CELL[0]
    a, b, c = _case(100, hold=0.3), _case(950, hold=0.05), _case(100, hold=0.05)
    srv, (ra, rb, rc) = _run([a, b, c], hbm_budget_bytes=1000 * bpc, max_slots=8)
    assert ra.t_admit <= rb.t_admit <= rc.t_admit
    assert rb.t_admit >= ra.t_done  # B started only once A released its footprint
    assert live.order == [id(a), id(b), id(c)]


def test_bytes_per_cell_estimate_grows_to_the_measured_footprint(live):
    srv, reqs = _run([_case(1000, law=1, true_bpc=5000.0), _case(1000, law=0, true_bpc=100.0)],
                     hbm_budget_bytes=1e12)
    assert srv.bpc[1] == pytest.approx(5000.0)
    # a measured figure below the conservative start does not lower it
    assert srv.bpc[0] == serving.DEFAULT_BYTES_PER_CELL[0]
    assert reqs[0].bytes == 5_000_000


def test_failing_request_is_reported_and_the_rest_are_served(live):
    cases = [_case(100), _case(100, fail=True), _case(100)]
    srv, reqs = _run(cases, hbm_budget_bytes=1e12, max_slots=2)
    assert reqs[1].status == -99 and "planted solve failure" in reqs[1].error
    assert reqs[0].status == 0 and reqs[2].status == 0
    assert srv._in_use == 0 and srv._running == 0
    assert all(r.done.is_set() for r in reqs)
    assert live.closed == 3  # the failed request's context is released too


def test_poisson_stream_and_latency_summary(live):
    cases = [_case(200, hold=0.02) for _ in range(12)]
    reqs, wall, srv = serving.serve_stream(cases, rate_per_s=200.0, seed=3, hbm_budget_bytes=1e12, max_slots=4)
    s = serving.summarize(reqs, wall)
    assert s["requests"] == 12 and s["converged"] == 12
    assert s["cells_total"] == 12 * 200
    lat = sorted(r.latency for r in reqs)
    assert min(lat) >= 0.02
    assert s["p50_latency_s"] <= s["p99_latency_s"] <= max(lat) + 1e-12
    assert s["solves_per_s"] == pytest.approx(12 / wall)
    # arrivals follow the seeded gaps: submission times are increasing
    t = [r.t_arrival for r in reqs]
    assert all(x < y for x, y in zip(t, t[1:]))


@pytest.fixture
def batches(monkeypatch):
    """A fake batch in place of jfnk.Batch: records each batch's requests, sleeps, returns a
    solution whose rows carry the problem's cell count (so each request's part can be checked)."""
    made = []

    class FakeBatch:
        def __init__(self, cases, **kw):
            self.cases = list(cases)
            self.sizes = [c.mesh.n_cells for c in self.cases]
            made.append(self)

        def setup(self):
            pass

        def solve(self, load_steps=1, raise_on_fail=True):
            time.sleep(max(c.hold for c in self.cases))
            if any(c.fail for c in self.cases):
                raise RuntimeError("planted batch failure")
            self.load_steps = load_steps
            u = np.concatenate([np.full((n, 3), float(n)) for n in self.sizes])
            return u, SimpleNamespace(), 0

        def problem_stats(self):
            return [SimpleNamespace(status=0, load_steps_done=self.load_steps) for _ in self.cases]

        def split(self, u):
            off = np.concatenate([[0], np.cumsum(self.sizes)])
            return [u[off[k]:off[k + 1]] for k in range(len(self.sizes))]

        def device_bytes(self):
            return 0

        def close(self):
            pass

    monkeypatch.setattr(serving.jfnk, "Batch", FakeBatch)
    import torch
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    return made


def test_lockstep_mode_groups_queued_requests_by_load_steps_and_budget(batches):
    """Requests queued while a batch runs form the next batch: only those with the head
    request's load steps, and only while their footprints fit the budget, in arrival order;
    each request receives its own part of the batch's solution."""
    bpc = serving.DEFAULT_BYTES_PER_CELL[0]
    srv = serving.Server(hbm_budget_bytes=1000 * bpc, max_slots=1, mode="lockstep")
    first = srv.submit(_case(100, hold=0.2))  # runs alone while the rest queue up
    time.sleep(0.05)
    rest = [srv.submit(_case(n, hold=0.01), load_steps=ls) for n, ls in
            [(200, 1), (300, 2), (250, 1), (600, 1), (150, 2)]]
    srv.drain()
    srv.close()
    groups = [[c.mesh.n_cells for c in b.cases] for b in batches]
    assert groups[0] == [100]
    # after the first batch: the head (200 cells, 1 step) with the next 1-step request that
    # fits (250); 600 would exceed the budget (200 + 250 + 600 > 1000 cells' worth)
    assert groups[1] == [200, 250]
    assert sorted(map(tuple, groups[2:])) == sorted([(300, 150), (600,)])
    for r in [first] + rest:
        assert r.status == 0 and np.all(r.u == r.cells)
    assert srv._in_use == 0 and srv._running == 0 and srv._inflight == 0


def test_lockstep_batch_failure_is_reported_on_each_of_its_requests(batches):
    srv = serving.Server(hbm_budget_bytes=1e15, max_slots=2, mode="lockstep")
    reqs = [srv.submit(_case(100, hold=0.05, fail=(k == 1))) for k in range(2)]
    srv.drain()
    srv.close()
    bad = [r for r in reqs if r.status == -99]
    assert bad and all("planted batch failure" in r.error for r in bad)
    assert all(r.done.is_set() for r in reqs)


def test_setup_ahead_prepares_queued_requests_while_the_slots_solve(live):
    """With setup_ahead = 2 and 2 slots, up to 4 requests hold a context (two solving, two
    set up and waiting), never more than 2 solve at once, every request is served, and a
    queued request's set-up starts before the solve ahead of it ends."""
    cases = [_case(100, hold=0.15, setup_hold=0.05, tag=k) for k in range(8)]
    srv, reqs = _run(cases, hbm_budget_bytes=1e15, max_slots=2, setup_ahead=2)
    assert all(r.status == 0 and r.error is None for r in reqs)
    assert live.max_solving == 2 and srv.max_solving == 2
    assert srv.max_concurrent == 4 and live.max_n == 4
    assert srv._in_use == 0 and srv._running == 0 and srv._solving == 0
    first = {}
    for t, what, tag in live.events:
        first.setdefault((what, tag), t)
    # request 2 (the first to wait) was set up while requests 0 and 1 were solving
    assert first[("setup-end", 2)] < first[("solve-end", 0)]
    # and a request waiting for its slot reports that wait
    assert max(r.t_wait for r in reqs) > 0.05


def test_setup_ahead_respects_the_memory_budget(live):
    one = serving.DEFAULT_BYTES_PER_CELL[0] * 1000
    srv, reqs = _run([_case(1000) for _ in range(6)], hbm_budget_bytes=2.5 * one, max_slots=1, setup_ahead=4)
    assert all(r.status == 0 for r in reqs)
    assert srv.max_concurrent == 2 and live.max_n == 2  # the budget, not the set-up allowance, bounds it
    assert srv.max_solving == 1


def test_setup_ahead_is_for_the_contexts_mode_only():
    with pytest.raises(ValueError):
        serving.Server(hbm_budget_bytes=1e12, mode="lockstep", setup_ahead=2)
    with pytest.raises(ValueError):
        serving.Server(hbm_budget_bytes=1e12, setup_ahead=-1)
