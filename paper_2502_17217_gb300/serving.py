"""Solve-request server on one GPU: continuous admission by HBM footprint.

Requests (a mesh + boundary conditions + material, and a number of load steps) arrive at any
time and queue in arrival order.  Two ways of putting them on the device:

  * mode "contexts" (default): a queued request is admitted as soon as a slot is free and its
    device footprint fits the memory budget; it gets its own context (mesh, state, Krylov
    basis and preconditioner resident on the device for its whole life) and its own CUDA
    stream, and runs its Newton-Krylov solve in a slot worker.  Requests admitted while
    others run overlap with them on the device, kernel by kernel; each starts as soon as it is
    admitted and retires as soon as it converges.  With setup_ahead = A > 0, up to A more
    requests are admitted while every slot is busy: their contexts are created and set up
    (topology, renumbering, aggregation and Galerkin products on the host, uploads and device
    geometry) while the slots solve, and each takes the next free slot as soon as it is ready,
    so that a queued request's set-up is off its critical path.
  * mode "lockstep": when a batch slot is free, the queued requests with the head request's
    number of load steps that fit the budget are concatenated into one batch (one index space,
    one iteration graph for all of them, each problem with its own Newton loop and Krylov
    scalars) and solved together; requests that arrive meanwhile wait for the next batch.

A request's arithmetic never depends on the others (separate contexts, or per-problem scalars
in a batch), so its result is the same alone and in the mix.  Latency is completion time minus
arrival time (queueing, set-up and solve).

The footprint of a request is estimated as bytes-per-cell x cells; the server starts from a
conservative figure per law and replaces it with the largest measured ratio
(jfnk_device_bytes / cells) of the requests it has run.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import jfnk

DEFAULT_BYTES_PER_CELL = {0: 2400.0, 1: 3200.0, 2: 3200.0}  # Hooke, neo-Hookean, St. Venant-Kirchhoff; refined by measurement


@dataclass
class Request:
    case: object
    load_steps: int = 1
    t_arrival: float = 0.0
    tag: object = None
    # filled by the server
    t_admit: float = 0.0
    t_done: float = 0.0
    u: np.ndarray | None = None
    status: int = 0
    stats: object = None
    bytes: int = 0
    t_setup: float = 0.0  # seconds of context creation and set-up (host work and uploads)
    t_wait: float = 0.0   # seconds set up and waiting for a solve slot (setup_ahead > 0)
    t_solve: float = 0.0  # seconds of the solve call
    error: str | None = None
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival

    @property
    def cells(self) -> int:
        return self.case.mesh.n_cells


class Server:
    """Continuous-admission JFNK solve server (one GPU).  mode "contexts": one context and
    stream per request, up to max_slots solving at once and up to setup_ahead more being set
    up or ready; mode "lockstep": batches of queued requests, up to max_slots batches at once."""

    MODES = ("contexts", "lockstep")

    def __init__(self, device: int = 0, hbm_budget_bytes: float | None = None, max_slots: int = 8,
                 mode: str = "contexts", setup_ahead: int = 0, **options):
        if mode not in self.MODES:
            raise ValueError(f"mode must be one of {self.MODES}")
        if setup_ahead < 0 or (setup_ahead and mode != "contexts"):
            raise ValueError("setup_ahead must be >= 0, and is for mode 'contexts' only")
        self.device = device
        self.mode = mode
        self.setup_ahead = setup_ahead
        self._slots = threading.BoundedSemaphore(max_slots)  # solves at once (mode 'contexts')
        self.options = dict(options)
        # a served request is solved once: the launch-shape autotuner's timing runs would cost
        # more than they save (the shapes never change the results)
        self.options.setdefault("autotune", 0)
        self.max_slots = max_slots
        if hbm_budget_bytes is None:
            import torch
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget_bytes = 0.8 * free
        self.budget = float(hbm_budget_bytes)
        self.bpc = dict(DEFAULT_BYTES_PER_CELL)
        self._queue: collections.deque[Request] = collections.deque()
        self._lock = threading.Condition()
        self._in_use = 0.0
        self._running = 0   # workers (requests holding a context, or batches in lockstep mode)
        self._inflight = 0  # requests on the device
        self._solving = 0   # requests in their solve (mode 'contexts')
        self.max_solving = 0
        self._stop = False
        self._workers: list[threading.Thread] = []
        self.completed: list[Request] = []
        self.max_concurrent = 0
        self.max_shared_footprint = 0.0  # largest admitted footprint total with > 1 request running
        self._dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self._dispatcher.start()

    # ---------------------------------------------------------------- client side
    def submit(self, case, load_steps: int = 1, tag=None) -> Request:
        r = Request(case=case, load_steps=load_steps, t_arrival=time.perf_counter(), tag=tag)
        with self._lock:
            self._queue.append(r)
            self._lock.notify_all()
        return r

    def drain(self):
        """Waits until every submitted request has completed."""
        with self._lock:
            while self._queue or self._running:
                self._lock.wait(0.05)

    def close(self):
        self.drain()
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        self._dispatcher.join()
        for w in self._workers:
            w.join()

    # ---------------------------------------------------------------- server side
    def footprint(self, case) -> float:
        return self.bpc[case.material.law] * case.mesh.n_cells

    def _dispatch(self):
        while True:
            with self._lock:
                while not self._stop and not self._admissible():
                    self._lock.wait(0.01)
                if self._stop and not self._queue:
                    return
                if not self._admissible():
                    continue
                group = [self._queue.popleft()]
                need = self.footprint(group[0].case)
                if self.mode == "lockstep":
                    # the queued requests with the head's load steps that still fit, in order
                    keep = collections.deque()
                    while self._queue:
                        q = self._queue.popleft()
                        nq = self.footprint(q.case)
                        if q.load_steps == group[0].load_steps and self._in_use + need + nq <= self.budget:
                            group.append(q)
                            need += nq
                        else:
                            keep.append(q)
                    self._queue = keep
                self._in_use += need
                self._running += 1
                self._inflight += len(group)
                self.max_concurrent = max(self.max_concurrent, self._inflight)
                if self._inflight > 1:
                    self.max_shared_footprint = max(self.max_shared_footprint, self._in_use)
                now = time.perf_counter()
                for r in group:
                    r.t_admit = now
            if self.mode == "lockstep":
                t = threading.Thread(target=self._work_batch, args=(group, need), daemon=True)
            else:
                t = threading.Thread(target=self._work, args=(group[0], need), daemon=True)
            self._workers = [w for w in self._workers if w.is_alive()]  # a long-lived server keeps no dead threads
            self._workers.append(t)
            t.start()

    def _admissible(self) -> bool:
        if not self._queue or self._running >= self.max_slots + self.setup_ahead:
            return False
        need = self.footprint(self._queue[0].case)
        # an oversized request runs alone rather than never
        return self._in_use + need <= self.budget or self._running == 0

    def _work(self, r: Request, need: float):
        s = None
        try:
            import torch
            torch.cuda.set_device(self.device)
            t0 = time.perf_counter()
            s = jfnk.Solver.from_case(r.case, device=self.device, **self.options)
            s.setup()
            t1 = time.perf_counter()
            with self._slots:  # the next free slot (at once unless set up ahead)
                ts = time.perf_counter()
                with self._lock:
                    self._solving += 1
                    self.max_solving = max(self.max_solving, self._solving)
                try:
                    u, st, rc = s.solve(load_steps=r.load_steps, raise_on_fail=False)
                finally:
                    with self._lock:
                        self._solving -= 1
            r.t_setup, r.t_wait, r.t_solve = t1 - t0, ts - t1, time.perf_counter() - ts
            r.u, r.stats, r.status = u, st, rc
            r.bytes = s.device_bytes()
        except Exception as e:  # reported on the request, the server keeps serving
            r.error = f"{type(e).__name__}: {e}"
            r.status = -99
        finally:
            if s is not None:  # the request's device memory is released on every path
                try:
                    s.close()
                except Exception as e:
                    r.error = r.error or f"close: {type(e).__name__}: {e}"
        r.t_done = time.perf_counter()
        self._retire([r], need)

    def _retire(self, group, need: float):
        with self._lock:
            for r in group:
                if r.bytes:
                    law = r.case.material.law
                    self.bpc[law] = max(self.bpc[law] if law in self.bpc else 0.0, r.bytes / r.cells)
                self.completed.append(r)
            self._in_use -= need
            self._running -= 1
            self._inflight -= len(group)
            self._lock.notify_all()
        for r in group:
            r.done.set()

    def _work_batch(self, group, need: float):
        """Lockstep mode: the group solved as one batch; each request gets its own part of the
        solution, its own statistics and an equal share of the batch's device bytes."""
        b = None
        try:
            import torch
            torch.cuda.set_device(self.device)
            t0 = time.perf_counter()
            b = jfnk.Batch([r.case for r in group], device=self.device, **self.options)
            b.setup()
            t1 = time.perf_counter()
            u, st, rc = b.solve(load_steps=group[0].load_steps, raise_on_fail=False)
            t2 = time.perf_counter()
            per = b.problem_stats()
            total = b.device_bytes()
            cells = sum(r.cells for r in group)
            for r, uk, ps in zip(group, b.split(u), per):
                r.u, r.stats, r.status = np.array(uk), ps, ps.status
                r.t_setup, r.t_solve = t1 - t0, t2 - t1
                r.bytes = int(total * r.cells / max(1, cells))
        except Exception as e:  # reported on every request of the batch, the server keeps serving
            for r in group:
                r.error = f"{type(e).__name__}: {e}"
                r.status = -99
        finally:
            if b is not None:
                try:
                    b.close()
                except Exception as e:
                    for r in group:
                        r.error = r.error or f"close: {type(e).__name__}: {e}"
        now = time.perf_counter()
        for r in group:
            r.t_done = now
        self._retire(group, need)


def serve_stream(cases, rate_per_s: float, seed: int = 0, load_steps=None, **server_kw):
    """Submits `cases` with Poisson arrivals at `rate_per_s` (seeded exponential gaps) and
    returns (requests, wall time from the first arrival to the last completion, server)."""
    from .inputs import splitmix64_uniform
    gaps = -np.log(1.0 - splitmix64_uniform(seed, len(cases), key=77)) / rate_per_s
    srv = Server(**server_kw)
    reqs = []
    t0 = time.perf_counter()
    t_next = t0
    for k, case in enumerate(cases):
        t_next += gaps[k]
        while True:
            now = time.perf_counter()
            if now >= t_next:
                break
            time.sleep(min(0.002, t_next - now))
        steps = load_steps[k] if load_steps is not None else 1
        reqs.append(srv.submit(case, load_steps=steps, tag=k))
    srv.drain()
    wall = max(r.t_done for r in reqs) - reqs[0].t_arrival
    srv.close()
    return reqs, wall, srv


def summarize(reqs, wall):
    lat = np.array([r.latency for r in reqs])
    ok = sum(1 for r in reqs if r.status == 0)
    return {"requests": len(reqs), "converged": ok, "solves_per_s": len(reqs) / wall, "wall_s": wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "cells_total": int(sum(r.cells for r in reqs))}
