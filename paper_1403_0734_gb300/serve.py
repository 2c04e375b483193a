"""Continuous-batching request loop over device-resident oriented graphs.

A request asks for an exact count (FFF_k) or a colour-sampled estimate
(cFFF_k, Sec. 6) on one of the resident graphs.  The server keeps `slots`
worker streams; a request is admitted, in arrival order, as soon as a slot
is free and its device footprint (kc_footprint) fits the memory budget next
to the requests already running -- it does not wait for the others to
finish, so the kernels of different requests overlap on the GPU.  Every
request's answer is exact and independent of what runs beside it (each call
has its own stream-ordered scratch).

The work of a request is one C-ABI call (kc_count / kc_estimate on the
request's stream); this module only orders, admits and times requests.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


class RequestError(RuntimeError):
    """A request's backend call failed; `results` holds every request's
    Result (failed ones with their error)."""

    def __init__(self, rid: int, error: str, results):
        super().__init__(f"request {rid} failed: {error}")
        self.rid = rid
        self.results = results


@dataclass
class Request:
    rid: int
    graph: int          # index into the server's graph list
    k: int
    colours: int = 0    # 0: exact count; >= 1: estimate with that many colours
    seed: int = 0
    arrival: float = 0.0  # seconds after the start of the stream


@dataclass
class Result:
    rid: int
    value: int              # q_k, or the sampled count S of an estimate
    estimate: float         # S * c^(k-2) for estimates, float(q_k) otherwise
    arrival: float
    start: float
    end: float
    error: str | None = None  # the backend's exception, if the request failed

    @property
    def latency(self) -> float:
        return self.end - self.arrival


def poisson_stream(num: int, rate: float, ngraphs: int, seed: int, kmin: int = 3, kmax: int = 6,
                   cmin: int = 2, cmax: int = 16, frac_exact: float = 0.5):
    """A seeded request stream: exponential inter-arrival times at `rate`
    requests/s, uniform graph, k uniform in [kmin, kmax], exact or sampled
    with probability frac_exact, colours uniform in [cmin, cmax], seed = id."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=num)) if rate > 0 else np.zeros(num)
    reqs = []
    for i in range(num):
        exact = rng.random() < frac_exact
        reqs.append(Request(i, int(rng.integers(ngraphs)), int(rng.integers(kmin, kmax + 1)),
                            0 if exact else int(rng.integers(cmin, cmax + 1)), i, float(t[i])))
    return reqs


class Server:
    """slots worker streams, FIFO admission under a device-memory budget."""

    def __init__(self, graphs, slots: int = 4, budget_bytes: int | None = None, backend=None,
                 footprint=None):
        self.graphs = graphs
        self.slots = slots
        self.budget = budget_bytes
        self._backend = backend or self._gpu_backend
        self._footprint = footprint or self._gpu_footprint
        self._cv = threading.Condition()
        self._queue: deque = deque()
        self._in_use = 0
        self._free_slots = slots
        self._results: list[Result] = []
        self._done = 0
        self._t0 = 0.0
        self._closing = False
        self.max_concurrent = 0
        self._running = 0

    # -- GPU backend: one C-ABI call on the slot's stream ---------------------
    def _gpu_footprint(self, req: Request) -> int:
        from . import kc
        return kc.footprint(self.graphs[req.graph], req.k)

    def _gpu_backend(self, req: Request, stream):
        from . import kc
        g = self.graphs[req.graph]
        if req.colours:
            s, est, _ = kc.estimate(g, req.k, req.colours, req.seed, stream=stream)
            return s, est
        q = kc.count(g, req.k, stream=stream)[0]
        return q, float(q)

    # -- loop ------------------------------------------------------------------
    def _now(self) -> float:
        return time.perf_counter() - self._t0

    def _worker(self, slot: int, stream_factory):
        stream = stream_factory() if stream_factory else None
        while True:
            with self._cv:
                while True:
                    if self._queue:
                        req, fp = self._queue[0]
                        fits = self.budget is None or self._in_use + fp <= self.budget or self._running == 0
                        if fits:
                            self._queue.popleft()
                            self._in_use += fp
                            self._running += 1
                            self.max_concurrent = max(self.max_concurrent, self._running)
                            break
                    elif self._closing:
                        return
                    self._cv.wait()
            start = self._now()
            value, est, err = 0, float("nan"), None
            try:
                value, est = self._backend(req, stream)
            except Exception as e:  # recorded per request; run() raises after the rest finish
                err = f"{type(e).__name__}: {e}"
            finally:
                end = self._now()
                with self._cv:  # the slot, its footprint and the request are always released
                    self._in_use -= fp
                    self._running -= 1
                    self._results.append(Result(req.rid, int(value), float(est), req.arrival, start, end, err))
                    self._done += 1
                    self._cv.notify_all()

    def run(self, requests, stream_factory=None, realtime: bool = True, raise_errors: bool = True):
        """Serve `requests` (arrival times relative to the start); returns the
        results ordered by request id and the makespan in seconds.  A request
        whose backend call raised still completes (its Result carries the
        error) and does not hold up the others; with raise_errors, run()
        raises RequestError for the first failed request once every request
        has finished."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        fps = [self._footprint(r) for r in reqs]
        if self.budget is not None and any(fp > self.budget for fp in fps):
            raise ValueError("a request needs more device memory than the budget")
        self._results, self._done, self._closing = [], 0, False
        self._t0 = time.perf_counter()
        workers = [threading.Thread(target=self._worker, args=(i, stream_factory), daemon=True)
                   for i in range(self.slots)]
        for w in workers:
            w.start()
        for r, fp in zip(reqs, fps):
            if realtime:
                delay = r.arrival - self._now()
                if delay > 0:
                    time.sleep(delay)
            with self._cv:
                self._queue.append((r, fp))
                self._cv.notify_all()
        with self._cv:
            self._closing = True
            self._cv.notify_all()
            while self._done < len(reqs):
                self._cv.wait()
        makespan = self._now()
        for w in workers:
            w.join()
        results = sorted(self._results, key=lambda x: x.rid)
        failed = [r for r in results if r.error is not None]
        if raise_errors and failed:
            raise RequestError(failed[0].rid, failed[0].error, results)
        return results, makespan


def latency_stats(results):
    lat = np.array([r.latency for r in results]) if results else np.zeros(1)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
