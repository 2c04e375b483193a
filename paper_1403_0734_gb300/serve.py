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

    @property
    def wait(self) -> float:
        return self.start - self.arrival

    @property
    def service(self) -> float:
        return self.end - self.start


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


class CostModel:
    """Online estimate of a request's service time, per request type (graph,
    k, exact or sampled): the mean of the types' observed times, or before
    any observation a prior proportional to the graph's edges times a
    per-k factor learned from all types."""

    def __init__(self, edges):
        self.edges = list(edges)
        self.obs: dict = {}
        self.per_edge: dict = {}

    @staticmethod
    def _type(req):
        return (req.graph, req.k, req.colours > 0)

    def estimate(self, req) -> float:
        o = self.obs.get(self._type(req))
        if o:
            return o[0] / o[1]
        pe = self.per_edge.get(req.k)
        if pe:
            return pe[0] / pe[1] * self.edges[req.graph]
        return 1e-3 * (1 + self.edges[req.graph] / 1e6) * req.k

    def observe(self, req, seconds: float):
        t = self._type(req)
        o = self.obs.setdefault(t, [0.0, 0])
        o[0] += seconds
        o[1] += 1
        pe = self.per_edge.setdefault(req.k, [0.0, 0.0])
        pe[0] += seconds
        pe[1] += max(1, self.edges[req.graph])


class Server:
    """slots worker streams, admission under a device-memory budget.

    policy "fifo": requests are admitted in arrival order; a request that
    does not fit the budget holds up the ones behind it.
    policy "edf": among the arrived requests that fit, the one with the
    earliest arrival + estimated service time (a CostModel) goes first, so a
    short request is not stuck behind long ones that arrived just before it,
    while a long request's turn still comes (its key does not grow)."""

    def __init__(self, graphs, slots: int = 4, budget_bytes: int | None = None, backend=None,
                 footprint=None, policy: str = "fifo", cost: CostModel | None = None):
        if policy not in ("fifo", "edf"):
            raise ValueError("policy is fifo or edf")
        self.policy = policy
        self.cost = cost
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
                        pick = self._pick()
                        if pick is not None:
                            req, fp = self._queue[pick]
                            del self._queue[pick]
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
                if self.cost is not None and err is None:
                    self.cost.observe(req, end - start)
                with self._cv:  # the slot, its footprint and the request are always released
                    self._in_use -= fp
                    self._running -= 1
                    self._results.append(Result(req.rid, int(value), float(est), req.arrival, start, end, err))
                    self._done += 1
                    self._cv.notify_all()

    def _fits(self, fp) -> bool:
        return self.budget is None or self._in_use + fp <= self.budget or self._running == 0

    def _pick(self):
        """Index in the queue of the request to admit now, or None."""
        if self.policy == "fifo":
            return 0 if self._fits(self._queue[0][1]) else None
        best, key = None, None
        for i, (req, fp) in enumerate(self._queue):
            if not self._fits(fp):
                continue
            kk = req.arrival + (self.cost.estimate(req) if self.cost else 0.0)
            if key is None or kk < key:
                best, key = i, kk
        return best

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
    """Latency percentiles, split into queue wait (arrival to start) and
    service (start to end), so a tail can be told apart: waiting behind other
    requests, or long requests themselves."""
    def pct(xs):
        a = np.array(xs) if xs else np.zeros(1)
        return float(np.percentile(a, 50) * 1e3), float(np.percentile(a, 99) * 1e3), float(a.mean() * 1e3)
    p50, p99, mean = pct([r.latency for r in results])
    w50, w99, wmean = pct([r.wait for r in results])
    s50, s99, smean = pct([r.service for r in results])
    return {"p50_ms": p50, "p99_ms": p99, "mean_ms": mean, "wait_p50_ms": w50, "wait_p99_ms": w99,
            "wait_mean_ms": wmean, "service_p50_ms": s50, "service_p99_ms": s99, "service_mean_ms": smean}
