"""Host logic of the continuous-batching server (no GPU): a fake backend that
sleeps and returns oracle counts stands in for the C-ABI call."""
import threading
import time

import pytest

import kcgen
import oracle
from paper_1403_0734_gb300 import serve


@pytest.fixture(scope="module")
def graphs():
    return [kcgen.random_small(22, 0.5, s) for s in range(4)]


def make_backend(graphs, delay, tracker):
    lock = threading.Lock()

    def backend(req, stream):
        with lock:
            tracker["running"] += 1
            tracker["peak"] = max(tracker["peak"], tracker["running"])
        time.sleep(delay)
        g = graphs[req.graph]
        if req.colours:
            s, est, _ = oracle.estimate(g, req.k, req.colours, req.seed)
            out = (s, est)
        else:
            q = oracle.count(g, req.k)[0]
            out = (q, float(q))
        with lock:
            tracker["running"] -= 1
        return out
    return backend


def expected(graphs, r):
    if r.colours:
        return oracle.estimate(graphs[r.graph], r.k, r.colours, r.seed)[0]
    return oracle.count(graphs[r.graph], r.k)[0]


def test_results_and_overlap(graphs):
    reqs = serve.poisson_stream(40, rate=400.0, ngraphs=len(graphs), seed=3)
    tr = {"running": 0, "peak": 0}
    srv = serve.Server(graphs, slots=4, backend=make_backend(graphs, 0.01, tr), footprint=lambda r: 100)
    res, makespan = srv.run(reqs)
    assert [r.rid for r in res] == list(range(40))
    for r, q in zip(res, sorted(reqs, key=lambda x: x.rid)):
        assert r.value == expected(graphs, q)
        assert r.start >= q.arrival - 1e-6 and r.end >= r.start
    assert tr["peak"] > 1  # admitted while others were still running
    st = serve.latency_stats(res)
    assert 0 < st["p50_ms"] <= st["p99_ms"]


def test_budget_limits_concurrency(graphs):
    reqs = serve.poisson_stream(16, rate=1000.0, ngraphs=len(graphs), seed=4)
    tr = {"running": 0, "peak": 0}
    # budget of one request at a time, although four slots are free
    srv = serve.Server(graphs, slots=4, budget_bytes=100, backend=make_backend(graphs, 0.005, tr),
                       footprint=lambda r: 100)
    res, _ = srv.run(reqs)
    assert tr["peak"] == 1 and srv.max_concurrent == 1
    assert all(r.value == expected(graphs, q) for r, q in zip(res, sorted(reqs, key=lambda x: x.rid)))
    # two at a time
    tr = {"running": 0, "peak": 0}
    srv = serve.Server(graphs, slots=4, budget_bytes=250, backend=make_backend(graphs, 0.005, tr),
                       footprint=lambda r: 100)
    srv.run(reqs)
    assert tr["peak"] <= 2


def test_oversized_request_rejected(graphs):
    srv = serve.Server(graphs, slots=2, budget_bytes=10, backend=lambda r, s: (0, 0.0), footprint=lambda r: 11)
    with pytest.raises(ValueError):
        srv.run(serve.poisson_stream(2, 10.0, len(graphs), 1))


def test_failing_request_does_not_hang_the_server(graphs):
    """A backend that raises (e.g. an allocation failure in the library) for
    some requests: every request still completes, the slots and footprint are
    released, the failure is reported per request and run() raises after the
    others have finished."""
    tracker = {"running": 0, "peak": 0}
    ok = make_backend(graphs, 0.002, tracker)

    def backend(req, stream):
        if req.rid % 5 == 3:
            raise MemoryError("device allocation failed")
        return ok(req, stream)

    reqs = serve.poisson_stream(40, 0.0, len(graphs), seed=3, kmin=3, kmax=4)
    srv = serve.Server(graphs, slots=3, budget_bytes=100, backend=backend, footprint=lambda r: 40)
    done = {}

    def run():
        try:
            srv.run(reqs, realtime=False)
        except serve.RequestError as e:
            done["err"] = e

    t = threading.Thread(target=run, daemon=True)
    t.start()
    t.join(timeout=60)
    assert not t.is_alive(), "server hung after a failed request"
    err = done["err"]
    assert err.rid == 3 and "MemoryError" in str(err)
    res = err.results
    assert len(res) == len(reqs) and srv._in_use == 0 and srv._running == 0
    for r, q in zip(res, sorted(reqs, key=lambda x: x.rid)):
        if q.rid % 5 == 3:
            assert r.error is not None
        else:
            assert r.error is None and r.value == expected(graphs, q)
    # the same server runs a clean stream afterwards
    res2, _ = serve.Server(graphs, slots=3, backend=ok, footprint=lambda r: 1).run(
        serve.poisson_stream(10, 0.0, len(graphs), seed=4, kmin=3, kmax=4), realtime=False)
    assert all(r.error is None for r in res2)


def test_edf_admission_lets_short_requests_pass(graphs):
    """A burst of long requests (k = 5, sleep 40 ms) followed by short ones
    (k = 3, 1 ms) on one slot: FIFO makes every short request wait for all the
    long ones; EDF (arrival + estimated cost, costs learned per request type)
    runs them as soon as their cost is known, and every answer is unchanged."""
    def backend(req, stream):
        time.sleep(0.04 if req.k == 5 else 0.001)
        return expected(graphs, req), float(expected(graphs, req))

    reqs = [serve.Request(i, i % len(graphs), 5, 0, i, 0.0) for i in range(6)]
    reqs += [serve.Request(6 + i, i % len(graphs), 3, 0, 6 + i, 0.001) for i in range(6)]
    stats = {}
    for policy in ("fifo", "edf"):
        cost = serve.CostModel([1000] * len(graphs))
        # teach the model both request types first (the type means are what EDF uses)
        cost.observe(reqs[0], 0.04)
        cost.observe(reqs[6], 0.001)
        for g in range(len(graphs)):
            cost.observe(serve.Request(0, g, 5, 0, 0, 0.0), 0.04)
            cost.observe(serve.Request(0, g, 3, 0, 0, 0.0), 0.001)
        srv = serve.Server(graphs, slots=1, backend=backend, footprint=lambda r: 1, policy=policy, cost=cost)
        res, _ = srv.run(reqs, realtime=False)
        for r, q in zip(res, sorted(reqs, key=lambda x: x.rid)):
            assert r.value == expected(graphs, q)
        short = [r for r in res if r.rid >= 6]
        stats[policy] = max(r.latency for r in short)
        st = serve.latency_stats(res)
        assert st["wait_p99_ms"] <= st["p99_ms"] + 1e-6
    assert stats["edf"] < stats["fifo"] / 2
