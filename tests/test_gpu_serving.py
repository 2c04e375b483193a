"""Serving on the GPU: requests over device-resident graphs, admitted while
others run on other streams; every answer equals the same request served
alone, bit for bit (exact counts and sampled counts)."""
import numpy as np
import pytest

import kcgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1403_0734_gb300.build as kb
    kb.build()
    import paper_1403_0734_gb300 as kc
    from paper_1403_0734_gb300 import serve
    graphs = [kcgen.rmat(s, 16, 0.57, 0.19, 0.19, 10 + s) for s in (9, 10, 11, 12, 12, 13)]
    G = [kc.orient(g.off, g.adj) for g in graphs]
    return torch, kc, serve, graphs, G


def solo(kc, G, r):
    if r.colours:
        return kc.estimate(G[r.graph], r.k, r.colours, r.seed)[0]
    return kc.count(G[r.graph], r.k)[0]


@pytest.mark.parametrize("slots,budget", [(4, None), (8, None), (4, "one")])
def test_mix_equals_alone(env, slots, budget):
    torch, kc, serve, graphs, G = env
    reqs = serve.poisson_stream(150, rate=2000.0, ngraphs=len(G), seed=7)
    srv = serve.Server(G, slots=slots)
    if budget == "one":
        srv.budget = max(kc.footprint(G[r.graph], r.k) for r in reqs)
    res, makespan = srv.run(reqs, stream_factory=torch.cuda.Stream)
    want = {r.rid: solo(kc, G, r) for r in reqs}
    assert all(x.value == want[x.rid] for x in res)
    assert len(res) == len(reqs) and makespan > 0
    if budget is None:
        assert srv.max_concurrent > 1


def test_footprint_positive(env):
    torch, kc, serve, graphs, G = env
    for g in G:
        for k in (3, 6):
            assert kc.footprint(g, k) >= 256
            assert kc.footprint(g, k, per_vertex=True) >= kc.footprint(g, k) + 8 * g.n
