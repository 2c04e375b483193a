"""GPU: counts captured into a CUDA graph and replayed (launch-bound small
graphs and batches replay one graph instead of many launches).  Every replay
must give the same exact counts as the direct call and the oracle."""
import numpy as np
import pytest

import kcgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1403_0734_gb300.build as kb
    kb.build()
    import paper_1403_0734_gb300 as kc
    return kc


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_count_replayed_from_cuda_graph(kc, k):
    import torch
    g = kcgen.chung_lu(20000, 200000, 2.1, 2000.0, 1)
    G = kc.orient(g.off, g.adj)
    ot, opo, opv = oracle.count(g, k, per_owner=True, per_vertex=True)
    n = g.n
    tot = torch.zeros(2, dtype=torch.int64, device="cuda")
    pv = torch.zeros(n, dtype=torch.int64, device="cuda")
    po = torch.zeros(n, dtype=torch.int64, device="cuda")
    kc.count(G, k)  # the graph's orientation is complete before the capture
    s = torch.cuda.Stream()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=s):
        kc.count_device(G, k, tot, pv, po)
    for _ in range(3):
        tot.fill_(-1)
        pv.fill_(-1)
        po.fill_(-1)
        cg.replay()
        torch.cuda.synchronize()
        assert int(tot[0].item()) == ot and int(tot[1].item()) == 0
        assert np.array_equal(pv.cpu().numpy().view(np.uint64), opv)
        assert np.array_equal(po.cpu().numpy().view(np.uint64), opo)
    G.free()


def test_batch_object_captured_and_replayed(kc):
    import torch
    params = kcgen.batch_params(48, seed=7, nmax=3000)
    graphs = [kcgen.chung_lu(n, m, 2.3, w, s) for (n, m, w, s) in params]
    Gs = [kc.orient(g.off, g.adj) for g in graphs]
    k = 4
    want = [oracle.count(g, k)[0] for g in graphs]
    assert kc.count_batch(Gs, k) == want
    b = kc.Batch(Gs, k)
    out = torch.zeros(2 * len(Gs), dtype=torch.int64, device="cuda")
    b.count(out)
    torch.cuda.synchronize()
    assert [int(x) for x in out[0::2].tolist()] == want and int(out[1::2].abs().sum()) == 0
    s = torch.cuda.Stream()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=s):
        b.count(out)
    for _ in range(3):
        out.fill_(-1)
        cg.replay()
        torch.cuda.synchronize()
        assert [int(x) for x in out[0::2].tolist()] == want
    # with a tuned plan attached to the first graph
    kc.set_tuning(Gs[0], kc.tune(Gs, k))
    b2 = kc.Batch(Gs, k)
    b2.count(out)
    torch.cuda.synchronize()
    assert [int(x) for x in out[0::2].tolist()] == want
    b.free()
    b2.free()
    for G in Gs:
        G.free()
