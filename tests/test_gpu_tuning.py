"""GPU: the autotuner's plans change speed only, never results.

kc_tune measures per owner class the ordered search (1, 4 or 16 parts per
owner) against the pivoting counter on the class's heaviest owners; counts
with any attached plan must equal the oracle's bit for bit, for single graphs
(totals, per-vertex, per-owner) and batches.  On graphs made of disjoint
K_50 blocks (near-complete G+(u)) the pivoting counter, which closes whole
cliques by binomial coefficients, must be chosen for the wide classes.
"""
import json
import os
from math import comb

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
    kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_DFS)
    return kc


def all_plans():
    """Every single-choice plan: all classes DFS with 1/4/16 parts, or pivot."""
    for algo, parts in ((1, 1), (1, 4), (1, 16), (0, 1)):
        yield {"algo": [algo] * 7, "parts": [parts] * 7}


@pytest.mark.parametrize("name,maker,ks", [
    ("planted", lambda: kcgen.planted_core(30000, 300000, 1200, 0.3, 3), (4, 5, 6)),
    ("sbm_dense", lambda: kcgen.sbm(1980, 30, 1.0, 30000, 2), (4, 6)),
    ("chunglu_20k", lambda: kcgen.chung_lu(20000, 200000, 2.1, 2000.0, 1), (4, 5, 6)),
])
def test_plans_keep_counts(kc, name, maker, ks):
    g = maker()
    G = kc.orient(g.off, g.adj)
    for k in ks:
        ot, opo, opv = oracle.count(g, k, per_owner=True, per_vertex=True)
        for pv in (False, True):
            tuned = kc.tune(G, k, per_vertex=pv)
            assert tuned["k"] == k and tuned["per_vertex"] == pv
            for plan in [tuned, *[dict(p, k=k, per_vertex=pv) for p in all_plans()]]:
                kc.set_tuning(G, plan)
                total, pvv, po = kc.count(G, k, per_vertex=pv, per_owner=True)
                assert total == ot and np.array_equal(po, opo), (name, k, pv, plan)
                if pv:
                    assert np.array_equal(pvv, opv), (name, k, plan)
        kc.set_tuning(G, None)
    G.free()


def test_pivot_chosen_on_dense_blocks(kc):
    """Disjoint K_50 blocks: every G+(u) is complete, where pivoting is far
    cheaper than enumerating ordered chains."""
    g = kcgen.sbm(20000, 50, 1.0, 490000, 4)  # exactly the 400 blocks' pairs: no other edges
    assert g.m == 400 * comb(50, 2)
    G = kc.orient(g.off, g.adj)
    plan = kc.tune(G, 7)
    # the class holding the blocks' widest owners (|Gamma+| 33..49)
    assert plan["algo"][5] == kc.KC_ALGO_PIVOT, plan
    kc.set_tuning(G, plan)
    assert kc.count(G, 7)[0] == 400 * comb(50, 7)  # C(50, 7) 7-cliques in each block
    G.free()


def test_batch_plan_and_cache(kc, tmp_path):
    graphs = [kcgen.chung_lu(n, m, 2.3, max(1.0, (2 * m) ** 0.5), s)
              for (n, m, s) in ((800, 6000, 1), (3000, 30000, 2), (200, 1500, 3), (5000, 90000, 4))]
    Gs = [kc.orient(g.off, g.adj) for g in graphs]
    want = [oracle.count(g, 4)[0] for g in graphs]
    assert kc.count_batch(Gs, 4) == want
    plan = kc.tune(Gs, 4)
    for p in [plan, *[dict(p, k=4, per_vertex=False) for p in all_plans()]]:
        kc.set_tuning(Gs[0], p)
        assert kc.count_batch(Gs, 4) == want
    kc.set_tuning(Gs[0], None)
    cache = kc.TuningCache(str(tmp_path / "plans.json"))
    p1 = cache.plan(Gs[3], 5)
    assert os.path.exists(tmp_path / "plans.json")
    cache2 = kc.TuningCache(str(tmp_path / "plans.json"))
    assert cache2.plan(Gs[3], 5) == json.loads(json.dumps(p1))  # served from the file
    assert kc.count(Gs[3], 5)[0] == oracle.count(graphs[3], 5)[0]
    with pytest.raises(kc.KcError):
        kc.set_tuning(Gs[0], dict(plan, algo=[7] * 7))
    for G in Gs:
        G.free()
