"""GPU parity on irregular graphs whose hubs reach the widest bitmap classes.

The counting kernels pick a layout by the width of an owner's bitmap row,
W = ceil(|Gamma+(u)| / 32) words.  The 16-word (|Gamma+| 257..512) and
32-word (513..1024) classes run the split search (one owner's first level
shared by several CTAs) and, on the Chung-Lu workload, hold most of the
counting time.  These tests compare those classes element by element with
the oracle on graphs with irregular structure, not only on closed forms:

* a planted-core graph (power-law background plus a sparse random core whose
  vertices become hubs): every owner, per-vertex and per-owner, k = 5, 6, 7;
* the Chung-Lu benchmark graph itself (n = 10^6, m ~ 2*10^7): per-owner counts
  of its 200 widest owners and a seeded uniform sample, k = 4 and 5; a sample
  of owners up to 128 wide at k = 6 (the widest owners' k = 6 counts are
  beyond the oracle's reach), plus the per-owner / per-vertex invariants;
* the dense-block SBM (40,000 blocks of K_50, m = 5*10^7) at k = 7: sampled
  owners against the oracle, including the lowest-ranked vertex of blocks,
  whose q_{u,6} = C(49, 6) is the largest.

Every clique is counted once by its smallest vertex (Sec. 3), so per-owner
counts are unique and compared exactly.
"""
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
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)
    kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_DFS)
    yield kc
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)
    kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_DFS)


_cache = {}


def cached(key, fn):
    if key not in _cache:
        _cache[key] = fn()
    return _cache[key]


def planted():
    return cached("planted", lambda: kcgen.planted_core(100000, 1000000, 3000, 0.2, 7))


def planted_oracle(k):
    return cached(("planted", k), lambda: oracle.count(planted(), k, per_owner=True, per_vertex=True))


def widths(kc, G):
    dp = np.diff(kc.export(G)["off_plus"])
    return dp, int(((dp > 256) & (dp <= 512)).sum()), int(((dp > 512) & (dp <= 1024)).sum())


@pytest.mark.parametrize("algo", ["dfs", "pivot"])
@pytest.mark.parametrize("k", [5, 6, 7])
def test_planted_core_hub_classes(kc, algo, k):
    g = planted()
    kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_DFS if algo == "dfs" else kc.KC_ALGO_PIVOT)
    try:
        G = kc.orient(g.off, g.adj)
        _, w16, w32 = widths(kc, G)
        assert w16 > 0 and w32 > 0, (w16, w32)  # both wide classes are populated
        ot, opo, opv = planted_oracle(k)
        total, pv, po = kc.count(G, k, per_vertex=True, per_owner=True)
        assert total == ot
        assert np.array_equal(po, opo)
        assert np.array_equal(pv, opv)
        assert kc.count(G, k)[0] == ot  # total-only kernels
        _, _, po2 = kc.count(G, k, per_owner=True)
        assert np.array_equal(po2, opo)
        G.free()
    finally:
        kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_DFS)


@pytest.mark.parametrize("maxw", [4, 8, 16])
def test_planted_core_global_tiles(kc, maxw):
    """The wide owners forced onto global-memory tiles."""
    g = planted()
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, maxw)
    try:
        G = kc.orient(g.off, g.adj)
        for k in (5, 6):
            ot, opo, opv = planted_oracle(k)
            total, pv, po = kc.count(G, k, per_vertex=True, per_owner=True)
            assert total == ot and np.array_equal(po, opo) and np.array_equal(pv, opv), (maxw, k)
        G.free()
    finally:
        kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)


def test_planted_core_estimate(kc):
    """cFFF_k sampled counts on the wide classes (colour filter in the build)."""
    g = planted()
    G = kc.orient(g.off, g.adj)
    for k, c, seed in ((5, 2, 3), (6, 4, 9), (6, 8, 1)):
        s, est, po = kc.estimate(G, k, c, seed, per_owner=True)
        os_, oest, opo = oracle.estimate(g, k, c, seed, per_owner=True)
        assert s == os_ and est == oest and np.array_equal(po, opo), (k, c, seed)
    G.free()


def chung_lu_1m():
    return cached("cl1m", lambda: kcgen.chung_lu_1m(1))


def test_chung_lu_1m_sampled_owners(kc):
    g = chung_lu_1m()
    G = kc.orient(g.off, g.adj)
    ex = kc.export(G)
    dp_rank = np.diff(ex["off_plus"])
    dp = np.empty(g.n, np.int64)
    dp[ex["perm"]] = dp_rank  # d+ by caller id
    assert int(((dp > 256) & (dp <= 512)).sum()) > 0
    rng = np.random.default_rng(2024)
    widest = np.argsort(-dp, kind="stable")[:200]
    uniform = rng.choice(g.n, 200, replace=False)
    for k in (4, 5):
        total, pv, po = kc.count(G, k, per_vertex=True, per_owner=True)
        assert int(pv.sum()) == k * total and int(po.sum()) == total
        for own in (widest, uniform):
            assert np.array_equal(po[own], oracle.count_owners(g, k, own)), k
    # k = 6: owners up to 128 wide (4-word rows) against the oracle
    total, pv, po = kc.count(G, 6, per_vertex=True, per_owner=True)
    assert int(pv.sum()) == 6 * total and int(po.sum()) == total
    mid = np.flatnonzero((dp >= 65) & (dp <= 128))
    light = np.flatnonzero((dp >= 5) & (dp <= 64))
    sample = np.concatenate([rng.choice(mid, min(150, mid.size), replace=False),
                             rng.choice(light, 150, replace=False)])
    assert np.array_equal(po[sample], oracle.count_owners(g, 6, sample))
    G.free()


def test_sbm_dense_k7_sampled_owners(kc):
    g = kcgen.sbm_2m(1, 1.0)
    G = kc.orient(g.off, g.adj)
    total = kc.count(G, 7)[0]
    _, _, po = kc.count(G, 7, per_owner=True)
    assert int(po.sum()) == total
    assert total >= 40000 * 99884400  # every K_50 block alone holds C(50, 7) 7-cliques
    rng = np.random.default_rng(77)
    ex = kc.export(G)
    # lowest-ranked vertex of the blocks holding 64 sampled vertices: its
    # Gamma+ spans its whole block, q_{u,6} >= C(49, 6)
    perm, rank = ex["perm"], ex["rank"]
    sample = rng.choice(g.n, 2000, replace=False)
    heads = []
    for v in sample[:64]:
        nb = g.adj[g.off[v]:g.off[v + 1]]
        blk = np.concatenate([[v], nb])
        heads.append(int(blk[np.argmin(rank[blk])]))
    own = np.unique(np.concatenate([sample, np.array(heads)]))
    want = oracle.count_owners(g, 7, own)
    assert np.array_equal(po[own], want)
    assert int(want.max()) >= 13983816  # C(49, 6): a block head was sampled
    G.free()
