"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer results are compared bit for bit (totals, per-vertex membership
counts, per-owner counts, cFFF sampled counts); the cFFF estimate is compared
exactly too, since both sides round S * c^(k-2) the same way.  Graphs are
seeded and synthetic; sizes are chosen so the oracle finishes in seconds
while every owner class (bitmap width 1..32 words and the global-tile path)
is exercised, with ragged last words.
"""
from math import comb

import numpy as np
import pytest

import kcgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["pivot", "dfs"])
def kc(request):
    """The library, once with each Reduce 3 counter (pivoting tree, ordered DFS)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1403_0734_gb300.build as kb
    kb.build()
    import paper_1403_0734_gb300 as kc
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)
    kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_PIVOT if request.param == "pivot" else kc.KC_ALGO_DFS)
    yield kc
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)
    kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_DFS)


def elem_sym(values, k):
    e = [1] + [0] * k
    for a in values:
        for j in range(k, 0, -1):
            e[j] += e[j - 1] * a
    return e[k]


GRAPHS = {
    "er_1000": lambda: kcgen.er_1000(),
    "chunglu_20k": lambda: kcgen.chung_lu(20000, 200000, 2.1, 2000.0, 1),
    "sbm_20k": lambda: kcgen.sbm(20000, 50, 0.3, 500000, 1),
    "rmat_s12": lambda: kcgen.rmat(12, 16, 0.57, 0.19, 0.19, 1),
    "rmat_s14": lambda: kcgen.rmat(14, 16, 0.57, 0.19, 0.19, 1),
    "chunglu_50k": lambda: kcgen.chung_lu(50000, 1000000, 2.1, 5000.0, 1),
}
_cache = {}


def graph(name):
    if name not in _cache:
        _cache[name] = GRAPHS[name]()
    return _cache[name]


def quantise_work(w):
    """q(w) = min(31, max(0, 2 b + f - 20)): b = floor(log2(w + 1)), f = the
    bit of w + 1 below its leading one (the queue's work-estimate order, kc.h)."""
    x = int(w) + 1
    b = x.bit_length() - 1
    f = (x >> (b - 1)) & 1 if b >= 1 else 0
    return min(31, max(0, 2 * b + f - 20))


def expected_queue(offp, adjp):
    """The documented owner queue from an oriented CSR: groups by bitmap
    width (|Gamma+| > 1024 first ... 1..32, then 0), |Gamma+| descending in
    the 1..32 group, quantised work estimate sum |Gamma+(x)| descending in
    the wider groups, ties by rank."""
    dplus = np.diff(offp)
    n = dplus.size
    key = np.zeros(n, dtype=np.int64)
    for r in range(n):
        d = int(dplus[r])
        if d == 0:
            key[r] = 7 << 5
        elif d <= 32:
            key[r] = (6 << 5) | (32 - d)
        else:
            cls = 5 if d <= 64 else 4 if d <= 128 else 3 if d <= 256 else 2 if d <= 512 else 1 if d <= 1024 else 0
            w = int(dplus[adjp[offp[r]:offp[r + 1]]].sum())
            key[r] = (cls << 5) | (31 - quantise_work(w))
    return np.lexsort((np.arange(n), key))


def check_count(kc, g, G, k):
    total, pv, po = kc.count(G, k, per_vertex=True, per_owner=True)
    ot, opo, opv = oracle.count(g, k, per_owner=True, per_vertex=True)
    assert total == ot, (g.name, k, total, ot)
    assert np.array_equal(po, opo), (g.name, k)
    assert np.array_equal(pv, opv), (g.name, k)
    # the total without per-vertex work takes another kernel variant
    t2, _, _ = kc.count(G, k)
    assert t2 == ot


# ------------------------------------------------------------ orientation

@pytest.mark.parametrize("name", ["er_1000", "chunglu_20k", "sbm_20k", "rmat_s12"])
def test_orientation_matches_oracle(kc, name):
    g = graph(name)
    G = kc.orient(g.off, g.adj, validate=True)
    ex = kc.export(G)
    perm, rank, offp, adjp = oracle.oriented(g)
    assert np.array_equal(ex["perm"], perm)
    assert np.array_equal(ex["rank"], rank)
    assert np.array_equal(ex["off_plus"], offp)
    assert np.array_equal(ex["adj_plus"], adjp)
    dplus = np.diff(offp)
    assert np.array_equal(ex["queue"], expected_queue(offp, adjp))
    assert G.max_dplus == int(dplus.max())
    assert G.wedges == int((dplus * (dplus - 1) // 2).sum())
    assert G.m == g.m


def test_orientation_long_rows(kc):
    # complete graph: rows of every length 0..n-1, all through the block and
    # warp fill kernels; equal degrees, so the order is by id
    g = kcgen.complete(300)
    G = kc.orient(g.off, g.adj)
    ex = kc.export(G)
    assert np.array_equal(ex["perm"], np.arange(300))
    for r in (0, 1, 150, 298, 299):
        assert np.array_equal(ex["adj_plus"][ex["off_plus"][r]:ex["off_plus"][r + 1]], np.arange(r + 1, 300))


def test_orientation_cta_rows(kc):
    """Rows longer than a warp handles (one CTA per row, kept entries sorted
    in shared memory): K_1100 whose vertex v also carries pi(v) pendant
    leaves, pi a seeded permutation, so the order of the core follows pi and
    not the ids; each core row's Gamma+ is the core vertices of larger pi."""
    n = 1100
    pi = np.random.default_rng(5).permutation(n)
    iu, ju = np.triu_indices(n, 1)
    leaves_of = np.repeat(np.arange(n), pi)
    leaf_ids = n + np.arange(leaves_of.size)
    e = np.concatenate([np.stack([iu, ju], 1), np.stack([leaves_of, leaf_ids], 1)])
    g = kcgen.from_edges(n + leaves_of.size, e)
    G = kc.orient(g.off, g.adj, validate=True)
    ex = kc.export(G)
    rank = ex["rank"]
    for v in range(0, n, 37):
        want = np.sort(rank[np.flatnonzero(pi > pi[v])])
        r = rank[v]
        assert np.array_equal(ex["adj_plus"][ex["off_plus"][r]:ex["off_plus"][r + 1]], want), v
    assert np.array_equal(np.argsort(rank[:n]), np.argsort(pi))  # the core ordered by degree = n - 1 + pi
    assert G.max_dplus == n - 1


def test_orientation_global_sort_rows(kc):
    """A row with more than 8192 kept entries (sorted in place in global
    memory): K_8300 built directly as a CSR; equal degrees, so the order is
    the id order and row r of the oriented CSR is r+1..n-1."""
    n = 8300
    off = np.arange(n + 1, dtype=np.int64) * (n - 1)
    full = np.tile(np.arange(n, dtype=np.int32), n).reshape(n, n)
    adj = full[~np.eye(n, dtype=bool)].astype(np.int32)
    del full
    G = kc.orient(off, adj)
    ex = kc.export(G)
    assert np.array_equal(ex["perm"], np.arange(n))
    for r in (0, 1, 2, 100, 4000, 8298, 8299):
        assert np.array_equal(ex["adj_plus"][ex["off_plus"][r]:ex["off_plus"][r + 1]], np.arange(r + 1, n)), r
    assert G.max_dplus == n - 1 and G.m == n * (n - 1) // 2
    G.free()


# ------------------------------------------------------------ exact counts

@pytest.mark.parametrize("name,ks", [("er_1000", (3, 4, 5)), ("chunglu_20k", (3, 4, 5, 6, 7)),
                                     ("sbm_20k", (3, 4, 5, 6, 7)), ("rmat_s12", (3, 4, 5, 6)),
                                     ("rmat_s14", (3, 4, 5)), ("chunglu_50k", (3, 4))])
def test_counts_match_oracle(kc, name, ks):
    g = graph(name)
    G = kc.orient(g.off, g.adj)
    for k in ks:
        check_count(kc, g, G, k)


@pytest.mark.parametrize("maxw", [1, 2, 4])
def test_global_tile_path_matches_oracle(kc, maxw):
    """Owners wider than `maxw` words are forced onto the global-memory tiles."""
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, maxw)
    try:
        for name, ks in (("rmat_s14", (3, 4, 5)), ("chunglu_20k", (3, 4, 6))):
            g = graph(name)
            G = kc.orient(g.off, g.adj)
            for k in ks:
                check_count(kc, g, G, k)
    finally:
        kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)


def test_wide_dense_owners_match_oracle(kc):
    # G(n, p) dense: owners with |Gamma+| in the 8-, 16- and 32-word classes
    for n, p, seed, ks in ((700, 0.45, 1, (3, 4)), (1400, 0.5, 2, (3,))):
        g = kcgen.random_small(n, p, seed)
        G = kc.orient(g.off, g.adj)
        assert G.max_dplus > 256
        for k in ks:
            check_count(kc, g, G, k)


@pytest.mark.parametrize("complement", [1, 0])
@pytest.mark.parametrize("n,p,k", [(160, 0.86, 5), (150, 0.88, 5), (90, 0.95, 6), (140, 0.78, 5)])
def test_dense_random_per_vertex(kc, n, p, k, complement):
    """Dense G(n, p): the candidate sets closed by the last-three-levels
    count are dense enough (p >= 0.86) for the complement count of
    per-vertex mode, or just below its switch (p = 0.78, sets at density
    ~0.78 and below); with the complement count on and off, both ways of
    closing them are compared with the oracle, element by element."""
    g = kcgen.random_small(n, p, 3)
    G = kc.orient(g.off, g.adj)
    assert G.max_dplus > 64
    kc.set_param(kc.KC_PARAM_COMPLEMENT, complement)
    try:
        check_count(kc, g, G, k)
    finally:
        kc.set_param(kc.KC_PARAM_COMPLEMENT, 1)


def test_complement_count_with_saturated_non_degrees(kc):
    """A dense candidate set in which one element has more than 254
    non-neighbours (its byte in the per-warp non-degree table saturates and
    the count falls back to its row).  K_500 on core = S + T (|S| = 200,
    |T| = 300); a vertex a adjacent to S only; 5 pendants on every vertex of
    T and 400 on a, so that by degree S < T < a.  An owner in S has G+(u) =
    (S above it) + T + a, 16-word rows, and at k = 5 each of its first-level
    sets holds a with its 300 non-neighbours T.  Closed forms: q_k =
    C(500, k) + C(200, k-1); memberships C(200, k-1) for a, C(499, k-1) +
    C(199, k-2) on S, C(499, k-1) on T, 0 on the pendants."""
    S, T = np.arange(200), np.arange(200, 500)
    a = 500
    core = np.arange(500)
    iu, ju = np.triu_indices(500, 1)
    edges = [np.stack([core[iu], core[ju]], axis=1), np.stack([np.full(200, a), S], axis=1)]
    nxt = 501
    pend_t = np.stack([np.repeat(T, 5), nxt + np.arange(1500)], axis=1)
    nxt += 1500
    pend_a = np.stack([np.full(400, a), nxt + np.arange(400)], axis=1)
    nxt += 400
    g = kcgen.from_edges(nxt, np.concatenate(edges + [pend_t, pend_a]), "k500_split_core")
    G = kc.orient(g.off, g.adj)
    assert 257 <= G.max_dplus <= 512
    for k in (4, 5, 6):
        total, pv, _ = kc.count(G, k, per_vertex=True)
        assert total == comb(500, k) + comb(200, k - 1), k
        assert int(pv[a]) == comb(200, k - 1)
        assert np.all(pv[S] == comb(499, k - 1) + comb(199, k - 2))
        assert np.all(pv[T] == comb(499, k - 1))
        assert np.all(pv[501:] == 0)
        assert kc.count(G, k)[0] == total  # totals on symmetric rows (k = 6) and upper rows


@pytest.mark.parametrize("n,ks", [(31, (3, 5, 8, 31, 32)), (33, (3, 4, 7, 32)), (64, (3, 4, 6)),
                                  (65, (3, 5)), (200, (3, 4, 5, 7)), (520, (3, 4)), (1100, (3, 4)),
                                  (1500, (3,))])
def test_complete_graph_closed_form(kc, n, ks):
    g = kcgen.complete(n)
    G = kc.orient(g.off, g.adj)
    for k in ks:
        total, pv, po = kc.count(G, k, per_vertex=True, per_owner=True)
        assert total == comb(n, k)
        assert np.all(pv == comb(n - 1, k - 1))
        assert [int(x) for x in po] == [comb(n - 1 - r, k - 1) for r in range(n)]


@pytest.mark.parametrize("parts,ks", [((10,) * 60, (3, 4, 5)), ((7, 9, 11, 13) * 12, (3, 4, 6)),
                                      ((3,) * 400, (3, 4))])
def test_complete_multipartite_closed_form(kc, parts, ks):
    g = kcgen.complete_multipartite(parts, shuffle_seed=5)
    label = np.repeat(np.arange(len(parts)), parts)[np.random.default_rng(5).permutation(sum(parts))]
    G = kc.orient(g.off, g.adj)
    for k in ks:
        total, pv, _ = kc.count(G, k, per_vertex=True)
        assert total == elem_sym(parts, k)
        for v in range(0, g.n, 17):
            rest = [a for i, a in enumerate(parts) if i != label[v]]
            assert int(pv[v]) == elem_sym(rest, k - 1)


def test_uint64_scale_counts(kc):
    # counts far above 2^32 with little search work: the last two levels are
    # closed by popcounts, so K_{600,600,600,600} (k = 4) has 600^4 ~ 1.3e11
    # cliques but only ~2e6 search nodes; K_{2000,2000,2000} (k = 3) has 8e9
    for parts, k in (((600,) * 4, 4), ((2000,) * 3, 3)):
        g = kcgen.complete_multipartite(parts, shuffle_seed=1)
        G = kc.orient(g.off, g.adj)
        total, pv, _ = kc.count(G, k, per_vertex=True)
        assert total == elem_sym(parts, k) and total > 2**32
        assert int(pv.sum()) == k * total


# ------------------------------------------------------------ cFFF_k

@pytest.mark.parametrize("name", ["chunglu_20k", "sbm_20k", "rmat_s12"])
def test_estimate_matches_oracle(kc, name):
    g = graph(name)
    G = kc.orient(g.off, g.adj)
    for k in (3, 4, 5, 6):
        for c, seed in ((2, 1), (3, 7), (4, 1), (8, 2), (16, 3)):
            s, est, po = kc.estimate(G, k, c, seed, per_owner=True)
            os_, oest, opo = oracle.estimate(g, k, c, seed, per_owner=True)
            assert s == os_, (name, k, c, seed, s, os_)
            assert est == oest
            assert np.array_equal(po, opo)


def test_estimate_one_colour_is_exact(kc):
    g = graph("chunglu_20k")
    G = kc.orient(g.off, g.adj)
    for k in (3, 5):
        s, est, _ = kc.estimate(G, k, 1, 99)
        assert s == kc.count(G, k)[0] and est == float(s)


def test_estimate_global_tiles(kc):
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 1)
    try:
        g = graph("rmat_s14")
        G = kc.orient(g.off, g.adj)
        for k, c in ((3, 2), (4, 3), (5, 2)):
            assert kc.estimate(G, k, c, 5)[0] == oracle.estimate(g, k, c, 5)[0]
    finally:
        kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)


@pytest.mark.parametrize("name", ["chunglu_20k", "sbm_20k", "rmat_s12"])
def test_estimate_pairs_matches_oracle(kc, name):
    """Plain pair sampling (Sec. 6): sampled count and per-owner counts
    bit-exact, estimate identical."""
    g = graph(name)
    G = kc.orient(g.off, g.adj)
    for k in (3, 4, 5, 6):
        for p, seed in ((0.5, 1), (0.3, 7), (0.9, 2), (0.1, 3)):
            s, est, po = kc.estimate_pairs(G, k, p, seed, per_owner=True)
            os_, oest, opo = oracle.estimate_pairs(g, k, p, seed, per_owner=True)
            assert s == os_, (name, k, p, seed, s, os_)
            assert est == oest
            assert np.array_equal(po, opo)


def test_estimate_pairs_edges_and_tiles(kc):
    g = graph("chunglu_20k")
    G = kc.orient(g.off, g.adj)
    for k in (3, 5):  # p = 1 keeps every pair
        s, est, _ = kc.estimate_pairs(G, k, 1.0, 99)
        assert s == kc.count(G, k)[0] and est == float(s)
    for bad in (0.0, -0.5, 1.5, float("nan")):
        with pytest.raises(kc.KcError):
            kc.estimate_pairs(G, 3, bad, 1)
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 1)
    try:
        g = graph("rmat_s14")
        G = kc.orient(g.off, g.adj)
        for k, p in ((3, 0.5), (4, 0.7), (5, 0.8)):
            assert kc.estimate_pairs(G, k, p, 5)[0] == oracle.estimate_pairs(g, k, p, 5)[0]
    finally:
        kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)


@pytest.mark.parametrize("name", ["er_1000", "chunglu_20k", "sbm_20k", "rmat_s14", "chunglu_50k"])
@pytest.mark.parametrize("maxw", [32, 1])
def test_triangle_path_matches_oracle(kc, name, maxw):
    """k = 3 through the triangle path (no bitmaps) and through the bitmap
    path: totals, memberships and owner counts equal the oracle's.  n = 50000
    has owners whose Gamma+ spans more ranks than the direct table holds;
    maxw = 1 sends every owner wider than 32 to the widest-owner slot."""
    g = graph(name)
    G = kc.orient(g.off, g.adj)
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, maxw)
    try:
        for tri in (1, 0):
            kc.set_param(kc.KC_PARAM_TRI, tri)
            check_count(kc, g, G, 3)
    finally:
        kc.set_param(kc.KC_PARAM_TRI, 1)
        kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)


# ------------------------------------------------------------ edge cases

def test_edge_cases(kc):
    # isolated vertices only
    g = kcgen.empty(10)
    G = kc.orient(g.off, g.adj)
    assert kc.count(G, 1)[0] == 10 and kc.count(G, 2)[0] == 0 and kc.count(G, 3)[0] == 0
    # no vertices at all
    G = kc.orient(np.zeros(1, np.int64), np.zeros(0, np.int32))
    assert kc.count(G, 3)[0] == 0 and kc.count(G, 1)[0] == 0
    # k above the clique number, k = 1 and 2 with per-vertex outputs
    g = graph("er_1000")
    G = kc.orient(g.off, g.adj)
    assert kc.count(G, 6)[0] == 0
    t, pv, po = kc.count(G, 1, per_vertex=True, per_owner=True)
    assert t == g.n and np.all(pv == 1) and np.all(po == 1)
    t, pv, po = kc.count(G, 2, per_vertex=True, per_owner=True)
    assert t == g.m and np.array_equal(pv, g.degrees().astype(np.uint64))
    assert np.array_equal(po, oracle.count(g, 2, per_owner=True)[1])
    # invalid k
    for k in (0, -1, 33):
        with pytest.raises(kc.KcError):
            kc.count(G, k)
    with pytest.raises(kc.KcError):
        kc.estimate(G, 3, 0, 1)


def test_validate_rejects_malformed(kc):
    g = kcgen.cycle(6)
    bad = g.adj.copy()
    bad[0], bad[1] = bad[1], bad[0]  # unsorted row
    with pytest.raises(kc.KcError):
        kc.orient(g.off, bad, validate=True)
    asym = kcgen.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    a = asym.adj.copy()
    a[-1] = 0  # row 3 now says (3, 0) without (0, 3)
    with pytest.raises(kc.KcError):
        kc.orient(asym.off, a, validate=True)


def test_cycle_tie_break_and_small_graphs(kc):
    for g in (kcgen.cycle(3), kcgen.cycle(10), kcgen.star(40), kcgen.path(5)):
        G = kc.orient(g.off, g.adj, validate=True)
        for k in (2, 3, 4):
            check_count(kc, g, G, k)


@pytest.mark.parametrize("seed", range(6))
def test_random_small_graphs(kc, seed):
    g = kcgen.random_small(40 + 7 * seed, 0.35 + 0.08 * seed, 100 + seed)
    G = kc.orient(g.off, g.adj, validate=True)
    for k in range(3, 9):
        check_count(kc, g, G, k)


# ------------------------------------------------------------ API forms

def test_one_shot_and_device_pointer_forms(kc):
    import torch
    g = graph("rmat_s12")
    ot, opo, opv = oracle.count(g, 4, per_owner=True, per_vertex=True)
    t, pv, po = kc.count_csr(g.off, g.adj, 4, per_vertex=True, per_owner=True, validate=True)
    assert t == ot and np.array_equal(pv, opv) and np.array_equal(po, opo)
    s, est = kc.estimate_csr(g.off, g.adj, 4, 3, 7)
    assert (s, est) == oracle.estimate(g, 4, 3, 7)[:2]
    # inputs and outputs resident on the device
    off = torch.from_numpy(g.off).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    G = kc.orient(off, adj)
    total = torch.zeros(2, dtype=torch.int64, device="cuda")
    dpv = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    dpo = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    kc.count_device(G, 4, total, dpv, dpo)
    torch.cuda.synchronize()
    assert int(total[0]) == ot and int(total[1]) == 0
    assert np.array_equal(dpv.cpu().numpy().view(np.uint64), opv)
    assert np.array_equal(dpo.cpu().numpy().view(np.uint64), opo)


def test_repeatable(kc):
    g = graph("chunglu_20k")
    G = kc.orient(g.off, g.adj)
    a = kc.count(G, 5, per_vertex=True)
    b = kc.count(G, 5, per_vertex=True)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


# ------------------------------------------------------------ parts and batches

@pytest.mark.parametrize("maxw", [32, 1])
def test_parts_add_up_to_the_count(kc, maxw):
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, maxw)
    try:
        g = graph("rmat_s14")
        G = kc.orient(g.off, g.adj)
        for k in (3, 4, 5):
            t, pv, po = kc.count(G, k, per_vertex=True, per_owner=True)
            for nparts in (2, 3, 7):
                parts = [kc.count_part(G, k, p, nparts, per_vertex=True, per_owner=True) for p in range(nparts)]
                assert sum(x[0] for x in parts) == t
                spv = np.zeros(g.n, np.uint64)
                spo = np.zeros(g.n, np.uint64)
                owners = np.zeros(g.n, np.int64)
                for x in parts:
                    spv += x[1]
                    spo += x[2]
                    owners += (x[2] > 0)
                assert np.array_equal(spv, pv) and np.array_equal(spo, po)
                assert owners.max() <= 1  # every owner counted by one part
    finally:
        kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)


def test_part_arguments(kc):
    g = graph("er_1000")
    G = kc.orient(g.off, g.adj)
    for bad in ((3, 0, 0), (3, 2, 2), (3, -1, 2), (2, 0, 2)):
        with pytest.raises(kc.KcError):
            kc.count_part(G, bad[0], bad[1], bad[2])


@pytest.mark.parametrize("maxw", [32, 1])
def test_batch_matches_solo_counts(kc, maxw):
    graphs = kcgen.batch_workload(48, seed=3, nmin=20, nmax=4000)
    Gs = [kc.orient(g.off, g.adj) for g in graphs]
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, maxw)
    try:
        for k in (1, 2, 3, 4, 5):
            batch = kc.count_batch(Gs, k)
            solo = [kc.count(G, k)[0] for G in Gs]
            assert batch == solo, k
        for i in (0, 7, 31):
            assert kc.count_batch(Gs, 4)[i] == oracle.count(graphs[i], 4)[0]
    finally:
        kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)


def test_batch_edge_cases(kc):
    assert kc.count_batch([], 4) == []
    G = kc.orient(np.zeros(1, np.int64), np.zeros(0, np.int32))
    H = kc.orient(kcgen.complete(40).off, kcgen.complete(40).adj)
    assert kc.count_batch([G, H, G], 5) == [0, comb(40, 5), 0]


# ------------------------------------------------------------ listing (Sec. 3)

def _rows(a):
    """Rows as a lexicographically sorted array (for set comparison)."""
    a = np.ascontiguousarray(a, dtype=np.int32)
    if len(a) == 0:
        return a
    return a[np.lexsort(a.T[::-1])]


def check_listing(kc, g, G, k, cap):
    got = kc.list_cliques(G, k, cap=cap)
    want = oracle.list_cliques(g, k)
    assert got.shape == want.shape, (g.name, k, got.shape, want.shape)
    # rows are unique and in precedence order with the owner first, on both sides
    assert np.array_equal(_rows(got), _rows(want)), (g.name, k)


@pytest.mark.parametrize("name,ks", [("er_1000", (1, 2, 3, 4)), ("chunglu_20k", (3, 4, 5)),
                                     ("rmat_s12", (3, 4, 5)), ("sbm_20k", (4, 6))])
def test_listing_matches_oracle(kc, name, ks):
    g = graph(name)
    G = kc.orient(g.off, g.adj)
    for k in ks:
        check_listing(kc, g, G, k, cap=1 << 22)


def test_listing_small_runs_and_wide_owners(kc):
    """Runs as small as the largest owner's count (many runs), owners in the
    32-word class, and every owner above 32 in the widest-owner tiles."""
    g = kcgen.random_small(700, 0.45, 1)
    G = kc.orient(g.off, g.adj)
    _, po, _ = oracle.count(g, 4, per_owner=True)
    check_listing(kc, g, G, 4, cap=int(po.max()))
    g2 = graph("rmat_s12")
    G2 = kc.orient(g2.off, g2.adj)
    kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 1)
    try:
        for k in (3, 4):
            _, po2, _ = oracle.count(g2, k, per_owner=True)
            check_listing(kc, g2, G2, k, cap=int(po2.max()) + 7)
    finally:
        kc.set_param(kc.KC_PARAM_SMEM_MAX_WORDS, 32)


def test_listing_device_buffer_cancel_and_errors(kc):
    import torch
    g = graph("chunglu_20k")
    G = kc.orient(g.off, g.adj)
    k = 4
    q, po, _ = oracle.count(g, k, per_owner=True)
    cap = int(po.max()) * 3
    buf = torch.empty(cap * k, dtype=torch.int32, device="cuda")
    seen = []

    def fn(arg):
        ptr, count = arg
        seen.append(buf[: count * k].view(count, k).cpu().numpy().copy())
        return False

    assert kc.list_runs(G, k, fn, cap=cap, device_buffer=buf) == q
    assert len(seen) > 1
    assert np.array_equal(_rows(np.concatenate(seen)), _rows(oracle.list_cliques(g, k)))
    # the callback stops the listing after its first run
    first = []
    with pytest.raises(kc.KcError) as ei:
        kc.list_runs(G, k, lambda rows: first.append(len(rows)) or True, cap=cap)
    assert ei.value.status == kc.KC_ECANCELED and len(first) == 1
    # a buffer smaller than one owner's cliques
    with pytest.raises(kc.KcError) as ei:
        kc.list_runs(G, k, lambda rows: False, cap=int(po.max()) - 1)
    assert ei.value.status == kc.KC_ENOMEM
    # empty graph, k above the clique number
    G0 = kc.orient(np.zeros(1, np.int64), np.zeros(0, np.int32))
    assert kc.list_cliques(G0, 3).shape == (0, 3)
    ge = graph("er_1000")
    assert kc.list_cliques(kc.orient(ge.off, ge.adj), 7).shape == (0, 7)
