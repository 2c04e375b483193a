"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: the
definition of q_k written out as brute force over k-subsets, closed forms
(complete and complete multipartite graphs), invariants the paper proves, or
exhaustive enumeration of colourings.  A plausible slip in the oracle (a
dropped term, a wrong comparison in the total order, a swapped index in the
pair test, a wrong colour scale) fails at least one test here.
"""
from itertools import combinations, product
from math import comb, isqrt

import numpy as np
import pytest

import kcgen
import oracle

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def elem_sym(values, k):
    """Elementary symmetric polynomial e_k(values) (exact integers)."""
    e = [1] + [0] * k
    for a in values:
        for j in range(k, 0, -1):
            e[j] += e[j - 1] * a
    return e[k]


def py_cliques(g, k):
    """All k-cliques of a tiny graph as sorted tuples (itertools brute force)."""
    nbr = [set(g.adj[g.off[v]:g.off[v + 1]].tolist()) for v in range(g.n)]
    return [S for S in combinations(range(g.n), k)
            if all(b in nbr[a] for a, b in combinations(S, 2))]


def py_owner_counts(g, k):
    """owner(u) = #{k-cliques whose minimum under (degree, id) is u} (Sec. 3)."""
    deg = g.degrees()
    own = np.zeros(g.n, dtype=np.uint64)
    for S in py_cliques(g, k):
        own[min(S, key=lambda v: (deg[v], v))] += 1
    return own


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_complete_graph_closed_form(n):
    g = kcgen.complete(n)
    for k in range(1, n + 2):
        total, po, pv = oracle.count(g, k, per_owner=True, per_vertex=True)
        assert total == comb(n, k)
        # every vertex lies in C(n-1, k-1) cliques
        assert all(int(x) == comb(n - 1, k - 1) for x in pv)
        # equal degrees: the order is by id, so vertex r owns C(n-1-r, k-1)
        assert [int(x) for x in po] == [comb(n - 1 - r, k - 1) for r in range(n)]


@pytest.mark.parametrize("parts", [(1, 1, 1), (2, 3), (3, 3, 3), (1, 2, 3, 4), (2, 2, 2, 2, 2), (5, 1, 4, 2)])
def test_complete_multipartite_closed_form(parts):
    g = kcgen.complete_multipartite(parts, shuffle_seed=7)
    label = np.repeat(np.arange(len(parts)), parts)[np.random.default_rng(7).permutation(sum(parts))]
    for k in range(1, len(parts) + 2):
        total, _, pv = oracle.count(g, k, per_vertex=True)
        assert total == elem_sym(parts, k)
        for v in range(g.n):
            rest = [a for i, a in enumerate(parts) if i != label[v]]
            assert int(pv[v]) == elem_sym(rest, k - 1)


@pytest.mark.parametrize("n,r", [(10, 3), (12, 4), (13, 5)])
def test_turan_graph(n, r):
    parts = [n // r + (1 if i < n % r else 0) for i in range(r)]
    g = kcgen.complete_multipartite(parts)
    for k in range(3, r + 2):
        assert oracle.count(g, k)[0] == elem_sym(parts, k)


@pytest.mark.parametrize("maker", [lambda: kcgen.empty(9), lambda: kcgen.star(12),
                                   lambda: kcgen.path(10), lambda: kcgen.cycle(7),
                                   lambda: kcgen.from_edges(8, [(0, 1), (2, 3), (4, 5), (6, 7)])])
def test_triangle_free_families(maker):
    g = maker()
    for k in range(3, 7):
        assert oracle.count(g, k)[0] == 0


def test_k1_k2_and_small_cycle():
    g = kcgen.cycle(3)
    assert oracle.count(g, 3)[0] == 1
    g = kcgen.random_small(20, 0.3, 5)
    assert oracle.count(g, 1)[0] == g.n
    assert oracle.count(g, 2)[0] == g.m


def test_star_owner_counts_follow_degree_first_order():
    # leaves have degree 1 < d(centre): every edge is owned by its leaf
    g = kcgen.star(9)
    _, po, _ = oracle.count(g, 2, per_owner=True)
    assert int(po[0]) == 0 and all(int(x) == 1 for x in po[1:])


# ----------------------------------------------------------------- brute force

@pytest.mark.parametrize("n,p,seed", [(12, 0.5, 1), (18, 0.7, 2), (25, 0.4, 3), (30, 0.6, 4), (16, 0.9, 5)])
def test_matches_brute_force(n, p, seed):
    g = kcgen.random_small(n, p, seed)
    for k in range(1, 8):
        total, po, pv = oracle.count(g, k, per_owner=True, per_vertex=True)
        bf, bpv = oracle.brute_force(g, k, per_vertex=True)
        assert total == bf
        assert np.array_equal(pv, bpv)
        assert int(po.sum()) == total


@pytest.mark.parametrize("n,p,seed", [(10, 0.6, 11), (14, 0.5, 12), (13, 0.8, 13)])
def test_owner_counts_match_python_definition(n, p, seed):
    g = kcgen.random_small(n, p, seed)
    for k in range(2, 6):
        _, po, _ = oracle.count(g, k, per_owner=True)
        assert np.array_equal(po, py_owner_counts(g, k))


def test_brute_force_matches_itertools():
    g = kcgen.random_small(14, 0.55, 21)
    for k in range(1, 7):
        assert oracle.brute_force(g, k)[0] == len(py_cliques(g, k))


def test_er_1000_triangles_brute_force():
    # the 1000-vertex / 10^4-edge Erdos-Renyi workload: all C(1000,3) triples
    g = kcgen.er_1000()
    assert g.n == 1000 and g.m == 10000
    bf, _ = oracle.brute_force(g, 3)
    assert oracle.count(g, 3)[0] == bf


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("seed", [1, 2])
def test_membership_and_owner_sums(seed):
    g = kcgen.chung_lu(3000, 30000, 2.1, 300.0, seed)
    for k in range(3, 7):
        total, po, pv = oracle.count(g, k, per_owner=True, per_vertex=True)
        assert int(pv.sum()) == k * total
        assert int(po.sum()) == total


def test_relabelling_invariance():
    g = kcgen.chung_lu(800, 8000, 2.3, 120.0, 3)
    perm = np.random.default_rng(9).permutation(g.n)
    h = kcgen.relabel(g, perm)
    for k in range(3, 7):
        tg, _, pg = oracle.count(g, k, per_vertex=True)
        th, _, ph = oracle.count(h, k, per_vertex=True)
        assert tg == th
        assert np.array_equal(ph[perm], pg)


def test_disjoint_union_adds():
    a = kcgen.random_small(15, 0.6, 31)
    b = kcgen.complete(7)
    u = kcgen.disjoint_union(a, b)
    for k in range(3, 7):
        assert oracle.count(u, k)[0] == oracle.count(a, k)[0] + comb(7, k)


def test_orientation_invariants():
    """Sum of d+ = m, max d+ <= 2 sqrt(m) (Thm I), sum of |E(G+(u))| = q_3,
    and Gamma+ lists are exactly the higher neighbours in the order."""
    g = kcgen.chung_lu(5000, 50000, 2.1, 600.0, 4)
    perm, rank, offp, adjp = oracle.oriented(g)
    dplus = np.diff(offp)
    assert int(dplus.sum()) == g.m
    assert int(dplus.max()) <= 2 * isqrt(g.m) + 2
    deg = g.degrees()
    key = deg * (g.n + 1) + np.arange(g.n)
    assert np.array_equal(np.argsort(key, kind="stable"), perm)
    for r in range(0, g.n, 97):
        row = adjp[offp[r]:offp[r + 1]]
        assert np.all(np.diff(row) > 0) and np.all(row > r)
    # edges of G+(u) summed over u = triangles
    q3, po, _ = oracle.count(g, 3, per_owner=True)
    total_edges = 0
    nbr = [set(g.adj[g.off[v]:g.off[v + 1]].tolist()) for v in range(g.n)]
    for u in range(0, g.n):
        L = oracle.gamma_plus(g, u)
        e = sum(1 for a, b in combinations(L.tolist(), 2) if b in nbr[a])
        assert e == int(po[u])
        total_edges += e
    assert total_edges == q3


def test_threads_do_not_change_results():
    g = kcgen.chung_lu(4000, 40000, 2.1, 500.0, 5)
    for k in (3, 5):
        a = oracle.count(g, k, per_owner=True, per_vertex=True, nthreads=1)
        b = oracle.count(g, k, per_owner=True, per_vertex=True, nthreads=4)
        assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_owner_range_partition_sums():
    g = kcgen.chung_lu(3000, 30000, 2.1, 300.0, 6)
    full = oracle.count(g, 4)[0]
    cuts = [0, 700, 1500, 2999, 3000]
    parts = sum(oracle.count(g, 4, u_range=(a, b))[0] for a, b in zip(cuts, cuts[1:]))
    assert parts == full


# ------------------------------------------------------------ cFFF (Sec. 6)

def test_splitmix_published_vectors():
    # splitmix64 seeded with 0 yields 0xE220A8397B1DCDAF first (Vigna's
    # reference generator); the colour hash with seed 0 and key 1 is exactly
    # that output.
    assert oracle.colour_hash(0, 0, 1) == 0xE220A8397B1DCDAF
    assert kcgen._load().kg_splitmix64_output(0) == 0xE220A8397B1DCDAF
    assert [kcgen._load().kg_splitmix64_output((1234567 + i * 0x9E3779B97F4A7C15) % 2**64)
            for i in range(3)] == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_colour_reduction():
    for (s, u, x) in [(1, 2, 3), (99, 0, 0), (2**63, 12345, 678)]:
        h = oracle.colour_hash(s, u, x)
        for c in (1, 2, 3, 10, 16, 2**31 + 7):
            assert oracle.colour(s, u, x, c) == (h * c) >> 64
        assert oracle.colour(s, u, x, 1) == 0


def test_colour_uniformity():
    c, N = 7, 70000
    counts = np.bincount([oracle.colour(42, u, u * 31 + 5, c) for u in range(N)], minlength=c)
    chi2 = float(((counts - N / c) ** 2 / (N / c)).sum())
    assert chi2 < 30.0  # 6 dof: P(chi2 > 30) ~ 4e-5


def test_one_colour_is_exact():
    g = kcgen.chung_lu(2000, 20000, 2.1, 250.0, 8)
    for k in range(2, 7):
        s, est, _ = oracle.estimate(g, k, 1, seed=5)
        assert s == oracle.count(g, k)[0]
        assert est == float(s)


def test_estimate_scaling():
    for (s, c, k) in [(0, 4, 5), (12345, 10, 3), (99, 16, 7), (2**40 + 3, 3, 6)]:
        assert oracle._load().oracle_scale_estimate(s, c, k) == float(s) * float(c ** (k - 2))


def test_hashed_colouring_equals_explicit_colouring():
    g = kcgen.chung_lu(1500, 15000, 2.1, 200.0, 9)
    k, c, seed = 4, 3, 77
    s, _, po = oracle.estimate(g, k, c, seed, per_owner=True)
    for u in range(0, g.n, 37):
        L = oracle.gamma_plus(g, u)
        col = [oracle.colour(seed, u, int(x), c) for x in L]
        assert oracle.owner_coloured(g, u, k, col) == int(po[u])
    assert int(po.sum()) == s


@pytest.mark.parametrize("k,c", [(3, 2), (4, 2), (4, 3), (5, 2)])
def test_estimator_unbiased_exhaustive(k, c):
    """E[q_u * c^(k-2)] = q_{u,k-1} exactly, over all c^d colourings of Gamma+(u)
    (the expectation claim of Sec. 6 / App. B), for owners with small d+."""
    g = kcgen.random_small(16, 0.6, 17)
    checked = 0
    for u in range(g.n):
        L = oracle.gamma_plus(g, u)
        d = len(L)
        if d < k - 1 or d > 7:
            continue
        exact = oracle.owner_coloured(g, u, k, [0] * d)
        acc = 0
        for col in product(range(c), repeat=d):
            acc += oracle.owner_coloured(g, u, k, list(col)) * c ** (k - 2)
        assert acc == exact * c ** d
        checked += 1
    assert checked >= 3


def test_estimator_mean_over_seeds():
    g = kcgen.chung_lu(2000, 20000, 2.1, 250.0, 10)
    k, c, S = 4, 4, 64
    exact = oracle.count(g, k)[0]
    ests = np.array([oracle.estimate(g, k, c, seed)[1] for seed in range(1, S + 1)])
    assert abs(ests.mean() - exact) <= 4.0 * ests.std(ddof=1) / np.sqrt(S) + 1e-9


# ---------------------------------------------------- plain pair sampling (Sec. 6)

def test_pair_threshold_is_exact_probability():
    """thr = floor(p 2^64); for p >= 2^-11 the kept fraction thr / 2^64 is p."""
    from fractions import Fraction
    for p in (0.5, 0.25, 0.1, 0.3, 0.999, 2.0 ** -11):
        thr = oracle.pair_threshold(p)
        assert Fraction(thr, 2 ** 64) == Fraction(p)


def test_pair_hash_symmetric_and_owner_dependent():
    for (u, x, y) in [(0, 1, 2), (5, 100, 7), (2**31 - 1, 0, 2**31 - 2)]:
        assert oracle.pair_hash(9, u, x, y) == oracle.pair_hash(9, u, y, x)
    hs = {oracle.pair_hash(9, u, 3, 4) for u in range(64)}
    assert len(hs) == 64
    assert oracle.pair_hash(9, 0, 3, 4) != oracle.pair_hash(10, 0, 3, 4)


def test_pair_keep_frequency():
    """Each pair is kept with probability p: 4e4 pairs, within 5 sigma."""
    p = 0.3
    thr = oracle.pair_threshold(p)
    N = 40000
    kept = sum(oracle.pair_hash(11, u, x, x + 1 + u % 7) < thr for u in range(200) for x in range(200))
    assert abs(kept - p * N) <= 5 * np.sqrt(N * p * (1 - p))


def test_pairs_p1_is_exact():
    g = kcgen.chung_lu(2000, 12000, 2.1, 200.0, 3)
    for k in (3, 4, 5):
        s, est, po = oracle.estimate_pairs(g, k, 1.0, 5, per_owner=True)
        q, qo, _ = oracle.count(g, k, per_owner=True)
        assert s == q and est == float(q) and np.array_equal(po, qo)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_pairs_brute_force(k):
    """S = number of (k-1)-subsets Q of Gamma+(u), over all u, whose pairs are
    all edges and all emitted by Map 2 (hash below the threshold) -- the
    sampled cliques of Sec. 6 -- by itertools."""
    g = kcgen.random_small(18, 0.55, 23)
    nbr = [set(g.adj[g.off[v]:g.off[v + 1]].tolist()) for v in range(g.n)]
    deg = [len(s) for s in nbr]
    p, seed = 0.6, 77
    thr = oracle.pair_threshold(p)
    S = 0
    for u in range(g.n):
        gp = [x for x in nbr[u] if (deg[u], u) < (deg[x], x)]
        for Q in combinations(gp, k - 1):
            if all(b in nbr[a] and oracle.pair_hash(seed, u, a, b) < thr for a, b in combinations(Q, 2)):
                S += 1
    s, est, _ = oracle.estimate_pairs(g, k, p, seed)
    assert s == S
    assert S > 0


@pytest.mark.parametrize("k", [3, 4])
def test_pairs_estimator_unbiased_exhaustive(k):
    """E[q_u / p^((k-1)(k-2)/2)] = q_{u,k-1} exactly over all 2^C(d,2) sets of
    emitted pairs of Gamma+(u) weighted by p^|K| (1-p)^(P-|K|) (Claim in
    App. B), with p = 1/3 in exact rationals."""
    from fractions import Fraction
    g = kcgen.random_small(14, 0.7, 5)
    p = Fraction(1, 3)
    e = (k - 1) * (k - 2) // 2
    checked = 0
    for u in range(g.n):
        d = len(oracle.gamma_plus(g, u))
        if d < k - 1 or d > 5:
            continue
        pairs = [(i, j) for i in range(d) for j in range(i + 1, d)]
        P = len(pairs)
        exact = oracle.owner_pairs(g, u, k, np.ones((d, d), np.uint8))
        acc = Fraction(0)
        for bits in range(1 << P):
            kept = np.zeros((d, d), np.uint8)
            nk = 0
            for t, (i, j) in enumerate(pairs):
                if bits >> t & 1:
                    kept[i, j] = 1
                    nk += 1
            acc += p ** nk * (1 - p) ** (P - nk) * oracle.owner_pairs(g, u, k, kept)
        assert acc / p ** e == exact
        checked += 1
    assert checked >= 3


def test_pairs_hashed_equals_explicit():
    """The hashed Map 2 filter equals the explicit kept-pair matrix built from
    the same hash, owner by owner."""
    g = kcgen.random_small(30, 0.5, 8)
    k, p, seed = 4, 0.5, 3
    thr = oracle.pair_threshold(p)
    _, _, po = oracle.estimate_pairs(g, k, p, seed, per_owner=True)
    for u in range(g.n):
        L = oracle.gamma_plus(g, u)
        d = len(L)
        kept = np.zeros((max(d, 1), max(d, 1)), np.uint8)
        for i in range(d):
            for j in range(i + 1, d):
                kept[i, j] = oracle.pair_hash(seed, u, int(L[i]), int(L[j])) < thr
        assert oracle.owner_pairs(g, u, k, kept) == int(po[u])


def test_pairs_scaling():
    """fl(S) / p^e, e = (k-1)(k-2)/2: with p = 1/2 the scale is exactly 2^e."""
    g = kcgen.chung_lu(2000, 12000, 2.1, 200.0, 3)
    for k in (3, 4, 5, 6):
        e = (k - 1) * (k - 2) // 2
        s, est, _ = oracle.estimate_pairs(g, k, 0.5, 1)
        assert est == s * 2.0 ** e


def test_pairs_mean_over_seeds():
    g = kcgen.chung_lu(2000, 20000, 2.1, 250.0, 10)
    k, p, S = 4, 0.5, 64
    exact = oracle.count(g, k)[0]
    ests = np.array([oracle.estimate_pairs(g, k, p, seed)[1] for seed in range(1, S + 1)])
    assert abs(ests.mean() - exact) <= 4.0 * ests.std(ddof=1) / np.sqrt(S) + 1e-9


# ------------------------------------------------------------ listing (Sec. 3)

@pytest.mark.parametrize("seed", [3, 4, 5])
def test_listing_matches_brute_force(seed):
    """Every k-clique exactly once (as a set), each row in precedence order
    with the owner first, the number of rows q_k."""
    g = kcgen.random_small(25, 0.5, seed)
    for k in (1, 2, 3, 4, 5, 6):
        L = oracle.list_cliques(g, k)
        assert len(L) == oracle.count(g, k)[0]
        got = sorted(tuple(sorted(r)) for r in L.tolist())
        assert got == sorted(py_cliques(g, k))
        for r in L.tolist():
            assert all(oracle.precedes(g, r[i], r[i + 1]) for i in range(k - 1))


def test_listing_complete_graph():
    g = kcgen.complete(12)
    for k in (3, 5, 12):
        L = oracle.list_cliques(g, k)
        assert len(L) == comb(12, k)
        assert len({tuple(sorted(r)) for r in L.tolist()}) == comb(12, k)


def test_count_owners_matches_per_owner_and_closed_form():
    """oracle.count_owners (explicit owner lists) agrees with the per-owner
    output of the full count, and with K_n's closed form: the vertex of rank
    r owns C(n-1-r, k-1) k-cliques (Sec. 3: each clique counted by its
    smallest vertex)."""
    g = kcgen.chung_lu(3000, 20000, 2.1, 300.0, 2)
    rng = np.random.default_rng(1)
    for k in (1, 2, 3, 4, 5):
        _, po, _ = oracle.count(g, k, per_owner=True)
        own = rng.choice(g.n, 300, replace=False)
        assert np.array_equal(oracle.count_owners(g, k, own), po[own]), k
    kn = kcgen.complete(20)
    for k in (3, 6):
        got = oracle.count_owners(kn, k, np.arange(20))
        assert [int(x) for x in got] == [comb(19 - r, k - 1) for r in range(20)]
