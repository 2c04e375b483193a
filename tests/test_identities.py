"""Counting identities the GPU path relies on, checked by brute force on
small random graphs (no oracle and no CUDA involved).

The ordered search closes a dense candidate set C that still needs three
vertices through the complement of G[C] (per-vertex mode): with c = |C|,
d_v the degree of v in G[C], nb_v = c - 1 - d_v, X_v the non-neighbours of
v in C and M the number of non-edges of G[C], the triangles of G[C] through
v number

    t_v = C(d_v, 2) - M + nb_v + sum_{a in X_v} (nb_a - 1) - nonedges(X_v).

(The triangles through v are the edges inside N(v): C(d_v, 2) pairs less
the non-edges among them, and every non-edge of G[C] either touches v,
lies inside N(v), or has an end in X_v.)  The per-clique memberships and the
total sum_v t_v / 3 of the k-clique count follow from it.

The second identity (4-cliques through each vertex of a dense graph, from
its sparse complement) is not used by the kernels yet; it is pinned here as
the basis of the next level of the complement count.
"""
import itertools

import numpy as np
import pytest


def triangles_through(A):
    n = A.shape[0]
    t = np.zeros(n, dtype=np.int64)
    for a, b, c in itertools.combinations(range(n), 3):
        if A[a, b] and A[a, c] and A[b, c]:
            t[[a, b, c]] += 1
    return t


def complement_formula(A):
    n = A.shape[0]
    deg = A.sum(axis=1)
    nb = n - 1 - deg
    M = int(nb.sum()) // 2
    out = np.zeros(n, dtype=np.int64)
    for v in range(n):
        X = [a for a in range(n) if a != v and not A[v, a]]
        s1 = sum(int(nb[a]) - 1 for a in X)
        ne = sum(1 for a, b in itertools.combinations(X, 2) if not A[a, b])
        out[v] = int(deg[v]) * (int(deg[v]) - 1) // 2 - (M - int(nb[v]) - s1 + ne)
    return out


@pytest.mark.parametrize("seed", range(12))
def test_complement_triangle_identity(seed):
    rng = np.random.default_rng(seed)
    for n in (3, 5, 9, 17, 33):
        for p in (0.5, 0.8, 0.95, 1.0):
            U = np.triu(rng.random((n, n)) < p, 1)
            A = (U | U.T).astype(np.int64)
            t = triangles_through(A)
            assert np.array_equal(complement_formula(A), t), (seed, n, p)
            assert int(t.sum()) % 3 == 0


def test_complement_identity_special_cases():
    # complete graph: no non-edges, t_v = C(n-1, 2)
    n = 12
    A = np.ones((n, n), dtype=np.int64) - np.eye(n, dtype=np.int64)
    assert np.all(complement_formula(A) == (n - 1) * (n - 2) // 2)
    # complete multipartite K_{3,3,3}: t_v = 3 * 3 (one vertex from each other part)
    lab = np.repeat(np.arange(3), 3)
    A = (lab[:, None] != lab[None, :]).astype(np.int64)
    assert np.all(complement_formula(A) == 9)
    # empty graph: no triangles
    A = np.zeros((7, 7), dtype=np.int64)
    assert np.all(complement_formula(A) == 0)


# --- the next level: 4-cliques through each vertex of a dense graph -------
#
# Not used by the kernels yet.  It is the identity a first-level complement
# count would rest on (k = 6 closed per first-level vertex e1 instead of per
# pair (e1, e2)).  K_v = sum over edge sets F of the complement with
# |V(F) + v| = j <= 4 of (-1)^|F| C(c - j, 4 - j).  Grouping F by shape gives
# terms in n̄ (complement degrees), M (complement edges), cherries,
# triangles and 3-edge paths of the complement around v, plus, for each
# 4-set q through v with e_q >= 4 complement edges inside,
# C(e_q, 4) - C(e_q, 5) + C(e_q, 6).

def k4_through_complement(A):
    from math import comb
    n = A.shape[0]
    B = (~A.astype(bool)) & ~np.eye(n, dtype=bool)
    X = [np.flatnonzero(B[i]).tolist() for i in range(n)]
    nb = [len(x) for x in X]
    M = sum(nb) // 2
    P = sum(comb(d, 2) for d in nb)  # cherries (2-paths) of the complement
    tri = np.zeros(n, dtype=np.int64)
    for a, b, c in itertools.combinations(range(n), 3):
        if B[a, b] and B[a, c] and B[b, c]:
            tri[[a, b, c]] += 1
    T = int(tri.sum()) // 3
    c = n
    out = np.zeros(n, dtype=np.int64)
    for v in range(n):
        Xv = X[v]
        s1 = sum(nb[a] - 1 for a in Xv)
        K = comb(c - 1, 3) - nb[v] * comb(c - 2, 2) - (M - nb[v]) * (c - 3)        # |F| = 0, 1
        K += (comb(nb[v], 2) + s1) * (c - 3)                                      # |F| = 2 on 3 vertices
        K += sum(M - nb[v] - nb[a] + 1 for a in Xv) + P - comb(nb[v], 2) - s1     # |F| = 2 on 4 vertices
        K -= int(tri[v]) * (c - 3) + (T - int(tri[v]))                            # |F| = 3: triangles
        K -= comb(nb[v], 3) + sum(comb(nb[a] - 1, 2) for a in Xv)                 # |F| = 3: stars
        for a in Xv:                                                              # |F| = 3: paths
            for b in X[a]:
                if b != v:
                    K -= nb[b] - 1 - int(B[b, v])      # v - a - b - d
            for b in Xv:
                if b != a:
                    K -= nb[b] - 1 - int(B[b, a])      # a - v - b - d
        for t3 in itertools.combinations([u for u in range(n) if u != v], 3):    # |F| >= 4
            q = (v,) + t3
            e = sum(int(B[x, y]) for x, y in itertools.combinations(q, 2))
            K += comb(e, 4) - comb(e, 5) + comb(e, 6)
        out[v] = K
    return out


def k4_through_brute(A):
    n = A.shape[0]
    K = np.zeros(n, dtype=np.int64)
    for q in itertools.combinations(range(n), 4):
        if all(A[x, y] for x, y in itertools.combinations(q, 2)):
            K[list(q)] += 1
    return K


@pytest.mark.parametrize("seed", range(6))
def test_k4_complement_identity(seed):
    rng = np.random.default_rng(100 + seed)
    for n in (4, 7, 11, 15):
        for p in (0.6, 0.85, 0.95, 1.0):
            U = np.triu(rng.random((n, n)) < p, 1)
            A = (U | U.T).astype(np.int64)
            assert np.array_equal(k4_through_complement(A), k4_through_brute(A)), (seed, n, p)


def k4_through_complement_local(A):
    """The same K_v with the >= 4-edge term as subgraph counts of the
    complement through v (4-cycles, paws, diamonds, K4s), so that every term
    comes from per-vertex tables (nb, complement triangles tt, s1) and from
    pairs inside X_v -- no 4-set enumeration."""
    from math import comb
    n = A.shape[0]
    B = (~A.astype(bool)) & ~np.eye(n, dtype=bool)
    X = [set(np.flatnonzero(B[i]).tolist()) for i in range(n)]
    nb = [len(x) for x in X]
    M = sum(nb) // 2
    P = sum(comb(d, 2) for d in nb)
    tt = [sum(1 for a, b in itertools.combinations(sorted(X[w]), 2) if B[a, b]) for w in range(n)]
    T = sum(tt) // 3
    s1 = [sum(nb[a] - 1 for a in X[w]) for w in range(n)]
    c = n
    out = np.zeros(n, dtype=np.int64)
    for v in range(n):
        Xv = sorted(X[v])
        nv, t = nb[v], tt[v]
        K = comb(c - 1, 3) - nv * comb(c - 2, 2) - (M - nv) * (c - 3)
        K += (comb(nv, 2) + s1[v]) * (c - 3)
        K += nv * (M - nv + 1) - sum(nb[a] for a in Xv) + P - comb(nv, 2) - s1[v]
        K -= t * (c - 3) + (T - t) + comb(nv, 3) + sum(comb(nb[a] - 1, 2) for a in Xv)
        K -= sum(s1[a] for a in Xv) - nv * (nv - 1) + (nv - 1) * s1[v] - 4 * t   # 3-edge paths
        tris = [(a, b) for a, b in itertools.combinations(Xv, 2) if B[a, b]]
        c4 = sum(len(X[a] & X[b]) - 1 for a, b in itertools.combinations(Xv, 2))
        paw = (t * (nv - 2) + sum(nb[a] + nb[b] - 4 for a, b in tris)
               + sum(tt[a] - len(X[a] & X[v]) for a in Xv))
        dia = sum(comb(len(X[v] & X[a]), 2) for a in Xv) + sum(len(X[a] & X[b]) - 1 for a, b in tris)
        k4 = sum(len(X[v] & X[a] & X[b]) for a, b in tris) // 3
        out[v] = K + c4 + paw - dia + k4
    return out


@pytest.mark.parametrize("seed", range(6))
def test_k4_complement_local_form(seed):
    rng = np.random.default_rng(200 + seed)
    for n in (4, 8, 13, 17):
        for p in (0.5, 0.85, 0.95, 1.0):
            U = np.triu(rng.random((n, n)) < p, 1)
            A = (U | U.T).astype(np.int64)
            assert np.array_equal(k4_through_complement_local(A), k4_through_brute(A)), (seed, n, p)


def k4_word_level(rows, C):
    """The first-level complement count as a kernel would run it on bitmap
    words: X' = C & ~row(v) holds v itself, so every popcount of X' sets is
    corrected for the elements it holds (the corrections below).  Three
    passes: non-degrees (M, cherries P); S1 and complement triangles tt per
    element; then K_v from those tables and two-hop walks in the complement.
    Returns {v: K_v}, or None when G[C] is not dense (non-edges >= a quarter
    of the edges)."""
    from math import comb

    def popc(x):
        return bin(x).count("1")

    el = [v for v in range(len(rows)) if (C >> v) & 1]
    c = len(el)
    Xp = {v: C & ~rows[v] for v in el}
    nb = {v: c - 1 - popc(C & rows[v]) for v in el}
    nbsum = sum(nb.values())
    if 4 * nbsum >= c * (c - 1) - nbsum:
        return None
    M, P = nbsum // 2, sum(comb(nb[v], 2) for v in el)
    s1, tt = {}, {}
    for v in el:
        X = [a for a in el if a != v and (Xp[v] >> a) & 1]
        s1[v] = sum(nb[a] - 1 for a in X)
        tt[v] = sum(popc(Xp[v] & ~rows[a] & C) - 2 for a in X) // 2   # X' \ N(a) holds a and v
    T = sum(tt.values()) // 3
    K = {}
    for v in el:
        nv, t = nb[v], tt[v]
        sums = dict(nb=0, cnb=0, s1=0, tt=0, co=0, nbco=0, cco=0)
        W1 = W2 = W3 = 0
        for a in (a for a in el if a != v and (Xp[v] >> a) & 1):
            co = popc(Xp[v] & Xp[a]) - 2                  # |X_v & X_a|: X' sets hold v and a
            sums["nb"] += nb[a]; sums["cnb"] += comb(nb[a] - 1, 2); sums["s1"] += s1[a]; sums["tt"] += tt[a]
            sums["co"] += co; sums["nbco"] += nb[a] * co; sums["cco"] += comb(co, 2)
            for x in (x for x in el if x != a and (Xp[a] >> x) & 1):
                if x == v:
                    coxv, tri3, inv = nv, co, 0
                else:
                    inv = (Xp[v] >> x) & 1
                    coxv = popc(Xp[v] & Xp[x]) - 2 * inv
                    tri3 = popc(Xp[v] & Xp[a] & Xp[x]) - 1 - 2 * inv
                W1 += coxv - 1
                W2 += tri3
                W3 += tri3 if inv else 0
        k = comb(c - 1, 3) - nv * comb(c - 2, 2) - (M - nv) * (c - 3)
        k += (comb(nv, 2) + s1[v]) * (c - 3)
        k += nv * (M - nv + 1) - sums["nb"] + P - comb(nv, 2) - s1[v]
        k -= t * (c - 3) + (T - t) + comb(nv, 3) + sums["cnb"]
        k -= sums["s1"] - nv * (nv - 1) + (nv - 1) * s1[v] - 4 * t
        k += (W1 - nv * (nv - 1)) // 2                                   # 4-cycles
        k += t * (nv - 2) + sums["nbco"] - 4 * t + sums["tt"] - sums["co"]  # paws
        k -= sums["cco"] + W2 // 2 - t                                    # diamonds
        k += W3 // 6                                                      # K4s
        K[v] = k
    return K


@pytest.mark.parametrize("seed", range(4))
def test_k4_word_level_model(seed):
    rng = np.random.default_rng(300 + seed)
    checked = 0
    for _ in range(40):
        n = int(rng.integers(6, 20))
        p = rng.choice([0.85, 0.93, 1.0])
        U = np.triu(rng.random((n, n)) < p, 1)
        A = U | U.T
        rows = [sum(1 << j for j in range(n) if A[i, j]) for i in range(n)]
        sub = [v for v in range(n) if rng.random() < 0.75]
        if len(sub) < 4:
            continue
        K = k4_word_level(rows, sum(1 << v for v in sub))
        if K is None:
            continue
        b = k4_through_brute(A[np.ix_(sub, sub)].astype(np.int64))
        assert [K[v] for v in sub] == b.tolist()
        checked += 1
    assert checked > 10
