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
