"""Generator checks (no GPU): canonical CSR form, determinism, published RNG
vectors, and the stored workload fingerprints in tests/golden/."""
import hashlib
import json
import os

import numpy as np
import pytest

import kcgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "workloads.json")


def canonical(g):
    assert g.off[0] == 0 and g.off[-1] == 2 * g.m
    deg = np.diff(g.off)
    assert np.all(deg >= 0)
    src = np.repeat(np.arange(g.n), deg)
    assert np.all(g.adj >= 0) and np.all(g.adj < g.n)
    assert np.all(src != g.adj)  # no self-loops
    # rows strictly increasing (sorted, no repeats)
    same_row = src[1:] == src[:-1]
    assert np.all(g.adj[1:][same_row] > g.adj[:-1][same_row])
    # symmetric
    a = np.sort(src.astype(np.int64) * g.n + g.adj)
    b = np.sort(g.adj.astype(np.int64) * g.n + src)
    assert np.array_equal(a, b)


def fingerprint(g):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.off).tobytes())
    h.update(np.ascontiguousarray(g.adj).tobytes())
    return h.hexdigest()


def test_xoshiro_published_vector():
    out = np.zeros(4, dtype=np.uint64)
    kcgen._load().kg_xoshiro_from_state(1, 2, 3, 4, 4, out.ctypes.data)
    assert out.tolist() == [11520, 0, 1509978240, 1215971899390074240]


def test_pow_series_accuracy():
    lib = kcgen._load()
    for x, y in [(2.0, 0.5), (10.0, -1 / 1.1), (12345.678, -0.76923), (1.0001, 3.0), (7e5, -0.9)]:
        assert abs(lib.kg_pow_export(x, y) - x ** y) <= 4e-15 * abs(x ** y)


def test_from_edges_canonicalises():
    g = kcgen.from_edges(6, [(0, 1), (1, 0), (2, 2), (3, 4), (4, 3), (5, 0), (0, 5), (1, 2)])
    canonical(g)
    assert g.m == 4


@pytest.mark.parametrize("make", [lambda: kcgen.erdos_renyi(500, 3000, 3),
                                  lambda: kcgen.chung_lu(5000, 40000, 2.1, 500.0, 2),
                                  lambda: kcgen.sbm(2000, 50, 0.3, 20000, 4),
                                  lambda: kcgen.rmat(10, 16, 0.57, 0.19, 0.19, 5)])
def test_generators_canonical_and_deterministic(make):
    g1, g2 = make(), make()
    canonical(g1)
    assert fingerprint(g1) == fingerprint(g2)


def test_er_exact_edge_count():
    g = kcgen.er_1000()
    assert g.n == 1000 and g.m == 10000


def test_sbm_structure():
    g = kcgen.sbm(5000, 50, 1.0, 0, 6)   # disjoint K_50 blocks, ids shuffled
    assert g.m == 100 * 50 * 49 // 2
    assert np.all(np.diff(g.off) == 49)


def test_golden_fingerprints():
    """Generators give the same graphs on every machine (x86-64 and aarch64)."""
    with open(GOLDEN) as f:
        gold = json.load(f)
    for entry in gold["graphs"]:
        g = getattr(kcgen, entry["maker"])(*entry["args"])
        assert g.n == entry["n"] and g.m == entry["m"], entry["name"]
        assert fingerprint(g) == entry["sha256"], entry["name"]
