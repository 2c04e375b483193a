"""Seeded synthetic graph generators (shared input plumbing).

The same graphs feed the CUDA library and the CPU oracle.  This module holds
none of the clique-counting arithmetic: it only draws edges and returns a
canonical undirected simple graph in CSR form (rows sorted, both directions,
no self-loops, no repeats), which is the paper's input after its
preprocessing step (Sec. 4: "undirected", degree-labelled edges).

Workload recipes (Erdos-Renyi, Chung-Lu, stochastic block model, R-MAT) are
described in the generator docstrings; the C implementation is in kcgen.c and
is deterministic across x86-64 and aarch64.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from itertools import combinations

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.kg_free.argtypes = [P]
    lib.kg_free.restype = None
    lib.kg_n.argtypes = [P]
    lib.kg_n.restype = ctypes.c_int32
    lib.kg_m.argtypes = [P]
    lib.kg_m.restype = ctypes.c_int64
    lib.kg_off.argtypes = [P]
    lib.kg_off.restype = P
    lib.kg_adj.argtypes = [P]
    lib.kg_adj.restype = P
    lib.kg_from_edges.argtypes = [ctypes.c_int32, P, P, ctypes.c_int64]
    lib.kg_from_edges.restype = P
    lib.kg_erdos_renyi.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64]
    lib.kg_erdos_renyi.restype = P
    lib.kg_chung_lu.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64]
    lib.kg_chung_lu.restype = P
    lib.kg_sbm.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                           ctypes.c_int64, ctypes.c_uint64]
    lib.kg_sbm.restype = P
    lib.kg_rmat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_uint64]
    lib.kg_rmat.restype = P
    lib.kg_splitmix64_output.argtypes = [ctypes.c_uint64]
    lib.kg_splitmix64_output.restype = ctypes.c_uint64
    lib.kg_xoshiro_first.argtypes = [ctypes.c_uint64]
    lib.kg_xoshiro_first.restype = ctypes.c_uint64
    lib.kg_xoshiro_from_state.argtypes = [ctypes.c_uint64] * 4 + [ctypes.c_int32, P]
    lib.kg_xoshiro_from_state.restype = None
    lib.kg_pow_export.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.kg_pow_export.restype = ctypes.c_double
    _lib = lib
    return lib


@dataclass
class Graph:
    """Canonical undirected simple graph in CSR form (host numpy arrays)."""

    n: int
    m: int
    off: np.ndarray  # int64[n+1]
    adj: np.ndarray  # int32[2m]
    name: str = ""

    def degrees(self) -> np.ndarray:
        return np.diff(self.off).astype(np.int64)


def _take(ptr, name: str) -> Graph:
    lib = _load()
    if not ptr:
        raise MemoryError(f"kcgen: generator {name} failed (bad arguments or out of memory)")
    try:
        n = int(lib.kg_n(ptr))
        m = int(lib.kg_m(ptr))
        off = np.ctypeslib.as_array(ctypes.cast(lib.kg_off(ptr), ctypes.POINTER(ctypes.c_int64)),
                                    shape=(n + 1,)).copy()
        if m > 0:
            adj = np.ctypeslib.as_array(ctypes.cast(lib.kg_adj(ptr), ctypes.POINTER(ctypes.c_int32)),
                                        shape=(2 * m,)).copy()
        else:
            adj = np.zeros(0, dtype=np.int32)
    finally:
        lib.kg_free(ptr)
    return Graph(n, m, off, adj, name)


def from_edges(n: int, edges, name: str = "edges") -> Graph:
    """Canonical CSR from an edge list (pairs in either direction; self-loops
    and repeats are dropped)."""
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    src = np.ascontiguousarray(e[:, 0])
    dst = np.ascontiguousarray(e[:, 1])
    lib = _load()
    ptr = lib.kg_from_edges(int(n), src.ctypes.data, dst.ctypes.data, int(e.shape[0]))
    return _take(ptr, name)


def erdos_renyi(n: int, m: int, seed: int) -> Graph:
    """G(n, m): exactly m distinct uniform vertex pairs."""
    return _take(_load().kg_erdos_renyi(n, m, seed), f"er_n{n}_m{m}_s{seed}")


def chung_lu(n: int, m: int, gamma: float, wmax: float, seed: int) -> Graph:
    """Chung-Lu power law: weights a*(i+i0)^(-1/(gamma-1)) with max weight wmax
    and sum ~2m; m endpoint pairs drawn proportional to weight, self-loops and
    repeats dropped (realised m is a little lower), ids shuffled."""
    return _take(_load().kg_chung_lu(n, m, gamma, wmax, seed),
                 f"chunglu_n{n}_m{m}_g{gamma}_w{wmax}_s{seed}")


def sbm(n: int, block: int, p_in: float, m_total: int, seed: int) -> Graph:
    """Planted-community SBM: n/block blocks of `block` ids, intra pairs
    Bernoulli(p_in), then distinct uniform inter-block pairs up to m_total
    edges in all; ids shuffled."""
    return _take(_load().kg_sbm(n, block, p_in, m_total, seed),
                 f"sbm_n{n}_b{block}_p{p_in}_m{m_total}_s{seed}")


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int) -> Graph:
    """R-MAT with 2^scale vertices and edge_factor*2^scale draws; self-loops and
    repeats dropped; ids scrambled."""
    return _take(_load().kg_rmat(scale, edge_factor, a, b, c, seed),
                 f"rmat_s{scale}_ef{edge_factor}_s{seed}")


# --- small structured graphs (closed-form test families) -------------------

def complete(n: int) -> Graph:
    return from_edges(n, list(combinations(range(n), 2)) or np.zeros((0, 2)), f"K{n}")


def complete_multipartite(parts, shuffle_seed: int | None = None) -> Graph:
    """K_{a1,...,ar}: vertices split into parts, every cross-part pair an edge.
    With shuffle_seed, the vertex ids are permuted (numpy Generator)."""
    n = int(sum(parts))
    label = np.repeat(np.arange(len(parts)), parts)
    if shuffle_seed is not None:
        label = label[np.random.default_rng(shuffle_seed).permutation(n)]
    iu, ju = np.triu_indices(n, 1)
    keep = label[iu] != label[ju]
    e = np.stack([iu[keep], ju[keep]], axis=1)
    return from_edges(n, e, "K_" + ",".join(map(str, parts)))


def cycle(n: int) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"C{n}")


def star(n: int) -> Graph:
    return from_edges(n, [(0, i) for i in range(1, n)] or np.zeros((0, 2)), f"S{n}")


def path(n: int) -> Graph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)] or np.zeros((0, 2)), f"P{n}")


def empty(n: int) -> Graph:
    return from_edges(n, np.zeros((0, 2), dtype=np.int32), f"E{n}")


def disjoint_union(*gs: Graph) -> Graph:
    edges = []
    base = 0
    for g in gs:
        src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.off))
        edges.append(np.stack([src + base, g.adj.astype(np.int64) + base], axis=1))
        base += g.n
    e = np.concatenate(edges) if edges else np.zeros((0, 2))
    return from_edges(base, e, "+".join(g.name for g in gs))


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """Graph with vertex v renamed perm[v]."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.off))
    e = np.stack([perm[src], perm[g.adj]], axis=1)
    return from_edges(g.n, e, g.name + "_relabelled")


def random_small(n: int, p: float, seed: int) -> Graph:
    """G(n, p) for tiny test graphs (numpy Generator; not a benchmark input)."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    return from_edges(n, np.stack([iu[keep], ju[keep]], axis=1), f"gnp_{n}_{p}_{seed}")


def planted_core(n_bg: int, m_bg: int, core: int, p_core: float, seed: int, gamma: float = 2.1,
                 wmax: float = 2000.0) -> Graph:
    """A Chung-Lu power-law background (n_bg vertices, m_bg draws, exponent
    gamma, max weight wmax) with a G(core, p_core) random graph planted on
    `core` seeded-random vertices.  The planted vertices become hubs whose
    high-neighbourhoods hold hundreds of vertices but only a fraction p_core
    of the pairs, so clique counts stay moderate while |Gamma+| reaches the
    widest bitmap classes (numpy Generator for the core; not a benchmark
    input)."""
    bg = chung_lu(n_bg, m_bg, gamma, wmax, seed)
    rng = np.random.default_rng(seed)
    ids = rng.choice(n_bg, core, replace=False)
    iu, ju = np.triu_indices(core, 1)
    keep = rng.random(iu.shape[0]) < p_core
    src = np.repeat(np.arange(bg.n, dtype=np.int64), np.diff(bg.off))
    e = np.concatenate([np.stack([src, bg.adj.astype(np.int64)], axis=1),
                        np.stack([ids[iu[keep]], ids[ju[keep]]], axis=1)])
    return from_edges(n_bg, e, f"planted_cl{n_bg}_core{core}_p{p_core}_s{seed}")


# --- the five benchmark workloads -------------------------------------------

def er_1000(seed: int = 1) -> Graph:
    """Erdos-Renyi G(n=1000, m=10000), seed 1 (triangle workload)."""
    return erdos_renyi(1000, 10000, seed)


def chung_lu_1m(seed: int = 1) -> Graph:
    """Chung-Lu power law, n=10^6, 2*10^7 draws, exponent 2.1, max weight 20000."""
    return chung_lu(1_000_000, 20_000_000, 2.1, 20000.0, seed)


def sbm_2m(seed: int = 1, p_in: float = 0.3) -> Graph:
    """SBM, n=2*10^6, 40000 blocks of 50, p_in=0.3, m_total=5*10^7."""
    return sbm(2_000_000, 50, p_in, 50_000_000, seed)


# --- batched workload: many uneven Chung-Lu graphs --------------------------

def _sm64(x: int) -> int:
    """splitmix64 output for state x (integer arithmetic, platform independent)."""
    z = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def batch_params(num: int, seed: int = 1, nmin: int = 50, nmax: int = 20000, dmin: float = 8.0,
                 dmax: float = 64.0):
    """Per-graph (n, m, wmax, seed) of the batched workload: n log-uniform in
    [nmin, nmax], average degree uniform in [dmin, dmax], m = n * degree / 2,
    maximum Chung-Lu weight sqrt(2m); graph g is drawn with seed g + 1."""
    import math
    out = []
    for g in range(num):
        a = _sm64((seed << 32) ^ (2 * g)) >> 11
        b = _sm64((seed << 32) ^ (2 * g + 1)) >> 11
        u, v = a / 2.0 ** 53, b / 2.0 ** 53
        n = int(round(math.exp(math.log(nmin) + u * (math.log(nmax) - math.log(nmin)))))
        deg = dmin + v * (dmax - dmin)
        m = max(1, int(n * deg / 2))
        m = min(m, n * (n - 1) // 2)
        out.append((n, m, max(1.0, math.sqrt(2.0 * m)), g + 1))
    return out


def batch_workload(num: int, seed: int = 1, gamma: float = 2.3, **kw):
    """The uneven batch: Chung-Lu graphs (exponent gamma) with batch_params."""
    return [chung_lu(n, m, gamma, wmax, s) for (n, m, wmax, s) in batch_params(num, seed, **kw)]
