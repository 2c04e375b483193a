"""CPU oracle for k-clique counting (FFF_k), colour sampling (cFFF_k) and
plain pair sampling (Sec. 6).

TEST INFRASTRUCTURE: only tests/, the smoke check and the benchmark's
CPU-baseline leg import this package.  It shares no code with the CUDA
library (paper_1403_0734_gb300); neither imports the other.  The arithmetic
lives in kc_oracle.c (plain C, one owner at a time, following the paper's
rounds); this module only marshals numpy arrays.

Parity pins: see tests/test_oracle.py.  Functions whose result has no pin
beyond this oracle itself: none for counts; the paper's App. C counts of the
SNAP graphs are unpinned because the graphs are not available.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
P = ctypes.c_void_p
U64P = ctypes.POINTER(ctypes.c_uint64)

STATUS = {0: "ok", 1: "overflow", 2: "invalid argument", 3: "out of memory"}


class OracleError(RuntimeError):
    pass


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(_build.build())
    lib.oracle_precedes.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
    lib.oracle_precedes.restype = ctypes.c_int
    lib.oracle_order.argtypes = [P, ctypes.c_int32, P]
    lib.oracle_order.restype = ctypes.c_int
    lib.oracle_gamma_plus.argtypes = [P, P, ctypes.c_int32, P]
    lib.oracle_gamma_plus.restype = ctypes.c_int32
    lib.oracle_colour_hash.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32]
    lib.oracle_colour_hash.restype = ctypes.c_uint64
    lib.oracle_colour.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32]
    lib.oracle_colour.restype = ctypes.c_uint32
    lib.oracle_fff.argtypes = [P, P, ctypes.c_int32, ctypes.c_int, ctypes.c_uint32,
                               ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                               U64P, U64P, P, P]
    lib.oracle_fff.restype = ctypes.c_int
    lib.oracle_fff_owners.argtypes = [P, P, ctypes.c_int32, ctypes.c_int, P, ctypes.c_int32, ctypes.c_int, P]
    lib.oracle_fff_owners.restype = ctypes.c_int
    lib.oracle_owner_coloured.argtypes = [P, P, ctypes.c_int32, ctypes.c_int, P, U64P, U64P]
    lib.oracle_owner_coloured.restype = ctypes.c_int
    lib.oracle_scale_estimate.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int]
    lib.oracle_scale_estimate.restype = ctypes.c_double
    lib.oracle_pair_hash.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    lib.oracle_pair_hash.restype = ctypes.c_uint64
    lib.oracle_pair_threshold.argtypes = [ctypes.c_double]
    lib.oracle_pair_threshold.restype = ctypes.c_uint64
    lib.oracle_scale_pairs.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_int]
    lib.oracle_scale_pairs.restype = ctypes.c_double
    lib.oracle_fff_pairs.argtypes = [P, P, ctypes.c_int32, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_int, U64P, U64P, P]
    lib.oracle_fff_pairs.restype = ctypes.c_int
    lib.oracle_owner_pairs.argtypes = [P, P, ctypes.c_int32, ctypes.c_int, P, U64P, U64P]
    lib.oracle_owner_pairs.restype = ctypes.c_int
    lib.oracle_list.argtypes = [P, P, ctypes.c_int32, ctypes.c_int, P, ctypes.c_int64,
                                ctypes.POINTER(ctypes.c_int64)]
    lib.oracle_list.restype = ctypes.c_int
    lib.oracle_brute_force.argtypes = [P, P, ctypes.c_int32, ctypes.c_int, U64P, U64P, P]
    lib.oracle_brute_force.restype = ctypes.c_int
    lib.oracle_max_threads.argtypes = [ctypes.c_int]
    lib.oracle_max_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _csr(g):
    off = np.ascontiguousarray(g.off, dtype=np.int64)
    adj = np.ascontiguousarray(g.adj, dtype=np.int32)
    if adj.size == 0:
        adj = np.zeros(1, dtype=np.int32)
    return off, adj


def _check(st):
    if st != 0:
        raise OracleError(f"oracle: {STATUS.get(st, st)}")


def precedes(g, x: int, y: int) -> bool:
    off, _ = _csr(g)
    return bool(_load().oracle_precedes(off.ctypes.data, x, y))


def order(g) -> np.ndarray:
    """Vertices in increasing precedence (degree, then id)."""
    off, _ = _csr(g)
    out = np.empty(max(g.n, 1), dtype=np.int32)
    _check(_load().oracle_order(off.ctypes.data, g.n, out.ctypes.data))
    return out[: g.n]


def gamma_plus(g, u: int) -> np.ndarray:
    """Gamma+(u) in increasing precedence (original ids)."""
    off, adj = _csr(g)
    d = int(off[u + 1] - off[u])
    out = np.empty(max(d, 1), dtype=np.int32)
    ln = _load().oracle_gamma_plus(off.ctypes.data, adj.ctypes.data, u, out.ctypes.data)
    if ln < 0:
        raise OracleError("oracle: out of memory")
    return out[:ln]


def oriented(g):
    """Oriented CSR in rank space, as the oracle defines it: row r lists the
    ranks of Gamma+(order[r]) ascending.  Returns (order, rank, off_plus, adj_plus)."""
    perm = order(g)
    rank = np.empty(g.n, dtype=np.int64)
    rank[perm] = np.arange(g.n)
    rows = [np.sort(rank[gamma_plus(g, int(perm[r]))]) for r in range(g.n)]
    lens = np.array([len(x) for x in rows], dtype=np.int64)
    offp = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(lens, out=offp[1:])
    adjp = np.concatenate(rows).astype(np.int32) if rows and offp[-1] > 0 else np.zeros(0, np.int32)
    return perm, rank.astype(np.int32), offp, adjp


def colour_hash(seed: int, u: int, x: int) -> int:
    return int(_load().oracle_colour_hash(seed, u, x))


def colour(seed: int, u: int, x: int, c: int) -> int:
    return int(_load().oracle_colour(seed, u, x, c))


def _fff(g, k, colours, seed, per_owner, per_vertex, u_range, nthreads):
    off, adj = _csr(g)
    lo, hi = (0, g.n) if u_range is None else u_range
    po = np.zeros(max(g.n, 1), dtype=np.uint64) if per_owner else None
    pv = np.zeros(max(g.n, 1), dtype=np.uint64) if per_vertex else None
    tlo, thi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = _load().oracle_fff(off.ctypes.data, adj.ctypes.data, g.n, k, colours, seed, lo, hi,
                            nthreads, ctypes.byref(tlo), ctypes.byref(thi),
                            po.ctypes.data if po is not None else None,
                            pv.ctypes.data if pv is not None else None)
    _check(st)
    total = (int(thi.value) << 64) | int(tlo.value)
    return total, (po[: g.n] if po is not None else None), (pv[: g.n] if pv is not None else None)


def count(g, k: int, per_owner: bool = False, per_vertex: bool = False,
          u_range=None, nthreads: int = 0):
    """Exact FFF_k: returns (q_k, per_owner or None, per_vertex or None).
    u_range=(lo, hi) restricts the owners u to original ids lo..hi-1."""
    return _fff(g, k, 0, 0, per_owner, per_vertex, u_range, nthreads)


def count_owners(g, k: int, owners, nthreads: int = 0) -> np.ndarray:
    """Exact per-owner counts q_{u,k-1} for an explicit list of owners (the
    same Reduce 3 routine as count(), one owner per thread): out[i] is the
    count of owners[i]."""
    off, adj = _csr(g)
    own = np.ascontiguousarray(owners, dtype=np.int32)
    out = np.zeros(max(own.size, 1), dtype=np.uint64)
    _check(_load().oracle_fff_owners(off.ctypes.data, adj.ctypes.data, g.n, k,
                                     own.ctypes.data if own.size else None, int(own.size), nthreads,
                                     out.ctypes.data))
    return out[: own.size]


def estimate(g, k: int, colours: int, seed: int, per_owner: bool = False,
             u_range=None, nthreads: int = 0):
    """cFFF_k: returns (sampled count S, estimate S * c^(k-2), per_owner S_u)."""
    if colours < 1:
        raise ValueError("colours >= 1")
    s, po, _ = _fff(g, k, colours, seed, per_owner, False, u_range, nthreads)
    return s, float(_load().oracle_scale_estimate(s, colours, k)), po


def owner_coloured(g, u: int, k: int, colours_of_gamma_plus) -> int:
    """Reduce 3's count for owner u under an explicit colouring of Gamma+(u)."""
    off, adj = _csr(g)
    col = np.ascontiguousarray(colours_of_gamma_plus, dtype=np.uint32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.uint32)
    lo, hi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(_load().oracle_owner_coloured(off.ctypes.data, adj.ctypes.data, u, k,
                                         col.ctypes.data, ctypes.byref(lo), ctypes.byref(hi)))
    return (int(hi.value) << 64) | int(lo.value)


def pair_hash(seed: int, u: int, x: int, y: int) -> int:
    return int(_load().oracle_pair_hash(seed, u, x, y))


def pair_threshold(p: float) -> int:
    return int(_load().oracle_pair_threshold(p))


def estimate_pairs(g, k: int, p: float, seed: int, per_owner: bool = False, u_range=None, nthreads: int = 0):
    """Plain pair sampling (Sec. 6): returns (sampled count S,
    estimate S / p^((k-1)(k-2)/2), per_owner S_u or None)."""
    off, adj = _csr(g)
    lo, hi = (0, g.n) if u_range is None else u_range
    po = np.zeros(max(g.n, 1), dtype=np.uint64) if per_owner else None
    tlo, thi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(_load().oracle_fff_pairs(off.ctypes.data, adj.ctypes.data, g.n, k, float(p), seed, lo, hi, nthreads,
                                    ctypes.byref(tlo), ctypes.byref(thi),
                                    po.ctypes.data if po is not None else None))
    s = (int(thi.value) << 64) | int(tlo.value)
    return s, float(_load().oracle_scale_pairs(s, float(p), k)), (po[: g.n] if po is not None else None)


def owner_pairs(g, u: int, k: int, kept) -> int:
    """Reduce 3's count for owner u when Map 2 emitted exactly the pairs (i, j),
    i < j, with kept[i, j] set (indices of Gamma+(u) in precedence order)."""
    off, adj = _csr(g)
    kept = np.ascontiguousarray(kept, dtype=np.uint8)
    if kept.size == 0:
        kept = np.zeros(1, dtype=np.uint8)
    lo, hi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(_load().oracle_owner_pairs(off.ctypes.data, adj.ctypes.data, u, k, kept.ctypes.data,
                                      ctypes.byref(lo), ctypes.byref(hi)))
    return (int(hi.value) << 64) | int(lo.value)


def list_cliques(g, k: int) -> np.ndarray:
    """Every k-clique as a row of k ids in precedence order, owner first
    (Reduce 3's enumeration, Sec. 3); rows in owner-id order."""
    off, adj = _csr(g)
    cnt = ctypes.c_int64(0)
    _check(_load().oracle_list(off.ctypes.data, adj.ctypes.data, g.n, k, None, 0, ctypes.byref(cnt)))
    out = np.zeros((max(cnt.value, 1), k), dtype=np.int32)
    _check(_load().oracle_list(off.ctypes.data, adj.ctypes.data, g.n, k, out.ctypes.data, cnt.value,
                               ctypes.byref(cnt)))
    return out[: cnt.value]


def brute_force(g, k: int, per_vertex: bool = False):
    """q_k by testing every k-subset (n <= 4096)."""
    off, adj = _csr(g)
    pv = np.zeros(max(g.n, 1), dtype=np.uint64) if per_vertex else None
    lo, hi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(_load().oracle_brute_force(off.ctypes.data, adj.ctypes.data, g.n, k,
                                      ctypes.byref(lo), ctypes.byref(hi),
                                      pv.ctypes.data if pv is not None else None))
    total = (int(hi.value) << 64) | int(lo.value)
    return total, (pv[: g.n] if pv is not None else None)


def max_threads(nthreads: int = 0) -> int:
    return int(_load().oracle_max_threads(nthreads))
