"""Thin ctypes binding of libkc (include/kc.h).

Argument marshalling only: every step of the counting path runs in the CUDA
kernels behind the C ABI.  Host inputs are numpy arrays; device inputs are
torch CUDA tensors (PyTorch is used for device memory and streams only).
The binding refuses to run without the compiled library -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkc.so")

KC_OK, KC_EINVAL, KC_ENOMEM, KC_EOVERFLOW, KC_ETIMEOUT, KC_ECUDA, KC_ENOTSUP, KC_ECANCELED = range(8)
KC_DEVICE_PTRS = 0x1
KC_VALIDATE = 0x2
KC_MAX_K = 32
KC_PARAM_SMEM_MAX_WORDS = 1
KC_PARAM_LAUNCH_COUNT = 2
KC_PARAM_WORK_COUNT = 3
KC_PARAM_ALGO = 4
KC_PARAM_COMPACT_LO = 5
KC_PARAM_COMPACT_HI = 6
KC_PARAM_TRI = 7
KC_PARAM_COMPLEMENT = 8
KC_ALGO_PIVOT = 0
KC_ALGO_DFS = 1
KC_TUNE_PER_VERTEX = 0x10
CLASS_NAMES = ("global", "w32", "w16", "w8", "w4", "w2", "w1")  # owner classes, launch order

_P = ctypes.c_void_p
_lib = None


class KcError(RuntimeError):
    def __init__(self, status: int, what: str):
        lib = _load()
        msg = lib.kc_strerror(status).decode()
        if status == KC_ECUDA:
            msg += ": " + lib.kc_last_cuda_error().decode()
        super().__init__(f"{what}: {msg}")
        self.status = status


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int64), ("max_dplus", ctypes.c_int32),
                ("wedges", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class _Tuning(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("per_vertex", ctypes.c_int32), ("algo", ctypes.c_int32 * 7),
                ("parts", ctypes.c_int32 * 7), ("ms", ctypes.c_float * 7)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    lib.kc_strerror.argtypes = [ctypes.c_int]
    lib.kc_strerror.restype = ctypes.c_char_p
    lib.kc_last_cuda_error.argtypes = []
    lib.kc_last_cuda_error.restype = ctypes.c_char_p
    lib.kc_version.argtypes = []
    lib.kc_version.restype = ctypes.c_char_p
    lib.kc_build_csr.argtypes = [ctypes.c_int32, _P, _P, ctypes.c_int64, _P, _P, _P]
    lib.kc_build_csr.restype = st
    lib.kc_orient.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint, _P, ctypes.POINTER(_P)]
    lib.kc_orient.restype = st
    lib.kc_free.argtypes = [_P]
    lib.kc_free.restype = None
    lib.kc_info.argtypes = [_P, ctypes.POINTER(_Info)]
    lib.kc_info.restype = st
    lib.kc_export.argtypes = [_P, ctypes.c_uint, _P, _P, _P, _P, _P, _P]
    lib.kc_export.restype = st
    lib.kc_count.argtypes = [_P, ctypes.c_int, ctypes.c_uint, _P, _P, _P, _P]
    lib.kc_count.restype = st
    lib.kc_estimate.argtypes = [_P, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint, _P, _P, _P, _P]
    lib.kc_estimate.restype = st
    lib.kc_estimate_pairs.argtypes = [_P, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint, _P, _P, _P,
                                      _P]
    lib.kc_estimate_pairs.restype = st
    lib.kc_list.argtypes = [_P, ctypes.c_int, ctypes.c_uint, _P, ctypes.c_int64, LIST_FN, _P,
                            ctypes.POINTER(ctypes.c_uint64), _P]
    lib.kc_list.restype = st
    lib.kc_count_csr.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int, ctypes.c_uint, _P, _P, _P, _P]
    lib.kc_count_csr.restype = st
    lib.kc_estimate_csr.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                                    ctypes.c_uint64, ctypes.c_uint, _P, _P, _P]
    lib.kc_estimate_csr.restype = st
    lib.kc_footprint.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]
    lib.kc_footprint.restype = st
    lib.kc_count_part.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint, _P, _P, _P, _P]
    lib.kc_count_part.restype = st
    lib.kc_count_batch.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_uint, _P, _P]
    lib.kc_count_batch.restype = st
    lib.kc_count_static.argtypes = [_P, ctypes.c_int, ctypes.c_uint, _P, _P]
    lib.kc_count_static.restype = st
    lib.kc_batch_create.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_uint, _P, ctypes.POINTER(_P)]
    lib.kc_batch_create.restype = st
    lib.kc_batch_count.argtypes = [_P, _P, _P]
    lib.kc_batch_count.restype = st
    lib.kc_batch_free.argtypes = [_P]
    lib.kc_batch_free.restype = None
    lib.kc_round2_bytes.argtypes = [_P, ctypes.c_int, _P, _P]
    lib.kc_round2_bytes.restype = st
    lib.kc_tune.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_uint, _P, ctypes.POINTER(_Tuning)]
    lib.kc_tune.restype = st
    lib.kc_set_tuning.argtypes = [_P, ctypes.POINTER(_Tuning)]
    lib.kc_set_tuning.restype = st
    lib.kc_set_param.argtypes = [ctypes.c_int, ctypes.c_int64]
    lib.kc_set_param.restype = st
    lib.kc_get_param.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
    lib.kc_get_param.restype = st
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != KC_OK:
        raise KcError(status, what)


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a):
    if a is None:
        return None
    if _is_device(a):
        return a.data_ptr()
    return a.ctypes.data


def set_param(param: int, value: int):
    _check(_load().kc_set_param(param, value), "kc_set_param")


def get_param(param: int) -> int:
    v = ctypes.c_int64(0)
    _check(_load().kc_get_param(param, ctypes.byref(v)), "kc_get_param")
    return int(v.value)


def version() -> str:
    return _load().kc_version().decode()


def build_csr(n: int, src, dst):
    """Canonical CSR (symmetric, simple, sorted rows) from an edge list (host)."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    ne = int(src.shape[0])
    off = np.zeros(n + 1, dtype=np.int64)
    adj = np.empty(max(2 * ne, 1), dtype=np.int32)
    m = ctypes.c_int64(0)
    _check(_load().kc_build_csr(n, src.ctypes.data if ne else None, dst.ctypes.data if ne else None, ne,
                                off.ctypes.data, adj.ctypes.data, ctypes.byref(m)), "kc_build_csr")
    return off, adj[: 2 * m.value].copy(), int(m.value)


class Graph:
    """An oriented graph resident on the device (owns a kc_graph handle)."""

    def __init__(self, handle: int):
        self._h = handle
        info = _Info()
        _check(_load().kc_info(handle, ctypes.byref(info)), "kc_info")
        self.n = int(info.n)
        self.m = int(info.m)
        self.max_dplus = int(info.max_dplus)
        self.wedges = int(info.wedges)
        self.device_bytes = int(info.device_bytes)

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("graph already freed")
        return self._h

    def free(self):
        if self._h:
            _load().kc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def orient(off, adj, n: int | None = None, m: int | None = None, validate: bool = False, stream=None) -> Graph:
    """Round 1: degrees, (degree, id) order and Gamma+ lists on the device.
    off/adj are numpy arrays (host) or torch CUDA tensors (device)."""
    dev = _is_device(off)
    n = int(off.shape[0] - 1) if n is None else n
    m = int(adj.shape[0] // 2) if m is None else m
    if not dev:
        off = np.ascontiguousarray(off, dtype=np.int64)
        adj = np.ascontiguousarray(adj, dtype=np.int32)
    flags = (KC_DEVICE_PTRS if dev else 0) | (KC_VALIDATE if validate else 0)
    h = _P()
    _check(_load().kc_orient(_ptr(off), _ptr(adj) if m > 0 else None, n, m, flags,
                             _stream_handle(stream), ctypes.byref(h)), "kc_orient")
    return Graph(h.value)


def export(g: Graph, stream=None) -> dict:
    """Copy the oriented graph to the host: rank, perm, off_plus, adj_plus, queue."""
    n, m = g.n, g.m
    out = {"rank": np.empty(max(n, 1), np.int32), "perm": np.empty(max(n, 1), np.int32),
           "off_plus": np.empty(n + 1, np.int64), "adj_plus": np.empty(max(m, 1), np.int32),
           "queue": np.empty(max(n, 1), np.int32)}
    _check(_load().kc_export(g.handle, 0, out["rank"].ctypes.data, out["perm"].ctypes.data,
                             out["off_plus"].ctypes.data, out["adj_plus"].ctypes.data,
                             out["queue"].ctypes.data, _stream_handle(stream)), "kc_export")
    return {"rank": out["rank"][:n], "perm": out["perm"][:n], "off_plus": out["off_plus"],
            "adj_plus": out["adj_plus"][:m], "queue": out["queue"][:n]}


def count(g: Graph, k: int, per_vertex: bool = False, per_owner: bool = False, stream=None,
          out_pv=None, out_po=None):
    """FFF_k on the device.  Returns (q_k, per_vertex or None, per_owner or None)
    with host numpy uint64 arrays indexed by the caller's vertex ids.  out_pv /
    out_po: optional preallocated host uint64 arrays of n (e.g. pinned)."""
    if out_pv is not None:
        pv = out_pv
    else:
        pv = np.empty(max(g.n, 1), np.uint64) if per_vertex else None
    if out_po is not None:
        po = out_po
    else:
        po = np.empty(max(g.n, 1), np.uint64) if per_owner else None
    tot = ctypes.c_uint64(0)
    _check(_load().kc_count(g.handle, k, 0, ctypes.byref(tot), _ptr(pv), _ptr(po), _stream_handle(stream)),
           f"kc_count(k={k})")
    return int(tot.value), (pv[: g.n] if pv is not None else None), (po[: g.n] if po is not None else None)


def round2_bytes(g: Graph, k: int, stream=None) -> int:
    """Bytes of Gamma+ lists and offsets a count at k reads to build every
    G+(u) (kc_round2_bytes): the Round 2 input volume."""
    b = ctypes.c_uint64(0)
    _check(_load().kc_round2_bytes(g.handle, k, ctypes.byref(b), _stream_handle(stream)), "kc_round2_bytes")
    return int(b.value)


def footprint(g: Graph, k: int, per_vertex: bool = False, per_owner: bool = False,
              host_outputs: bool = True) -> int:
    """Device bytes a count/estimate call allocates while it runs (kc_footprint)."""
    b = ctypes.c_uint64(0)
    _check(_load().kc_footprint(g.handle, k, int(per_vertex), int(per_owner), int(host_outputs), ctypes.byref(b)),
           "kc_footprint")
    return int(b.value)


def count_part(g: Graph, k: int, part: int, nparts: int, per_vertex: bool = False, per_owner: bool = False,
               stream=None):
    """The share of FFF_k counted by owners part, part+nparts, ... of the work
    queue (kc_count_part).  Summing the parts gives count()."""
    pv = np.empty(max(g.n, 1), np.uint64) if per_vertex else None
    po = np.empty(max(g.n, 1), np.uint64) if per_owner else None
    tot = ctypes.c_uint64(0)
    _check(_load().kc_count_part(g.handle, k, part, nparts, 0, ctypes.byref(tot), _ptr(pv), _ptr(po),
                                 _stream_handle(stream)), f"kc_count_part(k={k}, {part}/{nparts})")
    return int(tot.value), (pv[: g.n] if pv is not None else None), (po[: g.n] if po is not None else None)


def count_part_device(g: Graph, k: int, part: int, nparts: int, total, per_vertex=None, per_owner=None,
                      stream=None):
    """Asynchronous kc_count_part into device tensors (as count_device)."""
    _check(_load().kc_count_part(g.handle, k, part, nparts, KC_DEVICE_PTRS, _ptr(total), _ptr(per_vertex),
                                 _ptr(per_owner), _stream_handle(stream)), f"kc_count_part(k={k}, {part}/{nparts})")


def count_batch(graphs, k: int, stream=None):
    """q_k of every graph in one launch sequence (kc_count_batch)."""
    hs = (_P * max(len(graphs), 1))(*[gr.handle for gr in graphs])
    out = np.zeros(max(len(graphs), 1), np.uint64)
    _check(_load().kc_count_batch(hs, len(graphs), k, 0, out.ctypes.data, _stream_handle(stream)),
           f"kc_count_batch(k={k})")
    return [int(x) for x in out[: len(graphs)]]


def count_device(g: Graph, k: int, total, per_vertex=None, per_owner=None, stream=None):
    """Asynchronous FFF_k into device tensors: total (2 x int64: lo, hi words of
    the uint64 count, hi != 0 means overflow), per_vertex/per_owner (n x int64,
    read as uint64)."""
    _check(_load().kc_count(g.handle, k, KC_DEVICE_PTRS, _ptr(total), _ptr(per_vertex), _ptr(per_owner),
                            _stream_handle(stream)), f"kc_count(k={k})")


def estimate(g: Graph, k: int, colours: int, seed: int, per_owner: bool = False, stream=None):
    """cFFF_k on the device.  Returns (sampled S, estimate S*c^(k-2), per_owner or None)."""
    po = np.empty(max(g.n, 1), np.uint64) if per_owner else None
    s = ctypes.c_uint64(0)
    est = ctypes.c_double(0.0)
    _check(_load().kc_estimate(g.handle, k, colours, seed, 0, ctypes.byref(s), ctypes.byref(est), _ptr(po),
                               _stream_handle(stream)), f"kc_estimate(k={k}, c={colours})")
    return int(s.value), float(est.value), (po[: g.n] if po is not None else None)


def estimate_pairs(g: Graph, k: int, p: float, seed: int, per_owner: bool = False, stream=None):
    """Plain pair sampling on the device (Sec. 6): every pair of Gamma+(u) is
    kept with probability p.  Returns (sampled S, estimate S / p^((k-1)(k-2)/2),
    per_owner or None)."""
    po = np.empty(max(g.n, 1), np.uint64) if per_owner else None
    s = ctypes.c_uint64(0)
    est = ctypes.c_double(0.0)
    _check(_load().kc_estimate_pairs(g.handle, k, float(p), seed, 0, ctypes.byref(s), ctypes.byref(est), _ptr(po),
                                     _stream_handle(stream)), f"kc_estimate_pairs(k={k}, p={p})")
    return int(s.value), float(est.value), (po[: g.n] if po is not None else None)


LIST_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64)


def list_runs(g: Graph, k: int, fn, cap: int = 1 << 20, device_buffer=None, stream=None) -> int:
    """k-clique listing (kc_list): fn(rows) is called once per run with the
    run's cliques -- a host numpy view (count, k) of int32 caller ids in
    precedence order, owner first, valid only during the call -- or, with
    device_buffer (a CUDA tensor of cap * k int32), with (pointer, count).
    fn returning a true value stops the listing (KcError KC_ECANCELED).
    Returns the number of cliques delivered."""
    flags = 0
    if device_buffer is not None:
        flags = KC_DEVICE_PTRS
        buf_ptr = _ptr(device_buffer)
        hbuf = None
    else:
        hbuf = np.empty((max(cap, 1), k), dtype=np.int32)
        buf_ptr = hbuf.ctypes.data

    def trampoline(_user, ptr, count):
        if hbuf is not None:
            return 1 if fn(hbuf[:count]) else 0
        return 1 if fn((ptr, count)) else 0

    cb = LIST_FN(trampoline)
    listed = ctypes.c_uint64(0)
    _check(_load().kc_list(g.handle, k, flags, buf_ptr, cap, cb, None, ctypes.byref(listed),
                           _stream_handle(stream)), f"kc_list(k={k})")
    return int(listed.value)


def list_cliques(g: Graph, k: int, cap: int = 1 << 20, stream=None) -> np.ndarray:
    """Every k-clique as rows of k caller ids (precedence order, owner first)."""
    parts = []
    list_runs(g, k, lambda rows: parts.append(rows.copy()), cap=cap, stream=stream)
    return np.concatenate(parts) if parts else np.zeros((0, k), dtype=np.int32)


def count_csr(off, adj, k: int, per_vertex: bool = False, per_owner: bool = False, validate: bool = False,
              stream=None):
    """One-shot FFF_k on a host CSR (orient, count, free)."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    n = int(off.shape[0] - 1)
    m = int(adj.shape[0] // 2)
    pv = np.empty(max(n, 1), np.uint64) if per_vertex else None
    po = np.empty(max(n, 1), np.uint64) if per_owner else None
    tot = ctypes.c_uint64(0)
    flags = KC_VALIDATE if validate else 0
    _check(_load().kc_count_csr(off.ctypes.data, adj.ctypes.data if m else None, n, m, k, flags,
                                ctypes.byref(tot), _ptr(pv), _ptr(po), _stream_handle(stream)),
           f"kc_count_csr(k={k})")
    return int(tot.value), (pv[:n] if pv is not None else None), (po[:n] if po is not None else None)


def estimate_csr(off, adj, k: int, colours: int, seed: int, validate: bool = False, stream=None):
    """One-shot cFFF_k on a host CSR.  Returns (sampled, estimate)."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    n = int(off.shape[0] - 1)
    m = int(adj.shape[0] // 2)
    s = ctypes.c_uint64(0)
    est = ctypes.c_double(0.0)
    flags = KC_VALIDATE if validate else 0
    _check(_load().kc_estimate_csr(off.ctypes.data, adj.ctypes.data if m else None, n, m, k, colours, seed, flags,
                                   ctypes.byref(s), ctypes.byref(est), _stream_handle(stream)),
           f"kc_estimate_csr(k={k})")
    return int(s.value), float(est.value)


def count_static(g: Graph, k: int, stream=None) -> int:
    """q_k like count(), but without any device allocation (kc_count_static):
    for callers that cannot allocate device memory when they count.  Calls
    share one static scratch array and must not overlap on the GPU."""
    tot = ctypes.c_uint64(0)
    _check(_load().kc_count_static(g.handle, k, 0, ctypes.byref(tot), _stream_handle(stream)),
           f"kc_count_static(k={k})")
    return int(tot.value)


# ------------------------------------------------------------------ tuning

def tune(graphs, k: int, per_vertex: bool = False, stream=None) -> dict:
    """Measure the per-class plan (counter and parts per owner) for k on one
    graph or a batch (kc_tune); returns it as a dict (apply with set_tuning)."""
    gl = graphs if isinstance(graphs, (list, tuple)) else [graphs]
    hs = (_P * len(gl))(*[g.handle for g in gl])
    t = _Tuning()
    _check(_load().kc_tune(hs, len(gl), k, KC_TUNE_PER_VERTEX if per_vertex else 0, _stream_handle(stream),
                           ctypes.byref(t)), f"kc_tune(k={k})")
    return {"k": int(t.k), "per_vertex": bool(t.per_vertex), "algo": [int(x) for x in t.algo],
            "parts": [int(x) for x in t.parts], "ms": [float(x) for x in t.ms]}


def set_tuning(g: Graph, plan: dict | None):
    """Attach a plan (from tune() or a cache) to g; None removes all plans."""
    if plan is None:
        _check(_load().kc_set_tuning(g.handle, None), "kc_set_tuning")
        return
    t = _Tuning(int(plan["k"]), int(bool(plan["per_vertex"])), (ctypes.c_int32 * 7)(*plan["algo"]),
                (ctypes.c_int32 * 7)(*plan["parts"]), (ctypes.c_float * 7)(*plan.get("ms", [0.0] * 7)))
    _check(_load().kc_set_tuning(g.handle, ctypes.byref(t)), "kc_set_tuning")


class TuningCache:
    """Plans cached in a JSON file, keyed by the graph's statistics (n, m,
    max |Gamma+|, wedges), k and the output mode, so a graph seen before (or
    one with the same statistics) is not measured again."""

    def __init__(self, path: str):
        import json
        self.path = path
        try:
            with open(path) as f:
                self.plans = json.load(f)
        except (OSError, ValueError):
            self.plans = {}

    @staticmethod
    def key(g: Graph, k: int, per_vertex: bool) -> str:
        return f"n={g.n},m={g.m},dmax={g.max_dplus},wedges={g.wedges},k={k},pv={int(per_vertex)}"

    def plan(self, g: Graph, k: int, per_vertex: bool = False, stream=None, apply: bool = True) -> dict:
        import json
        key = self.key(g, k, per_vertex)
        p = self.plans.get(key)
        if p is None:
            p = tune(g, k, per_vertex, stream)
            self.plans[key] = p
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.plans, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        if apply:
            set_tuning(g, p)
        return p


class Batch:
    """Graphs prepared once for repeated counts at one k (kc_batch_*): count()
    only launches kernels on the stream, so it can be captured into a CUDA
    graph (torch.cuda.graph) and replayed."""

    def __init__(self, graphs, k: int, stream=None):
        self.graphs = list(graphs)  # kept alive with the batch
        hs = (_P * len(self.graphs))(*[g.handle for g in self.graphs])
        h = _P()
        _check(_load().kc_batch_create(hs, len(self.graphs), k, 0, _stream_handle(stream), ctypes.byref(h)),
               f"kc_batch_create(k={k})")
        self._h = h.value
        self.k = k

    def count(self, totals, stream=None):
        """Counts into a device tensor of 2 * len(graphs) int64 (lo, hi words)."""
        _check(_load().kc_batch_count(self._h, _ptr(totals), _stream_handle(stream)), "kc_batch_count")

    def free(self):
        if self._h:
            _load().kc_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
