"""Multi-GPU helpers: one process per GPU, torch.distributed for the one
exchange the path has.

Owners are independent given the (replicated, read-only) oriented graph --
each clique is counted by its smallest vertex only (Sec. 3) -- so a count is
sharded by giving every rank one part of the owners (kc_count_part: greedy
LPT over the work estimate w(u)) and summing the partial results: the total,
and element-wise the n per-vertex and per-owner counts.  The sums are exact:
every unsigned 64-bit value travels as two 32-bit halves in int64 lanes (at
most 2^31 ranks), and is put back together after the reduction.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def _device():
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def sum_u64_arrays(arrays, device=None):
    """Exact element-wise sum over ranks of uint64 numpy arrays (same shapes on
    every rank); returns uint64 numpy arrays."""
    device = device or _device()
    out = []
    for a in arrays:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        halves = np.stack([a & 0xFFFFFFFF, a >> 32]).astype(np.int64)
        t = torch.from_numpy(halves).to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        h = t.cpu().numpy().astype(np.uint64)
        out.append(h[0] + (h[1] << np.uint64(32)))
    return out


def sum_u64_tensors(tensors):
    """Exact element-wise sum over ranks of int64 tensors that hold uint64
    values (two's complement), in place: each is reduced as its 32-bit halves
    and put back together (wrapping mod 2^64, as uint64 addition does)."""
    for t in tensors:
        halves = torch.stack([t & 0xFFFFFFFF, (t >> 32) & 0xFFFFFFFF])
        dist.all_reduce(halves, op=dist.ReduceOp.SUM)
        t.copy_(halves[0] + (halves[1] << 32))
    return tensors


def _sum_u64(values, device=None):
    """Exact sum over ranks of a list of unsigned 64-bit integers."""
    device = device or _device()
    t = torch.tensor([[v & 0xFFFFFFFF, v >> 32] for v in values], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [int(lo) + (int(hi) << 32) for lo, hi in t.tolist()]


def count_sharded(G, k: int, per_vertex: bool = False, per_owner: bool = False, counter=None, device=None):
    """q_k of G (and optionally the per-vertex / per-owner counts) counted
    jointly by all ranks: rank r counts part r of the owners (kc_count_part)
    and the partial results are summed exactly.  `counter(G, k, part, nparts,
    per_vertex, per_owner)` -> (total, pv, po) replaces kc_count_part (tests).
    Returns (total, pv or None, po or None) on every rank."""
    rank, world = dist.get_rank(), dist.get_world_size()
    if counter is None:
        from . import kc
        total, pv, po = kc.count_part(G, k, rank, world, per_vertex=per_vertex, per_owner=per_owner)
    else:
        total, pv, po = counter(G, k, rank, world, per_vertex, per_owner)
    total = _sum_u64([total], device)[0]
    arrays = [a for a in (pv, po) if a is not None]
    summed = iter(sum_u64_arrays(arrays, device)) if arrays else iter(())
    pv = next(summed) if pv is not None else None
    po = next(summed) if po is not None else None
    return total, pv, po


def reduce_step_stats(ms: float, work: list[int], device=None):
    """Benchmark aggregation: the slowest rank's step time and the sum of
    every rank's work counters (exact)."""
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, list(work)
    device = device or _device()
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item()), _sum_u64(list(work), device)
