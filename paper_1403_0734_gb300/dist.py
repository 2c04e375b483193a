"""Multi-GPU helpers: one process per GPU, torch.distributed for the one
exchange the path has.

Owners are independent given the (replicated, read-only) oriented graph --
each clique is counted by its smallest vertex only (Sec. 3) -- so a count is
sharded by giving every rank one part of the owners (kc_count_part) and
summing the partial totals.  The sum is exact: the 64-bit partials travel as
two 32-bit halves in int64 lanes.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def _sum_u64(values, device):
    """Exact sum over ranks of a list of unsigned 64-bit integers."""
    t = torch.tensor([[v & 0xFFFFFFFF, v >> 32] for v in values], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [int(lo) + (int(hi) << 32) for lo, hi in t.tolist()]


def count_sharded(G, k: int, counter=None, device=None) -> int:
    """q_k of G counted jointly by all ranks: rank r counts the owners at
    queue positions r, r + world, ... and the partials are summed.  `counter`
    (G, k, part, nparts) -> partial total; default kc_count_part."""
    rank, world = dist.get_rank(), dist.get_world_size()
    if counter is None:
        from . import kc
        partial = kc.count_part(G, k, rank, world)[0]
    else:
        partial = counter(G, k, rank, world)
    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    return _sum_u64([partial], device)[0]


def reduce_step_stats(ms: float, work: list[int], device=None):
    """Benchmark aggregation: the slowest rank's step time and the sum of
    every rank's work counters (exact)."""
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, list(work)
    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item()), _sum_u64(list(work), device)
