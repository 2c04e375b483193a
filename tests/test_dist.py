"""World-size-2 gloo run on CPU of the multi-GPU host logic: the sharded
count (owner parts + exact sum) and the benchmark's cross-rank reduction.
The per-rank partial comes from the oracle (owners of the part counted one
by one), standing in for kc_count_part on a GPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def oracle_part(g, k, part, nparts):
    """Owners at queue positions part, part+nparts, ... of the queue ordered
    by |Gamma+| descending, ties by rank (the library's queue), counted by
    the oracle."""
    import oracle
    perm, rank, offp, _ = oracle.oriented(g)
    dplus = np.diff(offp)
    queue = np.lexsort((np.arange(g.n), -dplus))  # ranks
    total = 0
    for r in queue[part::nparts]:
        u = int(perm[r])
        total += oracle.count(g, k, u_range=(u, u + 1))[0]
    return total


def worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import kcgen
    from paper_1403_0734_gb300 import dist as kd
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = kcgen.chung_lu(1200, 10000, 2.1, 150.0, 11)
    res = {}
    for k in (3, 4, 5):
        res[k] = kd.count_sharded(g, k, counter=oracle_part)
    ms, work = kd.reduce_step_stats(10.0 + rank, [2**40 + rank, 7])
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, res, ms, work))


def test_two_rank_sharded_count_and_stats():
    import oracle
    import kcgen
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    outs = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = kcgen.chung_lu(1200, 10000, 2.1, 150.0, 11)
    for rank, res, ms, work in outs:
        for k, v in res.items():
            assert v == oracle.count(g, k)[0]
        assert ms == 11.0
        assert work == [2**41 + 1, 14]
