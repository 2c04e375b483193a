"""World-size-2 gloo run on CPU of the multi-GPU host logic: the sharded
count (owner parts + exact sums of the total and of the per-vertex and
per-owner arrays) and the benchmark's cross-rank reduction.  The per-rank
partial comes from the oracle (the owners of the part counted one by one),
standing in for kc_count_part on a GPU; the part is the documented LPT
partition (kc.h, kc_count_part) restated here."""
import heapq
import os
import socket

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def lpt_parts(g, nparts):
    """Owners (caller ids) of each part: owners by w(u) = sum over Gamma+(u)
    of |Gamma+(x)| descending, each to the least loaded part (load + w + 1),
    lowest part on ties.  (Ties in w are broken here by vertex id; the
    library breaks them by queue position -- any partition gives the same
    sums, which is what this test checks.)"""
    import oracle
    perm, rank, offp, adjp = oracle.oriented(g)
    dplus = np.diff(offp)
    w = np.array([int(dplus[adjp[offp[r]:offp[r + 1]]].sum()) for r in range(g.n)], dtype=np.int64)
    order = sorted(range(g.n), key=lambda r: (-w[r], r))
    heap = [(0, p) for p in range(nparts)]
    parts = [[] for _ in range(nparts)]
    for r in order:
        load, p = heapq.heappop(heap)
        parts[p].append(int(perm[r]))
        heapq.heappush(heap, (load + int(w[r]) + 1, p))
    return parts


def oracle_part(g, k, part, nparts, per_vertex, per_owner):
    import oracle
    total = 0
    pv = np.zeros(g.n, np.uint64) if per_vertex else None
    po = np.zeros(g.n, np.uint64) if per_owner else None
    for u in lpt_parts(g, nparts)[part]:
        t, opo, opv = oracle.count(g, k, per_owner=per_owner, per_vertex=per_vertex, u_range=(u, u + 1))
        total += t
        if per_vertex:
            pv += opv
        if per_owner:
            po += opo
    return total, pv, po


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
        res[k] = kd.count_sharded(g, k, per_vertex=True, per_owner=True, counter=oracle_part)
    ms, work = kd.reduce_step_stats(10.0 + rank, [2**40 + rank, 7])
    big = kd.sum_u64_arrays([np.array([2**63 - 1 - rank, 2**32 + rank, 0], dtype=np.uint64)])[0]
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, res, ms, work, big))


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
    parts = lpt_parts(g, world)
    assert sorted(parts[0] + parts[1]) == list(range(g.n))  # a partition of the owners
    for rank, res, ms, work, big in outs:
        for k, (total, pv, po) in res.items():
            ot, opo, opv = oracle.count(g, k, per_owner=True, per_vertex=True)
            assert total == ot
            assert np.array_equal(pv, opv) and np.array_equal(po, opo)
        assert ms == 11.0
        assert work == [2**41 + 1, 14]
        assert [int(x) for x in big] == [2**64 - 3, 2**33 + 1, 0]  # exact near 2^64
