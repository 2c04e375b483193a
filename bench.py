#!/usr/bin/env python
"""bench.py -- k-clique counting throughput (FFF_k) on GB300.

One step = the whole hot path once over the Chung-Lu power-law workload
(n = 10^6, 2*10^7 endpoint draws, exponent 2.1, max weight 20000, seed 1):
orientation (degrees, (degree, id) order, Gamma+ lists, owner queue) from a
device-resident CSR, then exact counts for k = 3, 4, 5, 6 with per-vertex and
per-owner outputs written to device buffers.  value = cliques counted per
second (sum over k of q_k / step time).  The counts run with the plans of the
library's autotuner (kc_tune, measured once per graph statistics and kept in
a JSON cache: set-up, outside the timed steps); plans change speed only.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kc|reference]
                    [--shard] [--no-extras]

Under torchrun every rank counts its own graph (seed 1 + rank: weak
scaling); with --shard all ranks count one graph together (owners split by
the library's LPT partition, uint64 totals and per-vertex/per-owner arrays
summed exactly over NCCL: strong scaling; orientation and the partition are
set-up there).  Rank 0 prints one JSON line.  The line also carries the other
workloads (extra keys, measured once each after the timed steps): the SBM
workload and its dense-block variant (exact k = 4..7, cFFF_k relative errors
over 32 seeds), the batched workload (8192 uneven graphs: batched against one
call per graph, tuned against untuned, captured CUDA graph against direct
launches) and the serving workload (Poisson streams over 64 R-MAT graphs of
scales 16..20 at four loads).  --impl reference times the CPU oracle on the host cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
import traceback

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "k-cliques/sec and edges/sec at k=3..7 on 1 GB300; % HBM roofline; batched p50/p99"
UNIT = "k-cliques/s"
WORKLOAD = "chung_lu n=1e6 m~2e7 gamma=2.1 wmax=20000, exact k=3..6, per-vertex+per-owner"
# the headline graph, and a reduced one of the same degree law for profiler
# captures (its hubs still reach the 16-word class; a k = 6 count takes
# ~0.3 s instead of ~1.1 s)
GRAPHS = {"chunglu_1m": (1_000_000, 20_000_000, 2.1, 20000.0), "chunglu_300k": (300_000, 6_000_000, 2.1, 20000.0)}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")
# Word-operation peak of the counting kernels.  A word-op is one 32-bit AND
# of a candidate-set word with a bitmap row word, its population count, and
# the add of that count.  AND and add issue on the integer ALUs at 128 lanes
# per SM per clock; the population count runs on the narrower unit that
# serves POPC/FLO/BREV, at 16 lanes per SM per clock.  That unit is the
# narrowest one every word-op needs, so the peak is 16 x SMs x SM clock
# (the maximum SM clock of the measured peaks file).
POPC_LANES_PER_SM_CLK = 16
# L2 random-gather rate measured on this GPU (4-byte loads at random
# addresses of a 4 MB table, 8 warps per SM): the rate the orientation's one
# gather pass over the adjacency is bound by.
L2_GATHER_PER_S = 272e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["kc", "reference"], default="kc")
    ap.add_argument("--ks", default="3,4,5,6")
    ap.add_argument("--graph", choices=sorted(GRAPHS), default="chunglu_1m",
                    help="chunglu_300k: reduced graph for profiler captures (not a bench line)")
    ap.add_argument("--shard", action="store_true", help="N>1: all ranks count one graph (strong scaling)")
    ap.add_argument("--no-tune", action="store_true", help="count with the library's default knobs")
    ap.add_argument("--no-extras", action="store_true", help="skip the SBM / batched / serving workloads")
    ap.add_argument("--extras", default="cfff_chunglu,sbm,batch,serving")
    ap.add_argument("--batch-graphs", type=int, default=8192)
    ap.add_argument("--serve-graphs", type=int, default=64)
    # scales 21-22 hold exact k = 6 requests of 30-120 s each on one GB300
    # (R-MAT scale 22: q_6 = 3.4e14), which no bounded run can serve
    ap.add_argument("--serve-scales", default="16,20")
    ap.add_argument("--serve-seconds", type=float, default=25.0,
                    help="target duration of each serving run (sets its request count)")
    ap.add_argument("--serve-max-requests", type=int, default=20000)
    ap.add_argument("--algo", choices=["dfs", "pivot"], default="dfs",
                    help="process-wide Reduce 3 counter for classes without a plan")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0,
                    help="CPU budget of the oracle sample (all k together)")
    ap.add_argument("--tuning-cache", default=os.path.join(tempfile.gettempdir(), "kc_tuning_cache.json"))
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def sources_sha():
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_1403_0734_gb300", "csrc", "*"))):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.path = tempfile.mktemp(prefix="kc_clocks_", suffix=".csv")
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ CPU side

def oracle_sample(g, ks, budget_s: float, nthreads: int = 0):
    """Oracle (as it stands) over owners in id order, chunk by chunk, until the
    budget is spent; ids are a seeded shuffle of weight order, so a prefix of
    ids is a uniform sample of owners.  Returns (cliques, seconds, owners)."""
    import oracle
    cliques, secs, owners = 0, 0.0, 0
    per_k = budget_s / len(ks)
    for k in ks:
        t_k, lo, chunk = 0.0, 0, 64
        while t_k < per_k and lo < g.n:
            hi = min(g.n, lo + chunk)
            t0 = time.perf_counter()
            q = oracle.count(g, k, u_range=(lo, hi), nthreads=nthreads)[0]
            dt = time.perf_counter() - t0
            cliques += q
            t_k += dt
            lo = hi
            if dt < 0.25 * per_k / 8:
                chunk = min(chunk * 2, 1 << 16)
        secs += t_k
        owners = max(owners, lo)
    return cliques, secs, owners


def cpu_baseline(g, ks, budget_s):
    import oracle
    cores = oracle.max_threads(0)
    q, s, owners = oracle_sample(g, ks, budget_s)
    return {"value": q / s if s > 0 else None, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"owners with ids 0..{owners - 1} of {g.n} (uniform: ids are shuffled), "
                      f"k={','.join(map(str, ks))}, {q} cliques in {s:.1f} s on {cores} threads"}


def run_reference(args, ks):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import kcgen
    import oracle
    g = kcgen.chung_lu_1m(seed=1)
    cores = oracle.max_threads(0)
    budget = max(5.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        oracle_sample(g, ks, min(budget, 3.0))
    tot_q, tot_s = 0, 0.0
    owners = 0
    for _ in range(args.steps):
        q, s, owners = oracle_sample(g, ks, budget)
        tot_q += q
        tot_s += s
    value = tot_q / tot_s
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "bounded owner prefix"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"owners with ids 0..{owners - 1} per step, "
                                       f"{budget:.0f} s of oracle time per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ inputs

def _gen(spec):
    import kcgen
    kind, a = spec
    return getattr(kcgen, kind)(*a)


def generate(specs, workers=None):
    """Generate graphs in a spawn process pool (before any CUDA call)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    if not specs:
        return []
    workers = workers or min(16, os.cpu_count() or 1)
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen, specs, chunksize=max(1, len(specs) // (4 * workers))))


def serving_scales(args):
    import numpy as np
    lo, hi = (int(x) for x in args.serve_scales.split(","))
    rng = np.random.default_rng(5)
    return [int(rng.integers(lo, hi + 1)) for _ in range(args.serve_graphs)]


# ------------------------------------------------------------------ extras

def timed(fn, reps=1):
    import torch
    best = None
    out = None
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return out, best


def extra_sbm(kc, graphs, cache):
    """SBM (p_in = 0.3) and its dense-block variant (p_in = 1): exact k = 4..7
    with tuned plans (and the untuned time where it is cheap), cFFF_k relative
    error over 32 seeds for c in {4, 8, 16}."""
    import numpy as np
    import torch
    out = []
    for (label, g) in graphs:
        G = kc.orient(torch.from_numpy(g.off).cuda(), torch.from_numpy(g.adj).cuda())
        var = {"variant": label, "n": g.n, "m": g.m, "exact": {}, "estimate": {}}
        for k in (4, 5, 6, 7):
            plan = cache.plan(G, k, per_vertex=False)
            kc.count(G, k)
            q, dt = timed(lambda: kc.count(G, k)[0], reps=2)
            ent = {"q": q, "ms": dt * 1e3, "cliques_per_s": q / dt, "edges_per_s": g.m / dt,
                   "plan": {"algo": plan["algo"], "parts": plan["parts"]}}
            kc.set_tuning(G, None)
            if label == "sbm_p0.3" or k <= 5:  # untuned (dense blocks: seconds per call at k = 6, 7)
                qu, dtu = timed(lambda: kc.count(G, k)[0])
                assert qu == q
                ent["untuned_ms"] = dtu * 1e3
            kc.set_tuning(G, plan)
            var["exact"][str(k)] = ent
            for c in (4, 8, 16):
                ests, ts = [], []
                for seed in range(1, 33):
                    t0 = time.perf_counter()
                    ests.append(kc.estimate(G, k, c, seed)[1])
                    ts.append(time.perf_counter() - t0)
                e = np.array(ests)
                var["estimate"][f"{k},{c}"] = {
                    "rel_err_mean": float((np.abs(e - q) / q).mean()) if q else None,
                    "rel_err_of_mean": float(abs(e.mean() - q) / q) if q else None,
                    "rel_std": float(e.std(ddof=1) / q) if q else None, "ms": 1e3 * float(np.mean(ts)),
                    "speedup_vs_exact": dt / float(np.mean(ts))}
        out.append(var)
        G.free()
    return out


def extra_cfff_chunglu(kc, g, plans):
    """cFFF_k on the benchmark graph: sampled-count time against the exact
    total-only count for k = 4, 5, 6 and c = 8, 16 (one seed each)."""
    import torch
    G = kc.orient(torch.from_numpy(g.off).cuda(), torch.from_numpy(g.adj).cuda())
    out = {}
    for k in (4, 5, 6):
        q, dt = timed(lambda: kc.count(G, k)[0])
        for c in (8, 16):
            (s, est, _), de = timed(lambda: kc.estimate(G, k, c, 7))
            out[f"{k},{c}"] = {"exact_ms": dt * 1e3, "estimate_ms": de * 1e3, "speedup": dt / de,
                               "rel_err": abs(est - q) / q if q else None}
    G.free()
    return out


def extra_batch(kc, graphs):
    """8192 uneven Chung-Lu graphs, k = 4: one batched launch sequence against
    one call per graph; untuned against tuned; the prepared batch replayed
    from a captured CUDA graph against its direct launches."""
    import torch
    t0 = time.perf_counter()
    Gs = [kc.orient(g.off, g.adj) for g in graphs]
    orient_s = time.perf_counter() - t0
    edges = sum(g.m for g in graphs)
    k = 4
    kc.count_batch(Gs, k)
    tb, batch_s = timed(lambda: kc.count_batch(Gs, k), reps=2)
    q = sum(tb)
    t0 = time.perf_counter()
    plan = kc.tune(Gs, k)
    tune_s = time.perf_counter() - t0
    kc.set_tuning(Gs[0], plan)
    tt, tuned_s = timed(lambda: kc.count_batch(Gs, k), reps=2)
    assert tt == tb
    b = kc.Batch(Gs, k)
    out = torch.zeros(2 * len(Gs), dtype=torch.int64, device="cuda")
    b.count(out)
    _, direct_s = timed(lambda: b.count(out), reps=3)
    s = torch.cuda.Stream()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=s):
        b.count(out)
    cg.replay()
    _, graph_s = timed(cg.replay, reps=3)
    assert [int(x) for x in out[0::2].tolist()] == tb
    t0 = time.perf_counter()
    ts = [kc.count(G, k)[0] for G in Gs]
    single_s = time.perf_counter() - t0
    assert ts == tb
    b.free()
    for G in Gs:
        G.free()

    def rates(sec):
        return {"s": sec, "graphs_per_s": len(Gs) / sec, "cliques_per_s": q / sec, "edges_per_s": edges / sec}
    return {"graphs": len(Gs), "edges": edges, "k": k, "q_total": q, "orient_s": orient_s,
            "batched_untuned": rates(batch_s), "batched_tuned": rates(tuned_s), "tune_s": tune_s,
            "plan": {"algo": plan["algo"], "parts": plan["parts"]},
            "prepared_direct": rates(direct_s), "prepared_cuda_graph": rates(graph_s),
            "one_call_per_graph": rates(single_s), "speedup_batched_vs_per_graph": single_s / tuned_s}


def extra_serving(kc, graphs, scales, args):
    """Poisson streams over 64 device-resident R-MAT graphs (requests: exact
    k in [3, 6] or cFFF_k with c in [2, 16], 50/50), 8 stream slots, admission
    by device footprint; saturation from a burst, then loads 0.5, 0.8, 1.0,
    1.2 x saturation with EDF admission (and FIFO at 0.8 for comparison)."""
    import torch
    from paper_1403_0734_gb300 import serve
    Gs = [kc.orient(g.off, g.adj) for g in graphs]
    edges = [g.m for g in graphs]
    cost = serve.CostModel(edges)
    probe = serve.poisson_stream(100, 0.0, len(Gs), seed=11)
    srv = serve.Server(Gs, slots=8, policy="edf", cost=cost)
    res, span = srv.run(probe, stream_factory=torch.cuda.Stream, realtime=False)
    sat = len(probe) / span
    runs = []
    for load, policy in ((0.5, "edf"), (0.8, "edf"), (1.0, "edf"), (1.2, "edf"), (0.8, "fifo")):
        rate = load * sat
        num = int(min(args.serve_max_requests, max(100, args.serve_seconds * rate)))
        reqs = serve.poisson_stream(num, rate, len(Gs), seed=12)
        srv = serve.Server(Gs, slots=8, policy=policy, cost=cost)
        res, span = srv.run(reqs, stream_factory=torch.cuda.Stream)
        st = serve.latency_stats(res)
        by_id = sorted(reqs, key=lambda x: x.rid)
        exact = sum(r.value for r, q in zip(res, by_id) if q.colours == 0)
        runs.append({"load": load, "policy": policy, "requests": num, "offered_req_per_s": rate,
                     "req_per_s": len(reqs) / span, "exact_cliques_per_s": exact / span,
                     "max_concurrent": srv.max_concurrent, **st})
    for G in Gs:
        G.free()
    return {"graphs": len(Gs), "scales": [min(scales), max(scales)], "edges": sum(edges),
            "saturation_req_per_s": sat, "runs": runs}


# ------------------------------------------------------------------ main

def main():
    args = parse()
    ks = [int(x) for x in args.ks.split(",")]
    if args.impl == "reference":
        return run_reference(args, ks)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    shard = args.shard and world > 1
    extras = [] if (args.no_extras or rank != 0 or world > 1) else args.extras.split(",")

    # every input, generated before the first CUDA call
    import kcgen
    specs = [("chung_lu", (*GRAPHS[args.graph], 1 if shard else 1 + rank))]
    if "sbm" in extras:
        specs += [("sbm_2m", (1, 0.3)), ("sbm_2m", (1, 1.0))]
    nb = len(specs)
    if "batch" in extras:
        specs += [("chung_lu", (n, m, 2.3, w, s)) for (n, m, w, s) in kcgen.batch_params(args.batch_graphs, 1)]
    nbatch_end = len(specs)
    scales = serving_scales(args) if "serving" in extras else []
    specs += [("rmat", (s, 16, 0.57, 0.19, 0.19, 100 + i)) for i, s in enumerate(scales)]
    t0 = time.perf_counter()
    gen = generate(specs)
    gen_s = time.perf_counter() - t0
    g = gen[0]

    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    __graft_entry__.build() if rank == 0 else None
    if world > 1:
        dist.barrier()
    import paper_1403_0734_gb300 as kc
    from paper_1403_0734_gb300 import dist as kd

    kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_DFS if args.algo == "dfs" else kc.KC_ALGO_PIVOT)
    cache = kc.TuningCache(args.tuning_cache.replace(".json", f"_{rank}.json"))
    off_d = torch.from_numpy(g.off).cuda()
    adj_d = torch.from_numpy(g.adj).cuda()
    n = g.n
    tot = {k: torch.zeros(2, dtype=torch.int64, device="cuda") for k in ks}
    pv = {k: torch.zeros(n, dtype=torch.int64, device="cuda") for k in ks}
    po = {k: torch.zeros(n, dtype=torch.int64, device="cuda") for k in ks}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    # plans: measured once per graph statistics (cached), attached to each
    # step's new handle (a host-side table)
    plans = {}
    if not args.no_tune:
        G0 = kc.orient(off_d, adj_d)
        for k in ks:
            if k >= 4:
                plans[k] = cache.plan(G0, k, per_vertex=True, apply=False)
        G0.free()
    Gs = kc.orient(off_d, adj_d) if shard else None
    if shard:
        for k, p in plans.items():
            kc.set_tuning(Gs, p)
        for k in ks:  # the LPT partition, built once (set-up)
            kc.count_part_device(Gs, k, rank, world, tot[k], pv[k], po[k])
        torch.cuda.synchronize()

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        G = Gs if shard else kc.orient(off_d, adj_d)
        if not shard:
            for p in plans.values():
                kc.set_tuning(G, p)
        if evs:
            evs[1].record(stream)
        for i, k in enumerate(ks):
            if shard:
                kc.count_part_device(G, k, rank, world, tot[k], pv[k], po[k])
                kd.sum_u64_tensors([tot[k], pv[k], po[k]])
            else:
                kc.count_device(G, k, tot[k], pv[k], po[k])
            if evs:
                evs[2 + i].record(stream)
        return G

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        G = step()
        torch.cuda.synchronize()
        if not shard:
            G.free()

    kc.set_param(kc.KC_PARAM_LAUNCH_COUNT, 0)
    step_ms, orient_ms, k_ms = [], [], {k: [] for k in ks}
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.zero_()  # L2 (129 MB) flushed between timed steps
            sync_all()
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 + len(ks))]
            G = step(evs)
            sync_all()
            step_ms.append(evs[0].elapsed_time(evs[-1]))
            orient_ms.append(evs[0].elapsed_time(evs[1]))
            for i, k in enumerate(ks):
                k_ms[k].append(evs[1 + i].elapsed_time(evs[2 + i]))
            if not shard:
                G.free()
    launches = kc.get_param(kc.KC_PARAM_LAUNCH_COUNT)
    clocks = clk.summary()

    q = {k: int(tot[k][0].item()) for k in ks}
    assert all(int(tot[k][1].item()) == 0 for k in ks), "count overflow"
    for k in ks:  # invariants the paper fixes: memberships sum to k q_k, owners to q_k
        assert int(pv[k].sum().item()) == k * q[k] and int(po[k].sum().item()) == q[k]
    cliques = sum(q.values())
    ms = statistics.mean(step_ms)
    ms_all, (cliques_all, m_all) = kd.reduce_step_stats(ms, [cliques, g.m])
    if shard:  # one graph counted jointly: its cliques and edges once
        cliques_all, m_all = cliques, g.m

    pk, pk_kind = peaks()
    # roofline of the dominant call (counting at the largest k), untimed work count
    kmax = max(ks)
    kc.set_param(kc.KC_PARAM_WORK_COUNT, 1)
    G = kc.orient(off_d, adj_d)
    for p in plans.values():
        kc.set_tuning(G, p)
    kc.count(G, kmax, per_vertex=True, per_owner=True)
    work = kc.get_param(kc.KC_PARAM_WORK_COUNT)
    # the plain ordered search's word-ops (every dense set closed on its
    # edges): the work the complement count of the timed call avoids
    kc.set_param(kc.KC_PARAM_COMPLEMENT, 0)
    kc.count(G, kmax, per_vertex=True, per_owner=True)
    work_plain = kc.get_param(kc.KC_PARAM_WORK_COUNT)
    kc.set_param(kc.KC_PARAM_COMPLEMENT, 1)
    kc.set_param(kc.KC_PARAM_WORK_COUNT, 0)
    r2 = {k: kc.round2_bytes(G, k) for k in ks}
    G.free()
    kmax_ms = statistics.mean(k_ms[kmax])
    clock_mhz = float(pk.get("sm_max_mhz", 2070.0))
    num_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_wops = POPC_LANES_PER_SM_CLK * num_sms * clock_mhz * 1e6 / 1e12  # Tword-op/s
    achieved = work / (kmax_ms * 1e-3) / 1e12
    traffic = None
    try:
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        if tr.get("sources_sha") == sources_sha():
            traffic = tr.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    roofline = {"bound": "alu", "kernel": f"kc_count k={kmax} (counting kernels)", "achieved": achieved,
                "peak": peak_wops, "unit": "Tword-op/s", "frac": achieved / peak_wops, "traffic": traffic,
                "work_word_ops": work, "peak_kind": f"POPC lanes x SMs x {pk_kind} max SM clock",
                "plain_search_word_ops": work_plain,
                "effective_frac": work_plain / (kmax_ms * 1e-3) / 1e12 / peak_wops}
    hbm = float(pk.get("hbm_gbs", 6800.0))
    # orientation: HBM-streaming bytes ~ 20m + 32n; its one pass of 2m random
    # L2 gathers bounds it below HBM speed
    orient_bytes = 20 * g.m + 32 * g.n
    om = statistics.mean(orient_ms)
    orient_roof = {"bound": "hbm", "achieved": orient_bytes / (om * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                   "algorithmic_bytes": orient_bytes, "l2_gather_bound_ms": 2 * g.m / L2_GATHER_PER_S * 1e3}
    orient_roof["frac"] = orient_roof["achieved"] / hbm
    orient_roof["frac_of_gather_bound"] = orient_roof["l2_gather_bound_ms"] / om
    # Round 2 (the build of every G+(u)): its input bytes over the k = 3, 4 calls
    build_roof = {"bound": "hbm", "peak": hbm, "unit": "GB/s",
                  "per_k": {str(k): {"round2_bytes": r2[k], "ms": statistics.mean(k_ms[k]),
                                     "achieved": r2[k] / (statistics.mean(k_ms[k]) * 1e-3) / 1e9,
                                     "frac": r2[k] / (statistics.mean(k_ms[k]) * 1e-3) / 1e9 / hbm}
                            for k in ks if k <= 4}}

    # end to end through the C ABI with host buffers (pinned), one rank's view
    e2e = None
    if not args.no_e2e and not shard:
        off_h = torch.from_numpy(g.off).pin_memory().numpy()
        adj_h = torch.from_numpy(g.adj).pin_memory().numpy()
        outs = {k: (torch.empty(n, dtype=torch.int64).pin_memory().numpy().view(np.uint64),
                    torch.empty(n, dtype=torch.int64).pin_memory().numpy().view(np.uint64)) for k in ks}

        def e2e_step():
            Gh = kc.orient(off_h, adj_h)
            for p in plans.values():
                kc.set_tuning(Gh, p)
            s = 0
            for k in ks:
                s += kc.count(Gh, k, out_pv=outs[k][0], out_po=outs[k][1])[0]
            Gh.free()
            return s

        e2e_step()
        ts = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = e2e_step()
            ts.append(time.perf_counter() - t0)
            assert s == cliques
        h2d = g.off.nbytes + g.adj.nbytes
        d2h = len(ks) * (8 + 2 * 8 * n)
        e2e = {"value": cliques / statistics.mean(ts), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * statistics.mean(ts)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g, ks, args.cpu_seconds)

    extra = {}
    if extras:
        extra["generation_s"] = gen_s
    for name, fn in (("cfff_chunglu", lambda: extra_cfff_chunglu(kc, g, plans)),
                     ("sbm", lambda: extra_sbm(kc, [("sbm_p0.3", gen[1]), ("sbm_dense_p1.0", gen[2])], cache)),
                     ("batch", lambda: extra_batch(kc, gen[nb:nbatch_end])),
                     ("serving", lambda: extra_serving(kc, gen[nbatch_end:], scales, args))):
        if name in extras:
            try:
                extra[name] = fn()
            except Exception as e:  # a failing extra must not lose the headline line
                extra[name] = {"error": f"{type(e).__name__}: {e}", "trace": traceback.format_exc()[-800:]}

    if rank == 0:
        per_k = {str(k): {"q": q[k], "ms": statistics.mean(k_ms[k]),
                          "cliques_per_s": q[k] / (statistics.mean(k_ms[k]) * 1e-3),
                          "edges_per_s": g.m / ((statistics.mean(k_ms[k]) + om) * 1e-3)} for k in ks}
        mode = (f"sharded x{world}: one graph, owners split by LPT over w(u), NCCL sums"
                if shard else f"replicas x{world} (one graph per rank)")
        line = {"metric": METRIC, "value": cliques_all / (ms_all * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
                "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic",
                "config": {"workload": (WORKLOAD if args.graph == "chunglu_1m" else WORKLOAD.replace("n=1e6 m~2e7", "n=3e5 m~6e6"))
                           + (", seed 1" if shard else ", seed 1+rank"), "n": g.n, "m": g.m,
                           "ks": ks, "l2": "flushed between timed steps (512 MiB write)", "parallelism": mode,
                           "counter": "autotuned plans (kc_tune) per k" if plans else args.algo,
                           "orientation_in_step": not shard},
                "edges_per_s": m_all / (ms_all * 1e-3), "orient_ms": om, "per_k": per_k,
                "plans": {str(k): {"algo": p["algo"], "parts": p["parts"]} for k, p in plans.items()},
                "roofline": roofline, "orient_roofline": orient_roof, "build_roofline": build_roof,
                "clocks": clocks, "gpu_launches": launches, "e2e": e2e, "cpu_baseline": cpu, **extra}
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
