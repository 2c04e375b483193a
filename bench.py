#!/usr/bin/env python
"""bench.py -- k-clique counting throughput (FFF_k) on GB300.

One step = the whole hot path once over the Chung-Lu power-law workload
(n = 10^6, 2*10^7 endpoint draws, exponent 2.1, max weight 20000, seed 1):
orientation (degrees, (degree, id) order, Gamma+ lists, owner queue) from a
device-resident CSR, then exact counts for k = 3, 4, 5, 6 with per-vertex and
per-owner outputs written to device buffers.  value = cliques counted per
second (sum over k of q_k / step time).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kc|reference]

Under torchrun every rank counts its own graph (seed 1 + rank: weak
scaling); rank 0 prints one JSON line.  --impl reference times the CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "k-cliques/sec and edges/sec at k=3..7 on 1 GB300; % HBM roofline; batched p50/p99"
UNIT = "k-cliques/s"
WORKLOAD = "chung_lu n=1e6 m~2e7 gamma=2.1 wmax=20000 seed=1+rank, exact k=3..6, per-vertex+per-owner"
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["kc", "reference"], default="kc")
    ap.add_argument("--ks", default="3,4,5,6")
    ap.add_argument("--config", choices=["chunglu", "sbm", "batch", "serving"], default="chunglu",
                    help="chunglu: the benchmark line; sbm / batch / serving: the other workloads")
    ap.add_argument("--batch-graphs", type=int, default=8192)
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-graphs", type=int, default=64)
    ap.add_argument("--serve-scales", default="14,18")
    ap.add_argument("--serve-load", type=float, default=0.8,
                    help="arrival rate as a fraction of the measured saturation throughput")
    ap.add_argument("--algo", choices=["dfs", "pivot"], default="dfs",
                    help="Reduce 3 counter (ordered DFS or pivoting clique tree)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0,
                    help="CPU budget of the oracle sample (all k together)")
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


# ------------------------------------------------------------------ GPU side

def _gen(spec):
    import kcgen
    kind, a = spec
    return getattr(kcgen, kind)(*a)


def generate(specs, workers=None):
    """Generate graphs in a spawn process pool (before any CUDA call)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = workers or min(16, os.cpu_count() or 1)
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen, specs, chunksize=max(1, len(specs) // (4 * workers))))


def run_sbm(args):
    """SBM workload: exact counts k = 4..7 and cFFF_k relative error over 32
    seeds for c in {4, 8, 16}; also the dense-block variant (p_in = 1)."""
    import numpy as np
    import torch
    import kcgen
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_0734_gb300 as kc
    out = {"config": "sbm", "metric": METRIC, "unit": UNIT, "variants": []}
    for p_in in (0.3, 1.0):
        g = kcgen.sbm_2m(1, p_in)
        torch.cuda.synchronize()
        G = kc.orient(torch.from_numpy(g.off).cuda(), torch.from_numpy(g.adj).cuda())
        var = {"p_in": p_in, "n": g.n, "m": g.m, "exact": {}, "estimate": {}}
        for k in (4, 5, 6, 7):
            kc.count(G, k)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q = kc.count(G, k)[0]
            dt = time.perf_counter() - t0
            var["exact"][str(k)] = {"q": q, "ms": dt * 1e3, "cliques_per_s": q / dt}
            for c in (4, 8, 16):
                ests, ts = [], []
                for seed in range(1, 33):
                    t0 = time.perf_counter()
                    ests.append(kc.estimate(G, k, c, seed)[1])
                    ts.append(time.perf_counter() - t0)
                e = np.array(ests)
                rel = np.abs(e - q) / q if q else np.zeros_like(e)
                var["estimate"][f"{k},{c}"] = {
                    "mean_estimate": float(e.mean()), "rel_err_mean": float(rel.mean()) if q else None,
                    "rel_err_of_mean": float(abs(e.mean() - q) / q) if q else None,
                    "rel_std": float(e.std(ddof=1) / q) if q else None, "ms": 1e3 * float(np.mean(ts)),
                    "speedup_vs_exact": dt / float(np.mean(ts))}
        out["variants"].append(var)
        G.free()
    print(json.dumps(out))
    return 0


def run_batch(args):
    """Batched workload: uneven Chung-Lu graphs (n log-uniform in [50, 20000],
    exponent 2.3, average degree in [8, 64]) counted for k = 4 in one launch
    sequence, against one call per graph."""
    import kcgen
    import torch
    specs = [("chung_lu", (n, m, 2.3, w, s)) for (n, m, w, s) in kcgen.batch_params(args.batch_graphs, 1)]
    t0 = time.perf_counter()
    graphs = generate(specs)
    gen_s = time.perf_counter() - t0
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_0734_gb300 as kc
    torch.cuda.init()
    Gs = [kc.orient(g.off, g.adj) for g in graphs]
    edges = sum(g.m for g in graphs)
    k = 4
    kc.count_batch(Gs, k)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tb = kc.count_batch(Gs, k)
    batch_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ts = [kc.count(G, k)[0] for G in Gs]
    single_s = time.perf_counter() - t0
    assert tb == ts
    q = sum(tb)
    print(json.dumps({"config": "batch", "graphs": len(Gs), "edges": edges, "k": k, "q_total": q,
                      "batched": {"s": batch_s, "graphs_per_s": len(Gs) / batch_s, "cliques_per_s": q / batch_s,
                                  "edges_per_s": edges / batch_s},
                      "one_call_per_graph": {"s": single_s, "graphs_per_s": len(Gs) / single_s,
                                             "cliques_per_s": q / single_s, "edges_per_s": edges / single_s},
                      "speedup": single_s / batch_s, "generation_s": gen_s}))
    return 0


def run_serving(args):
    """Serving: Poisson stream over device-resident R-MAT graphs (edge factor
    16, a/b/c = .57/.19/.19), each request exact k in [3, 6] or cFFF_k with c
    in [2, 16]; admission by device footprint; p50/p99 latency."""
    import numpy as np
    import torch
    lo, hi = (int(x) for x in args.serve_scales.split(","))
    rng = np.random.default_rng(5)
    scales = [int(rng.integers(lo, hi + 1)) for _ in range(args.serve_graphs)]
    graphs = generate([("rmat", (s, 16, 0.57, 0.19, 0.19, 100 + i)) for i, s in enumerate(scales)])
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_0734_gb300 as kc
    from paper_1403_0734_gb300 import serve
    torch.cuda.init()
    Gs = [kc.orient(g.off, g.adj) for g in graphs]
    # saturation throughput: a burst with every request present at time 0
    probe = serve.poisson_stream(min(200, args.serve_requests), 0.0, len(Gs), seed=11)
    srv = serve.Server(Gs, slots=8)
    res, span = srv.run(probe, stream_factory=torch.cuda.Stream, realtime=False)
    sat = len(probe) / span
    reqs = serve.poisson_stream(args.serve_requests, args.serve_load * sat, len(Gs), seed=12)
    srv = serve.Server(Gs, slots=8)
    res, span = srv.run(reqs, stream_factory=torch.cuda.Stream)
    st = serve.latency_stats(res)
    exact = sum(r.value for r, q in zip(res, sorted(reqs, key=lambda x: x.rid)) if q.colours == 0)
    print(json.dumps({"config": "serving", "graphs": len(Gs), "scales": [lo, hi], "requests": len(reqs),
                      "saturation_req_per_s": sat, "offered_req_per_s": args.serve_load * sat,
                      "req_per_s": len(reqs) / span, "exact_cliques_per_s": exact / span,
                      "max_concurrent": srv.max_concurrent, **st}))
    return 0


def main():
    args = parse()
    ks = [int(x) for x in args.ks.split(",")]
    if args.impl == "reference":
        return run_reference(args, ks)
    if args.config == "sbm":
        return run_sbm(args)
    if args.config == "batch":
        return run_batch(args)
    if args.config == "serving":
        return run_serving(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    import kcgen

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    __graft_entry__.build() if rank == 0 else None
    if world > 1:
        dist.barrier()
    import paper_1403_0734_gb300 as kc

    kc.set_param(kc.KC_PARAM_ALGO, kc.KC_ALGO_DFS if args.algo == "dfs" else kc.KC_ALGO_PIVOT)
    g = kcgen.chung_lu_1m(seed=1 + rank)
    off_d = torch.from_numpy(g.off).cuda()
    adj_d = torch.from_numpy(g.adj).cuda()
    n = g.n
    tot = {k: torch.zeros(2, dtype=torch.int64, device="cuda") for k in ks}
    pv = {k: torch.zeros(n, dtype=torch.int64, device="cuda") for k in ks}
    po = {k: torch.zeros(n, dtype=torch.int64, device="cuda") for k in ks}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        G = kc.orient(off_d, adj_d)
        if evs:
            evs[1].record(stream)
        for i, k in enumerate(ks):
            kc.count_device(G, k, tot[k], pv[k], po[k])
            if evs:
                evs[2 + i].record(stream)
        return G

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    # warm-up
    for _ in range(args.warmup):
        G = step()
        torch.cuda.synchronize()
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
            G.free()
    launches = kc.get_param(kc.KC_PARAM_LAUNCH_COUNT)
    clocks = clk.summary()

    q = {k: int(tot[k][0].item()) for k in ks}
    assert all(int(tot[k][1].item()) == 0 for k in ks), "count overflow"
    for k in ks:  # invariants the paper fixes: memberships sum to k q_k, owners to q_k
        assert int(pv[k].sum().item()) == k * q[k] and int(po[k].sum().item()) == q[k]
    cliques = sum(q.values())
    ms = statistics.mean(step_ms)
    from paper_1403_0734_gb300 import dist as kd
    ms_all, (cliques_all, m_all) = kd.reduce_step_stats(ms, [cliques, g.m])

    # roofline of the dominant call (counting at the largest k), untimed work count
    kmax = max(ks)
    kc.set_param(kc.KC_PARAM_WORK_COUNT, 1)
    G = kc.orient(off_d, adj_d)
    kc.count(G, kmax, per_vertex=True, per_owner=True)
    work = kc.get_param(kc.KC_PARAM_WORK_COUNT)
    kc.set_param(kc.KC_PARAM_WORK_COUNT, 0)
    kmax_ms = statistics.mean(k_ms[kmax])
    pk, pk_kind = peaks()
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
                "work_word_ops": work, "peak_kind": f"derived from {pk_kind} max SM clock"}
    # orientation: HBM-bound streaming (algorithmic bytes ~ 20m + 32n)
    orient_bytes = 20 * g.m + 32 * g.n
    om = statistics.mean(orient_ms)
    orient_roof = {"bound": "hbm", "achieved": orient_bytes / (om * 1e-3) / 1e9,
                   "peak": float(pk.get("hbm_gbs", 6800.0)), "unit": "GB/s", "algorithmic_bytes": orient_bytes}
    orient_roof["frac"] = orient_roof["achieved"] / orient_roof["peak"]

    # end to end through the C ABI with host buffers (pinned), one rank's view
    e2e = None
    if not args.no_e2e:
        off_h = torch.from_numpy(g.off).pin_memory().numpy()
        adj_h = torch.from_numpy(g.adj).pin_memory().numpy()
        outs = {k: (torch.empty(n, dtype=torch.int64).pin_memory().numpy().view(np.uint64),
                    torch.empty(n, dtype=torch.int64).pin_memory().numpy().view(np.uint64)) for k in ks}

        def e2e_step():
            Gh = kc.orient(off_h, adj_h)
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

    if rank == 0:
        per_k = {str(k): {"q": q[k], "ms": statistics.mean(k_ms[k]),
                          "cliques_per_s": q[k] / (statistics.mean(k_ms[k]) * 1e-3),
                          "edges_per_s": g.m / ((statistics.mean(k_ms[k]) + om) * 1e-3)} for k in ks}
        line = {"metric": METRIC, "value": cliques_all / (ms_all * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": g.n, "m": g.m, "ks": ks,
                           "l2": "flushed between timed steps (512 MiB write)",
                           "parallelism": f"replicas x{world} (one graph per rank)", "counter": args.algo},
                "edges_per_s": m_all / (ms_all * 1e-3), "orient_ms": om, "per_k": per_k,
                "roofline": roofline, "orient_roofline": orient_roof, "clocks": clocks,
                "gpu_launches": launches, "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
