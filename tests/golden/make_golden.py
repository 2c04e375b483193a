"""Writes tests/golden/workloads.json: generator fingerprints and the
oracle's clique counts for small workloads.

Calls only kcgen (the input generators) and oracle/ (never the CUDA
library).  Run from the repository root:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import kcgen  # noqa: E402
import oracle  # noqa: E402

GRAPHS = [
    ("er_1000_seed1", "erdos_renyi", [1000, 10000, 1]),
    ("chunglu_20k", "chung_lu", [20000, 200000, 2.1, 2000.0, 1]),
    ("sbm_20k", "sbm", [20000, 50, 0.3, 500000, 1]),
    ("rmat_s12", "rmat", [12, 16, 0.57, 0.19, 0.19, 1]),
    ("chunglu_1m_2.1_20000", "chung_lu", [1000000, 20000000, 2.1, 20000.0, 1]),
]


def fingerprint(g):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.off).tobytes())
    h.update(np.ascontiguousarray(g.adj).tobytes())
    return h.hexdigest()


def main():
    out = {"graphs": [], "counts": []}
    for name, maker, args in GRAPHS:
        g = getattr(kcgen, maker)(*args)
        out["graphs"].append({"name": name, "maker": maker, "args": args,
                              "n": g.n, "m": g.m, "sha256": fingerprint(g)})
        if g.n <= 20000:
            for k in range(3, 8):
                q = oracle.count(g, k)[0]
                out["counts"].append({"graph": name, "k": k, "q": str(q), "by": "oracle"})
    g = kcgen.er_1000()
    out["counts"].append({"graph": "er_1000_seed1", "k": 3, "q": str(oracle.brute_force(g, 3)[0]),
                          "by": "brute_force"})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
