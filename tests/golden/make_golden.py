"""Writes workload_counts.json: oracle counts for the benchmark workloads.

Every expected value stored here is produced by the CPU oracle (``oracle/``)
on the seeded inputs of ``synth/``; nothing comes from the CUDA path.  The
input fingerprints let a test confirm that a machine regenerates the exact
same inputs before it compares counts.

    python tests/golden/make_golden.py [--threads N]
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import workloads as W  # noqa: E402


def fingerprint(g):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g["src"]).tobytes())
    h.update(np.ascontiguousarray(g["dst"]).tobytes())
    return h.hexdigest()[:32]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    args = ap.parse_args()
    T = args.threads
    out = {}
    plan = [
        ("er_n10000_m100000", W.er_10k_100k, ["triangle", "clique4", "lollipop", "lollipop_distinct"]),
        ("rmat_s16_ef16", lambda: W.rmat_graph(16, 1503 + 16), ["triangle", "clique4", "lollipop",
                                                                  "lollipop_distinct"]),
        ("rmat_s22_ef16", W.rmat22, ["triangle"]),
        ("chunglu_n1000000_g2.1", W.chunglu_1m, ["triangle", "clique4"]),
    ]
    for name, fn, pats in plan:
        t0 = time.time()
        g = fn()
        G = oracle.Graph(g["n"], g["src"], g["dst"])
        rec = {"n": g["n"], "raw_edges": int(len(g["src"])), "m": G.m, "fingerprint": fingerprint(g)}
        for p in pats:
            rec[p] = G.count(p, nthreads=T)
        if name == "rmat_s22_ef16":
            # sampled per-vertex triangle counts t(x), for full-size spot checks
            rng = np.random.default_rng(22)
            verts = np.sort(rng.choice(g["n"], 256, replace=False)).astype(np.uint32)
            hubs = np.argsort(-G.degrees())[:16].astype(np.uint32)
            verts = np.concatenate([hubs, verts])
            rec["vertex_triangles"] = {int(v): int(t) for v, t in zip(verts, G.vertex_triangles(verts))}
        out[name] = rec
        print(name, {k: v for k, v in rec.items() if k != "vertex_triangles"}, "%.1fs" % (time.time() - t0),
              flush=True)
    # the 4,096-query ego-net batch: expected counts of a sample of queries
    t0 = time.time()
    g = W.rmat20_ego_batch()
    G = oracle.Graph(g["n"], g["src"], g["dst"])
    off, pool, pq = g["offsets"], g["pool"], g["patterns"]
    sizes = np.diff(off)
    rng = np.random.default_rng(4)
    sample = sorted(set(range(8)) | set(rng.choice(len(pq), 56, replace=False).tolist()) |
                    set(np.argsort(-sizes)[:4].tolist()))
    rec = {"n": g["n"], "fingerprint": fingerprint(g), "n_queries": len(pq),
           "subset_fingerprint": __import__("hashlib").sha256(pool.tobytes() + off.tobytes()).hexdigest()[:32],
           "queries": {}}
    for q in sample:
        pat = "clique4" if pq[q] else "triangle"
        rec["queries"][int(q)] = {"pattern": pat, "size": int(sizes[q]),
                                  "count": G.induced(pool[off[q]:off[q + 1]]).count(pat, nthreads=T)}
    out["rmat_s20_ego4096"] = rec
    print("rmat_s20_ego4096", len(sample), "queries", "%.1fs" % (time.time() - t0), flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_counts.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
