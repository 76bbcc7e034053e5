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


def whole_graph(name, fn, pats, T):
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
    print(name, {k: v for k, v in rec.items() if k != "vertex_triangles"}, "%.1fs" % (time.time() - t0), flush=True)
    return rec


def ego_batch(T):
    """The 4,096-query ego-net batch: expected counts of a sample of queries."""
    t0 = time.time()
    g = W.rmat20_ego_batch()
    G = oracle.Graph(g["n"], g["src"], g["dst"])
    off, pool, pq = g["offsets"], g["pool"], g["patterns"]
    sizes = np.diff(off)
    rng = np.random.default_rng(4)
    sample = sorted(set(range(8)) | set(rng.choice(len(pq), 56, replace=False).tolist()) |
                    set(np.argsort(-sizes)[:4].tolist()))
    rec = {"n": g["n"], "fingerprint": fingerprint(g), "n_queries": len(pq),
           "subset_fingerprint": hashlib.sha256(pool.tobytes() + off.tobytes()).hexdigest()[:32], "queries": {}}
    for q in sample:
        pat = "clique4" if pq[q] else "triangle"
        rec["queries"][int(q)] = {"pattern": pat, "size": int(sizes[q]),
                                  "count": G.induced(pool[off[q]:off[q + 1]]).count(pat, nthreads=T)}
    print("rmat_s20_ego4096", len(sample), "queries", "%.1fs" % (time.time() - t0), flush=True)
    return rec


def serve_sample(T):
    """Serving workload: R-MAT scale 24 + ego nets (induced edges 100..1e6); 8
    queries per pattern among those with at most 200,000 induced edges."""
    t0 = time.time()
    q_total = 256
    g = W.rmat24_serve(n_queries=q_total)
    G = oracle.Graph(g["n"], g["src"], g["dst"])
    names = ("triangle", "clique4", "lollipop")
    off, pool, pq = g["offsets"], g["pool"], g["patterns"]
    rec = {"n": g["n"], "fingerprint": fingerprint(g), "n_queries": q_total,
           "subset_fingerprint": hashlib.sha256(pool.tobytes() + off.tobytes()).hexdigest()[:32], "queries": {}}
    per = {0: 0, 1: 0, 2: 0}
    for q in range(q_total):
        if per[pq[q]] >= 8:
            continue
        sub = G.induced(pool[off[q]:off[q + 1]])
        if sub.m > 200_000:
            continue
        per[pq[q]] += 1
        rec["queries"][q] = {"pattern": names[pq[q]], "size": int(off[q + 1] - off[q]), "induced_edges": sub.m,
                             "count": sub.count(names[pq[q]], nthreads=T)}
        if all(v >= 8 for v in per.values()):
            break
    print("rmat_s24_serve", len(rec["queries"]), "queries", "%.1fs" % (time.time() - t0), flush=True)
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    ap.add_argument("--only", default=None, help="recompute only this entry, keep the others")
    args = ap.parse_args()
    T = args.threads
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_counts.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    plan = {
        "er_n10000_m100000": lambda: whole_graph("er_n10000_m100000", W.er_10k_100k,
                                                 ["triangle", "clique4", "lollipop", "lollipop_distinct"], T),
        "rmat_s16_ef16": lambda: whole_graph("rmat_s16_ef16", lambda: W.rmat_graph(16, 1503 + 16),
                                             ["triangle", "clique4", "lollipop", "lollipop_distinct", "barbell"],
                                             T),
        "rmat_s22_ef16": lambda: whole_graph("rmat_s22_ef16", W.rmat22, ["triangle", "lollipop"], T),
        "chunglu_n1000000_g2.1": lambda: whole_graph("chunglu_n1000000_g2.1", W.chunglu_1m,
                                                     ["triangle", "clique4", "barbell"], T),
        "rmat_s20_ego4096": lambda: ego_batch(T),
        "rmat_s24_serve": lambda: serve_sample(T),
    }
    for name, fn in plan.items():
        if args.only is None or args.only == name:
            out[name] = fn()
            with open(path, "w") as f:
                json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
