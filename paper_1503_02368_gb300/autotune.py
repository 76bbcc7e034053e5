"""Autotuner for the layout threshold and the intersection launch shape.

Searches the set-level bitset threshold tau (Sec. 4.4's rule, which fixes the
stored layouts, so each value needs its own trie) and the execution knobs
(warps per CTA for heavy vertices, the light/heavy split, the warps per
intersection) on a workload, by
timing the real kernels through the C ABI, and writes the best setting per
graph class to a JSON file.  Counts must agree across every setting tried;
the tuner checks that too, since layouts and launch shapes change speed only.
"""
import json
import os
import time

import numpy as np

from . import eh as _eh

DEFAULT_TAUS = (8, 32, 128)
DEFAULT_WARPS = (4, 8, 16)
DEFAULT_LIGHT = (8, 16, 32)
DEFAULT_PAIR_WARPS = (1, 2, 4)
TUNED_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def _time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return best


def tune_batch(graph, patterns, offsets, pool, taus=DEFAULT_TAUS, warps=DEFAULT_WARPS, light=DEFAULT_LIGHT,
               reps=2, log=None):
    """Best (tau, cta_warps, light_max) for one eh_count_batch over the queries."""
    trials = []
    ref = None
    for tau in taus:
        trie = _eh.Trie(graph["src"], graph["dst"], graph["n"], tau=tau)
        for w in warps:
            for lm in light:
                xo = _eh.exec_opts(cta_warps=w, light_max=lm)
                out = {}

                def run():
                    out["c"], out["s"] = trie.count_batch(patterns, offsets, pool, xopts=xo)

                t = _time(run, reps)
                if ref is None:
                    ref = out["c"].copy()
                if out["s"].any() or not np.array_equal(out["c"], ref):
                    raise RuntimeError("counts differ between tuning settings (tau=%d warps=%d light=%d)"
                                       % (tau, w, lm))
                trials.append({"tau": tau, "cta_warps": w, "light_max": lm, "seconds": t})
                if log:
                    log(trials[-1])
        trie.close()
    best = min(trials, key=lambda r: r["seconds"])
    return best, trials


def tune_whole(graph, pattern="triangle", taus=DEFAULT_TAUS, warps=DEFAULT_WARPS, light=DEFAULT_LIGHT, reps=3,
               log=None, ratios=(32,), pair_warps=DEFAULT_PAIR_WARPS):
    """Best (tau, cta_warps, light_max, gallop_ratio, pair_warps) for a
    whole-graph count; pair_warps is the warps per intersection."""
    import torch
    trials = []
    ref = None
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    for tau in taus:
        trie = _eh.Trie(graph["src"], graph["dst"], graph["n"], tau=tau)
        for w in warps:
            for lm in light:
                for r in ratios:
                    for pw in pair_warps:
                        xo = _eh.exec_opts(cta_warps=w, light_max=lm, gallop_ratio=r, pair_warps=pw)
                        t = _time(lambda: trie.count_async(pattern, out.data_ptr(), xopts=xo), reps)
                        trie.status()
                        c = int(out.item())
                        if ref is None:
                            ref = c
                        if c != ref:
                            raise RuntimeError("counts differ between tuning settings")
                        trials.append({"tau": tau, "cta_warps": w, "light_max": lm, "gallop_ratio": r,
                                       "pair_warps": pw, "seconds": t})
                        if log:
                            log(trials[-1])
        trie.close()
    best = min(trials, key=lambda r: r["seconds"])
    return best, trials


def save(graph_class, best, trials, path=TUNED_PATH):
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[graph_class] = {"best": best, "trials": trials}
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def load(graph_class, path=TUNED_PATH):
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f).get(graph_class, {}).get("best")


def main(argv=None):
    """python -m paper_1503_02368_gb300.autotune [rmat_s22_triangle|rmat_s20_ego4096]:
    searches the named workload on the current GPU and stores the best setting."""
    import argparse
    import sys
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["rmat_s22_triangle", "rmat_s20_ego4096"])
    ap.add_argument("--taus", default=None)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from synth import workloads as W

    def log(r):
        print(json.dumps(r), flush=True)

    if a.workload == "rmat_s22_triangle":
        taus = tuple(int(x) for x in a.taus.split(",")) if a.taus else (256, 1024)
        best, trials = tune_whole(W.rmat22(), "triangle", taus=taus, warps=(8, 16), light=(16, 32),
                                  reps=a.reps, log=log)
    else:
        g = W.rmat20_ego_batch()
        pats = ["clique4" if p else "triangle" for p in g["patterns"]]
        taus = tuple(int(x) for x in a.taus.split(",")) if a.taus else (8, 32, 128)
        best, trials = tune_batch(g, pats, g["offsets"], g["pool"], taus=taus, reps=min(a.reps, 2), log=log)
    save(a.workload, best, trials)
    print("best", json.dumps(best))


if __name__ == "__main__":
    main()
