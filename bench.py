#!/usr/bin/env python
"""Benchmark: exact triangle COUNT(*) on the R-MAT scale-22 graph (edges/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl eh|reference]

One step = one whole-graph triangle count (eh_count_async) on the resident
trie: the layout-dispatched intersection kernel over every (u, v) pair of
the degree-pruned trie, plus its finalize kernel.  The trie build (index
creation) is outside the step, as in the paper's timing rule (Sec. 5.1.3);
the end-to-end figure (`e2e`) includes it, with the host edge list copied in
and the count copied out inside the timed region.

N > 1 (torchrun): every rank holds a replica of the trie and counts its part
of the work (eh_count_range_async: the heavy and light work lists cut into
N contiguous cost-balanced ranges); one 8-byte all-reduce sums the parts.  A
step is one whole-graph count on all ranks together (strong scaling); the
value is the graph's edges over the slowest rank's step time.

With no --workload the line also carries every other workload as extra keys:
the ER triangle count, the R-MAT-22 lollipop, the Chung-Lu 4-clique (with
the barbell and the selection queries), the 4,096-query batch against one
launch per query, and the R-MAT-24 serving loop, each with its own clock
record and exactness check.

The reference arm is the CPU oracle (plain nested-loop generic join) timed
on a bounded sample of the outer loop of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 2 ** 20
FLUSH_BYTES = 256 * 2 ** 20
METRIC = "triangle-count edges/sec (R-MAT scale 22, exact COUNT(*))"
WORKLOAD = "rmat_s22_ef16 triangle: R-MAT scale 22, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), seed 1505"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="eh", choices=["eh", "reference"])
    ap.add_argument("--tau", type=int, default=None,
                    help="bitset threshold; default: the autotuned value for the workload (else 32)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="default",
                    choices=["default", "triangle", "er", "lollipop", "clique4", "batch", "serve", "list", "order", "all"],
                    help="default: the headline line plus every workload (ER triangle, R-MAT-22 lollipop, Chung-Lu "
                         "4-clique, query batch, serving) as extra keys; triangle: the headline only; all: default "
                         "plus the listing and the ordering study; any other name: the headline plus that leg")
    ap.add_argument("--serve-queries", type=int, default=1500)
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="process group of the N > 1 path (nccl: the 8-byte sum on the device; gloo: through the "
                         "host, which also lets several ranks share one GPU)")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profile_traffic(kernel_src):
    """DRAM bytes per launch of the count kernel from the committed ncu summary,
    or None when the summary is missing or was taken on other kernel source."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "k_triangle_rmat_s22.md")
    if not os.path.exists(p):
        return None
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    vals = {}
    for line in open(p):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].rsplit(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("count.cu sha256[:16]") != h:
        return None
    try:
        return float(vals["dram bytes per launch (full size)"])
    except (KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_ms=50):
        self.index = index
        self.skip = 0
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", str(period_ms)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def _lines(self):
        with open(self.f.name) as g:
            return sum(1 for _ in g)

    def start(self, wait_s=3.0):
        """Wait for the sampler's first row, then count only rows written after this call."""
        self.pre = 0
        if self.p is None:
            return
        t0 = time.time()
        while self._lines() == 0 and self.p.poll() is None and time.time() - t0 < wait_s:
            time.sleep(0.02)
        self.skip = self._lines()

    def mark(self):
        """The timed region starts: rows written before it (the warm-up's) are
        kept aside, for a region too short to hold a sample of its own."""
        if self.p is None:
            return
        n = self._lines()
        self.pre, self.skip = n - self.skip, n

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows, warm = [], []
        for i, line in enumerate(open(self.f.name)):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            if i >= self.skip:
                rows.append(parts)
            elif i >= self.skip - getattr(self, "pre", 0):
                warm.append(parts)
        os.unlink(self.f.name)
        note = None
        if not rows and warm:
            rows, note = warm[-1:], "no sample fell inside the timed region: the last warm-up sample"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": reasons, "samples": 0 if note else len(rows)}
        if note:
            out["note"] = note
        return out


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x, world, device=None):
    """Max over ranks of a float (the slowest rank sets the job's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks_(t, world):
    """In-place sum of a rank's partial count tensor over all ranks (the one
    8-byte exchange of a partitioned count); identity on one rank."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t)
    return t


def part_count_host(cost, per_item, part, nparts):
    """A rank's share of a list under eh_range_bounds' split: the sum of
    per_item over its range of items (host arrays; the multi-rank test's
    stand-in for the device count of that range)."""
    import paper_1503_02368_gb300 as eh
    lo, hi = eh.range_bounds(cost, part, nparts)
    return int(per_item[lo:hi].sum())


def step_stats(step_ms):
    """Per-step times: min, median, max, and the paper's protocol (Sec. 5.1.3):
    the fastest and slowest runs dropped, the rest averaged."""
    srt = sorted(step_ms)
    return {"min": srt[0], "median": statistics.median(srt), "max": srt[-1],
            "trimmed_mean": statistics.mean(srt[1:-1] if len(srt) > 2 else srt)}


def timed_steps(fn, steps, warmup, stream, flush, clocks=None):
    """fn() `warmup` times untimed, then `steps` times, each bracketed by CUDA
    events on `stream` with the L2 flushed before it (a write larger than L2,
    outside the events).  `clocks` (a started Clocks) is marked at the start of
    the timed region and stopped after it.  Returns (per-step ms, clocks)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if clocks is not None:
        clocks.mark()
    for k in range(steps):
        flush.fill_(k)
        evs[k][0].record(stream)
        fn()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks is not None else None
    return [a.elapsed_time(b) for a, b in evs], clk


def roofline(alg_bytes, ms, kernel, note=None):
    """HBM roofline of one launch: algorithmic bytes over the measured time
    against the measured copy bandwidth."""
    hbm, peak_kind = measured_peaks()
    achieved = alg_bytes / (ms / 1e3) / 1e9
    r = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
         "frac": round(achieved / hbm, 4), "peak_kind": peak_kind, "alg_bytes_per_launch": alg_bytes,
         "kernel": kernel}
    if note:
        r["note"] = note
    return r


def aggregate(edges_per_rank, ms_per_rank_max, world):
    """Whole-job throughput: all ranks' edges over the slowest rank's time."""
    return world * edges_per_rank / (ms_per_rank_max / 1e3)


def cpu_model():
    """The host CPU's model string (x86 'model name', Arm implementer/part), else the machine."""
    import platform
    try:
        names, parts = set(), set()
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            k, v = k.strip(), v.strip()
            if k == "model name":
                names.add(v)
            elif k in ("CPU implementer", "CPU part"):
                parts.add("%s %s" % (k, v))
        if names:
            return "; ".join(sorted(names))
        if parts:
            return "%s (%s)" % (platform.machine(), ", ".join(sorted(parts)))
    except OSError:
        pass
    return platform.machine()


def cpu_baseline(g, seconds, seed=7):
    """The oracle, as it stands, on a bounded sample of the outer loop: on all
    host cores (the reported value), and single-threaded on a smaller sample."""
    import numpy as np
    import oracle
    cores = os.cpu_count() or 1
    G = oracle.Graph(g["n"], g["src"], g["dst"])
    rng = np.random.default_rng(seed)
    verts = rng.permutation(g["n"]).astype(np.uint32)

    def run(nthreads, budget, start):
        # grow the sample until it has run `budget` seconds
        done_edges, t_total, pos, chunk = 0, 0.0, start, 4096
        while t_total < budget and pos < len(verts):
            part = verts[pos:pos + chunk]
            t0 = time.perf_counter()
            _, e = G.triangles_outer(part, nthreads=nthreads)
            t_total += time.perf_counter() - t0
            done_edges += e
            pos += len(part)
            chunk = min(chunk * 2, 1 << 20)
        return done_edges, t_total, pos - start

    e_all, t_all, v_all = run(cores, seconds, 0)
    e_one, t_one, v_one = run(1, seconds / 3, 0)
    return {"value": e_all / t_all, "unit": "edges/s", "cores": cores, "kind": "oracle",
            "sample": "outer-loop vertices %d of %d (random order, seed %d), %d pruned edges, %.1f s; "
                      "oracle adjacency build excluded" % (v_all, g["n"], seed, e_all, t_all),
            "cpu": cpu_model(),
            "single_thread": {"value": e_one / t_one, "unit": "edges/s", "cores": 1,
                              "sample": "the first %d vertices of the same order, %d pruned edges, %.1f s"
                                        % (v_one, e_one, t_one)}}


def bench_batch(eh, local, tau=32, reps=3):
    """4,096 triangle/4-clique queries on R-MAT-20 ego nets: one persistent batch
    vs one query at a time (same kernels); counts must agree exactly, and the
    oracle's sampled queries must match."""
    import numpy as np
    import torch
    from synth import workloads as W
    from paper_1503_02368_gb300 import autotune
    g = W.rmat20_ego_batch()
    pats = ["clique4" if p else "triangle" for p in g["patterns"]]
    best = autotune.load("rmat_s20_ego4096")
    if best:
        tau = best["tau"]
    xo = eh.exec_opts(cta_warps=best["cta_warps"], light_max=best["light_max"]) if best else None
    trie = eh.Trie(g["src"], g["dst"], g["n"], tau=tau)
    c0, s0 = trie.count_batch(pats, g["offsets"], g["pool"], mode=0, xopts=xo)      # warm-up
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    clk.mark()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        c, st = trie.count_batch(pats, g["offsets"], g["pool"], mode=0, xopts=xo)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    clocks = clk.stop()
    clk = Clocks(local)
    clk.start()
    clk.mark()
    t0 = time.perf_counter()
    c1, s1 = trie.count_batch(pats, g["offsets"], g["pool"], mode=1, xopts=xo)
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t0
    clocks_one = clk.stop()
    gold = golden("rmat_s20_ego4096")
    exact = all(int(c0[int(q)]) == v["count"] for q, v in gold["queries"].items())
    same = bool(np.array_equal(c0, c) and np.array_equal(c0, c1) and not s0.any() and not s1.any())
    trie.close()
    nq = len(pats)
    return {"workload": "rmat_s20_ef16 + 4096 ego nets |S| log-uniform 64..65536, triangle/4-clique alternating",
            "queries": nq, "subset_ids": int(len(g["pool"])), "tau": tau,
            "exec": {"cta_warps": best["cta_warps"], "light_max": best["light_max"]} if best else "defaults",
            "batched_qps": nq / min(ts), "batched_s": min(ts), "batched_s_all": ts,
            "one_launch_per_query_qps": nq / t_one, "one_launch_per_query_s": t_one, "speedup": t_one / min(ts),
            "same_counts": same, "exact": bool(exact and same), "exact_queries_checked": len(gold["queries"]),
            "clocks": clocks, "clocks_one_per_query": clocks_one,
            "timing": "host wall clock around eh_count_batch (host subsets in, counts out), best of %d" % reps}


def golden(name):
    return json.load(open(os.path.join(ROOT, "tests", "golden", "workload_counts.json")))[name]


def bench_er(eh, local, steps=500, warmup=5):
    """Whole-graph triangle count on Erdos-Renyi G(n=10,000, m=100,000).  The
    trie (about 0.8 MB) fits L2 many times over; L2 is flushed before each
    timed count all the same, so each count starts from DRAM."""
    import torch
    from synth import workloads as W
    g = W.er_10k_100k()
    gold = golden("er_n10000_m100000")
    trie = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    m = trie.stats()["n_edges"]
    info = trie.info("triangle")
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    clk = Clocks(local)
    clk.start()
    ms, clocks = timed_steps(lambda: trie.count_async("triangle", out.data_ptr(), stream=stream), steps, warmup,
                             stream, flush, clk)
    trie.status(stream)
    c = int(out.item())
    t = statistics.mean(ms)
    trie.close()
    return {"workload": "er_n10000_m100000 triangle: Erdos-Renyi G(n=10,000, m=100,000), seed 1504",
            "m_unique_edges": m, "count": c, "exact": c == gold["triangle"], "ms": t,
            "edges_per_s": m / (t / 1e3), "steps": steps, "step_ms": step_stats(ms),
            "roofline": roofline(info["alg_bytes"], t, "k_triangle<0,8>",
                                 "the whole trie is L2-resident after the first touch; DRAM-cold start per count"),
            "clocks": clocks, "timing": "CUDA events per count, L2 flushed before each (outside the events)"}


def bench_lollipop(eh, local, trie, xo, info, m, steps=10):
    """Whole-graph lollipop count (join semantics) on the resident R-MAT-22
    trie: the triangle traversal, each triangle adding its vertices' degrees."""
    import numpy as np
    import torch
    gold = golden("rmat_s22_ef16")
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    clk = Clocks(local)
    clk.start()
    ms, clocks = timed_steps(lambda: trie.count_async("lollipop", out.data_ptr(), xopts=xo, stream=stream), steps,
                             3, stream, flush, clk)
    trie.status(stream)
    c = int(out.item())
    t = statistics.mean(ms)
    if "lollipop" in gold:
        exact, how = c == gold["lollipop"], "equal to the oracle's count"
    else:
        # no oracle count at this size: the per-vertex identity L = sum_x 2 t(x) d(x) with t(x)
        # from the per-vertex kernel, whose sampled values are the oracle's
        vt = trie.vertex_triangles()
        ok_t = all(int(vt[int(v)]) == tv for v, tv in gold["vertex_triangles"].items())
        ex = trie.export(1)
        d_old = np.zeros(len(ex["len"]), np.uint64)
        d_old[ex["new_to_old"]] = ex["len"]
        exact = ok_t and c == int((2 * vt.astype(object) * d_old.astype(object)).sum())
        how = "sum_x 2 t(x) d(x) with t(x) checked at the oracle's sampled vertices"
    return {"workload": WORKLOAD.replace("triangle", "lollipop (join semantics)"), "count": c, "exact": bool(exact),
            "exact_how": how, "ms": t, "step_ms": step_stats(ms), "vs_triangle": None,
            "intersections_per_s": m / (t / 1e3),
            "roofline": roofline(info["alg_bytes"], t, "k_triangle<1,%d>" % xo.cta_warps,
                                 "the triangle traversal's algorithmic bytes (the degrees are 4 bytes a vertex "
                                 "more, read once per staged set)"),
            "clocks": clocks, "timing": "CUDA events per count, L2 flushed before each (outside the events)"}


def bench_clique4(eh, local, reps=10):
    """Whole-graph 4-clique count on the Chung-Lu graph (n = 1e6, ~2e7 edges,
    gamma 2.1), CUDA events per count with L2 flushed before each, roofline on
    the 4-clique algorithmic bytes; then the barbell by its two-node GHD plan
    and the selection queries on the same trie."""
    import numpy as np
    import torch
    from synth import workloads as W
    g = W.chunglu_1m()
    gold = golden("chunglu_n1000000_g2.1")
    trie = eh.Trie(g["src"], g["dst"], g["n"], tau=256)
    m = trie.stats()["n_edges"]
    xo = eh.exec_opts(cta_warps=16)
    info = trie.info("clique4", xopts=xo)
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    clk = Clocks(local)
    clk.start()
    ms, clocks = timed_steps(lambda: trie.count_async("clique4", out.data_ptr(), xopts=xo, stream=stream), reps, 2,
                             stream, flush, clk)
    trie.status(stream)
    c = int(out.item())
    t = statistics.mean(ms)
    # the barbell by its two-node GHD plan on the same graph (per-vertex triangles, then the edge join)
    clk = Clocks(local)
    clk.start()
    ms_b, clocks_b = timed_steps(lambda: trie.count_async("barbell", out.data_ptr(), stream=stream), 5, 1, stream,
                                 flush, clk)
    trie.status(stream)
    cb = int(out.item())
    # selection queries (Sec. 5.3) with the selected vertex = the 1000th-highest degree
    deg = np.zeros(g["n"], np.int64)
    np.add.at(deg, g["src"], 1)
    np.add.at(deg, g["dst"], 1)
    node = int(np.argsort(-deg, kind="stable")[1000])
    sel = {"node": node}
    for p in ("clique4", "barbell"):
        trie.count_selected(p, node)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c_sel = trie.count_selected(p, node)
        sel[p] = {"count": c_sel, "ms": (time.perf_counter() - t0) * 1e3}
    sel["timing"] = "host clock around one synchronous eh_count_selected"
    trie.close()
    return {"workload": "chunglu_n1000000_g2.1 (w_max 5e4, mean degree 40) 4-clique", "m_unique_edges": m,
            "count": c, "exact": c == gold["clique4"], "ms": t, "step_ms": step_stats(ms),
            "edges_per_s": m / (t / 1e3), "cliques_per_s": c / (t / 1e3),
            "intersections_per_s": (m + int(gold.get("triangle", 0))) / (t / 1e3),
            "intersections": "level 1: one per pruned edge (x, y); level 2: one per z in S_xy, i.e. one per "
                             "triangle (the oracle's count)",
            "tau": 256, "cta_warps": 16,
            "roofline": roofline(info["alg_bytes"], t, "k_clique4<16>",
                                 "4-clique algorithmic bytes: level 1 as the triangle pass, level 2 the pairs "
                                 "(S_<z, N+(z)), S spills of more than 512 elements written and read"),
            "clocks": clocks, "timing": "CUDA events per count, L2 flushed before each (outside the events)",
            "barbell": {"count": cb, "exact": cb == gold.get("barbell"), "ms": statistics.mean(ms_b),
                        "step_ms": step_stats(ms_b), "clocks": clocks_b,
                        "plan": "GHD: per-vertex triangle counts, then the U(x,x') join on the aggregates"},
            "selection": sel}


def bench_list(eh, trie, xo, alg_bytes, gold, reps=3):
    """Triangle listing (eh_list) of the resident R-MAT-22 trie into a device
    buffer of 3 x uint32 per triangle: count pass, scan, write pass."""
    import torch
    rows = gold["triangle"]
    buf = torch.empty((rows, 3), dtype=torch.int32, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    n = trie.list_into("triangle", buf.data_ptr(), rows, xopts=xo)       # warm-up
    stream = torch.cuda.current_stream()
    ms = []
    for k in range(reps):
        flush.fill_(k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        n = trie.list_into("triangle", buf.data_ptr(), rows, xopts=xo, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = min(ms)
    hbm, peak_kind = measured_peaks()
    out_bytes = 12.0 * rows
    achieved = (alg_bytes + out_bytes) / (t / 1e3) / 1e9
    del buf, flush
    torch.cuda.empty_cache()
    return {"workload": WORKLOAD + " triangle listing (rows of 3 x uint32 original ids, ascending)",
            "rows": n, "exact_vs_oracle_count": n == rows, "ms": t, "ms_all": ms,
            "rows_per_s": n / (t / 1e3), "output_gb": out_bytes / 1e9,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 4), "peak_kind": peak_kind,
                         "alg_bytes_per_call": alg_bytes + out_bytes,
                         "alg_bytes_note": "one traversal's lower-bound bytes + 12 bytes per written row; "
                                           "the call runs the traversal twice (count pass, write pass)"},
            "timing": "CUDA events around eh_list (both passes, the scan and its 8-byte D2H), min of %d" % reps}


ORDER_STUDY_GAMMAS = (1.8, 2.1, 2.5, 3.0)
ORDER_STUDY_TAUS = (0, 32, 256)


def bench_order(eh, n=1 << 20, n_pairs=8_000_000, reps=3):
    """Node orderings x layout granularity on triangle counting (App. "Node
    Ordering"; the relation- vs set-level study of Sec. 4.3): Chung-Lu graphs
    with degree exponent gamma, tau = 0 (relation level: every set uint),
    set level (tau = 32, the memory-neutral default; tau = 256, the paper's)
    and block level (256-value blocks, tau = 256).
    Times: trie build (the ordering included) on the host clock, the count by
    CUDA events (median of reps, L2 flushed before each)."""
    import torch
    import synth
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    orderings = list(eh.ORDERINGS)
    res = {"workload": "Chung-Lu n=2^20, %d raw pairs, w_max 5e4, gamma in %s; triangle count" %
                       (n_pairs, list(ORDER_STUDY_GAMMAS)),
           "taus": list(ORDER_STUDY_TAUS), "graphs": {}}
    for gi, gamma in enumerate(ORDER_STUDY_GAMMAS):
        s, d = synth.chunglu(n, n_pairs, synth.key(1503, 120, gi), gamma=gamma)
        rows, count0, m = {}, None, None
        for o in orderings:
            row = {}
            for tau in ORDER_STUDY_TAUS:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                t = eh.Trie(s, d, n, tau=tau, ordering=o, order_seed=1)
                torch.cuda.synchronize()
                if tau == 0:
                    row["build_ms"] = (time.perf_counter() - t0) * 1e3
                    st = t.stats()
                    m = st["n_edges"]
                    row["max_out_degree"] = st["max_out_degree"]
                t.count_async("triangle", out.data_ptr())
                ms = []
                for k in range(reps):
                    flush.fill_(k)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    t.count_async("triangle", out.data_ptr())
                    b.record()
                    torch.cuda.synchronize()
                    ms.append(a.elapsed_time(b))
                t.status()
                c = int(out.item())
                if count0 is None:
                    count0 = c
                assert c == count0, "triangle count changed with the ordering or layout"
                row["tri_ms_tau%d" % tau] = statistics.median(ms)
                t.close()
            # block level: 256-value blocks, bitset when 256 <= tau * count (tau = 256)
            t = eh.Trie(s, d, n, tau=256, ordering=o, order_seed=1, block_layout=True)
            t.count_async("triangle", out.data_ptr())
            ms = []
            for k in range(reps):
                flush.fill_(k)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                t.count_async("triangle", out.data_ptr())
                b.record()
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            t.status()
            assert int(out.item()) == count0, "triangle count changed with the block layout"
            row["tri_ms_block256"] = statistics.median(ms)
            t.close()
            rows[o] = row
        res["graphs"]["gamma_%.1f" % gamma] = {"m_unique_edges": m, "triangles": count0, "orderings": rows}
    return res


def bench_serve(eh, local, n_queries=1500, tau=32):
    """Resident R-MAT-24; ego-net queries (induced edges log-uniform 100..1e6),
    patterns uniform over triangle / 4-clique / lollipop; closed-loop saturation,
    then Poisson arrivals at 0.5x, 0.8x, 1.0x of it; p50/p99 latency."""
    import numpy as np
    from synth import workloads as W
    g = W.rmat24_serve(n_queries=n_queries)
    names = ("triangle", "clique4", "lollipop")
    pats = [names[p] for p in g["patterns"]]
    subsets = [g["pool"][g["offsets"][q]:g["offsets"][q + 1]] for q in range(n_queries)]
    trie = eh.Trie(g["src"], g["dst"], g["n"], tau=tau)
    budget = 48 << 30
    res = {"workload": "rmat_s24_ef16 resident; ego nets with induced edges log-uniform 100..1e6; "
                       "triangle/4-clique/lollipop uniform", "queries": n_queries,
           "budget_bytes": budget, "max_batch": 64, "max_inflight": 4, "tau": tau}

    def run(arrivals):
        srv = eh.Server(trie, budget, max_batch=64, max_inflight=4)
        tk = [None] * len(arrivals)
        sub_t = [0.0] * len(arrivals)
        t_start = time.perf_counter()
        for q, at in enumerate(arrivals):
            now = time.perf_counter() - t_start
            if at > now:
                time.sleep(at - now)
            while True:
                t = srv.submit(pats[q], subsets[q])
                if t is not None:
                    break
                time.sleep(0.0005)
            tk[q] = t
            sub_t[q] = time.perf_counter() - t_start
        out = [srv.wait(t, timeout_ms=600000) for t in tk]
        t_end = time.perf_counter() - t_start
        lat = [sub_t[q] - arrivals[q] + srv.latency(tk[q]) for q in range(len(arrivals))]
        st = srv.stats()
        srv.close()
        return out, lat, t_end, st

    run([0.0] * min(64, n_queries))                      # warm-up (kernels loaded, pool warmed)
    clk = Clocks(local)
    clk.start()
    clk.mark()
    out, lat, span, st = run([0.0] * n_queries)          # saturation (closed loop)
    res["saturation_clocks"] = clk.stop()
    sat = n_queries / span
    res["saturation_qps"] = sat
    res["saturation_mean_batch"] = st["mean_batch"]
    counts = [c for c, _ in out]
    ok_status = all(s_ == 0 for _, s_ in out)
    # each result equals the query alone, and the oracle's sampled queries
    rng = np.random.default_rng(0)
    sample = rng.choice(n_queries, size=min(256, n_queries), replace=False)
    # the same queries one at a time (eh_count over the subset: one device batch,
    # one count launch per query): equal results, and the plain baseline's rate
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    alone = [trie.count(pats[q], subset=subsets[q]) for q in sample]
    torch.cuda.synchronize()
    t_alone = time.perf_counter() - t0
    alone_ok = all(alone[i] == counts[q] for i, q in enumerate(sample))
    res["same_alone_and_in_mix"] = bool(alone_ok and ok_status)
    res["one_query_at_a_time_qps"] = len(sample) / t_alone
    res["one_query_at_a_time_sample"] = "%d queries drawn uniformly from the %d, run one after another" % (
        len(sample), n_queries)
    res["speedup_vs_one_at_a_time"] = sat / res["one_query_at_a_time_qps"]
    gold = golden("rmat_s24_serve")
    gq = {int(q): v for q, v in gold["queries"].items() if int(q) < n_queries}
    res["exact_vs_oracle_sample"] = all(counts[q] == v["count"] and pats[q] == v["pattern"] for q, v in gq.items())
    res["exact_queries_checked"] = len(gq)
    res["open_loop"] = []
    same_all = True
    for frac in (0.5, 0.8, 1.0):
        lam = frac * sat
        gaps = rng.exponential(1.0 / lam, size=n_queries)
        arr = np.cumsum(gaps) - gaps[0]
        clk = Clocks(local)
        clk.start()
        clk.mark()
        out2, lat2, span2, st2 = run(list(arr))
        clocks = clk.stop()
        same = [c for c, _ in out2] == counts
        same_all &= same
        res["open_loop"].append({"rate_qps": lam, "achieved_qps": n_queries / span2,
                                 "p50_ms": 1e3 * float(np.percentile(lat2, 50)),
                                 "p99_ms": 1e3 * float(np.percentile(lat2, 99)),
                                 "mean_batch": st2["mean_batch"], "same_counts": same, "clocks": clocks})
    res["exact"] = bool(res["same_alone_and_in_mix"] and res["exact_vs_oracle_sample"] and same_all)
    trie.close()
    return res


def headline_config(n, m, world):
    """The headline workload's config (both arms): graph, layout and launch knobs."""
    from paper_1503_02368_gb300 import autotune
    tuned = autotune.load("rmat_s22_triangle")
    return {"workload": WORKLOAD, "n_vertices": n, "m_unique_edges": m,
            "tau": tuned["tau"] if tuned else 32, "cta_warps": tuned["cta_warps"] if tuned else 8,
            "light_max": tuned["light_max"] if tuned else 32, "gallop_ratio": tuned.get("gallop_ratio", 32) if tuned else 32,
            "pair_warps": tuned.get("pair_warps", 1) if tuned else 1,
            "tuning": "autotuned (paper_1503_02368_gb300/tuned.json)" if tuned else "fixed",
            "l2": "flushed between timed steps (256 MiB write, outside the events)",
            "parallelism": "1 GPU" if world == 1 else
            "count partitioned over %d GPUs (replicated trie, cost-balanced work ranges, one 8-byte all-reduce)"
            % world}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from synth import workloads as W
    g = W.rmat22()
    import numpy as np
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.time()
    G = oracle.Graph(g["n"], g["src"], g["dst"])
    build_s = time.time() - t0
    rng = np.random.default_rng(11)
    verts = rng.permutation(g["n"]).astype(np.uint32)
    per_step = max(1.0, min(10.0, 120.0 / max(1, args.steps + args.warmup)))
    # size one step's sample from a probe
    t0 = time.perf_counter()
    _, e = G.triangles_outer(verts[:20000], nthreads=cores)
    probe = time.perf_counter() - t0
    k = int(min(len(verts), max(1000, 20000 * per_step / max(probe, 1e-3))))
    pos = 20000
    for _ in range(args.warmup):
        G.triangles_outer(verts[pos % len(verts):pos % len(verts) + k], nthreads=cores)
        pos += k
    tot_e, tot_t = 0, 0.0
    for _ in range(args.steps):
        a = pos % len(verts)
        part = verts[a:a + k]
        t0 = time.perf_counter()
        _, e = G.triangles_outer(part, nthreads=cores)
        tot_t += time.perf_counter() - t0
        tot_e += e
        pos += k
    value = tot_e / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak" if world == 1 else "strong", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic", "config": headline_config(g["n"], G.m, max(world, args.gpus)),
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": cores, "kind": "oracle",
                             "sample": "%d random outer-loop vertices per step of %d (the pruned edges they own "
                                       "counted); adjacency build %.1f s excluded" % (k, g["n"], build_s)},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def run_eh(args):
    import torch

    world, rank, local = dist_env()
    local = local % max(1, torch.cuda.device_count())   # ranks beyond the GPU count share GPUs (gloo only)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        if args.dist_backend == "nccl":
            dist.init_process_group("nccl", device_id=dev)
        else:
            dist.init_process_group("gloo")
    import paper_1503_02368_gb300 as eh
    from synth import workloads as W

    g = W.rmat22()
    gold = golden("rmat_s22_ef16")
    cfg0 = headline_config(g["n"], None, world)
    tau = args.tau if args.tau is not None else cfg0["tau"]
    fixed = args.tau is not None and args.tau != cfg0["tau"]
    warps = 8 if fixed else cfg0["cta_warps"]
    light_max = 32 if fixed else cfg0["light_max"]
    ratio = 32 if fixed else cfg0["gallop_ratio"]
    pw = 1 if fixed else cfg0["pair_warps"]
    xo = eh.exec_opts(cta_warps=warps, light_max=light_max, gallop_ratio=ratio, pair_warps=pw)
    trie = eh.Trie(g["src"], g["dst"], g["n"], tau=tau)
    m = trie.stats()["n_edges"]
    info = trie.info("triangle", xopts=xo)
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    if world == 1:
        def step():
            trie.count_async("triangle", out.data_ptr(), xopts=xo, stream=stream)
    else:
        # one graph per step: this rank's share of the work ranges, then the 8-byte sum
        def step():
            trie.count_range_async("triangle", rank, world, out.data_ptr(), xopts=xo, stream=stream)
            sum_over_ranks_(out, world)

    clocks = Clocks(local)   # sampling through the warm-up and the timed region
    clocks.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    trie.status(stream)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, clk = timed_steps(step, args.steps, 0, stream, flush, clocks)
    if world > 1:
        dist.barrier()
    trie.status(stream)
    count = int(out.item())
    exact = count == gold["triangle"]
    ms = sum(step_ms) / len(step_ms)
    ms_max = reduce_max(ms, world, dev)
    value = m / (ms_max / 1e3)          # one whole graph per step, on all ranks together

    roof = roofline(info["alg_bytes"], ms, "k_triangle<0,%d,%d>" % (warps, pw))
    roof["traffic"] = profile_traffic(os.path.join(ROOT, "paper_1503_02368_gb300", "csrc", "count.cu"))
    hbm = roof["peak"]
    st_ach = info["alg_bytes_stored"] / (ms / 1e3) / 1e9
    roof["stored_layout"] = {"achieved": round(st_ach, 1), "frac": round(st_ach / hbm, 4),
                             "alg_bytes_per_launch": info["alg_bytes_stored"],
                             "definition": "every set at its stored layout's size (4|S| uint, 4 x words bitset), "
                                           "N+(u) once per u, N+(v) once per pair (at most 32 B per element of "
                                           "N+(u) past the 32:1 ratio), 8 B per edge"}
    roof["definition"] = ("lower bound over the stored layouts: N+(u) once in its cheaper form, per pair the "
                          "cheapest read of what of N+(v) can meet N+(u)_<v, 8 B per edge")
    if world > 1:
        roof["note"] = "per rank: the whole graph's bytes over the partitioned step's time"

    e2e = None
    if not args.no_e2e:
        # the public API end to end: host edge list (pinned) in, count out
        src_p = torch.from_numpy(g["src"]).pin_memory()
        dst_p = torch.from_numpy(g["dst"]).pin_memory()
        ns, nd = src_p.numpy(), dst_p.numpy()
        e2e_steps = max(2, min(5, args.steps))

        def e2e_step():
            t = eh.Trie(ns, nd, g["n"], tau=tau)
            if world == 1:
                c = t.count("triangle", xopts=xo)
            else:
                t.count_range_async("triangle", rank, world, out.data_ptr(), xopts=xo, stream=stream)
                c = int(sum_over_ranks_(out, world).item())
                t.status(stream)
            t.close()
            return c

        e2e_step()     # warm-up
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        ok = True
        for _ in range(e2e_steps):
            ok &= e2e_step() == gold["triangle"]
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
        e2e_ms = reduce_max(e2e_ms, world, dev)
        e2e = {"value": m / (e2e_ms / 1e3), "unit": "edges/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": int(ns.nbytes + nd.nbytes), "d2h_bytes_per_step": 8, "exact": bool(ok),
               "includes": "H2D of the raw edge list, trie build (sort, dedup, ordering, layouts), work plan, "
                           "count%s, D2H of the count, trie release" % (" (this rank's range + all-reduce)"
                                                                         if world > 1 else "")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(g, args.cpu_seconds)

    legs = {"default": ("er", "lollipop", "clique4", "batch", "serve"),
            "all": ("er", "lollipop", "clique4", "batch", "serve", "list", "order"),
            "triangle": ()}.get(args.workload, (args.workload,))
    extra = {}
    if world == 1:
        for leg in legs:
            if leg == "er":
                extra["er"] = bench_er(eh, local)
            elif leg == "lollipop":
                extra["lollipop"] = bench_lollipop(eh, local, trie, xo, info, m)
                extra["lollipop"]["vs_triangle"] = extra["lollipop"]["ms"] / ms
            elif leg == "list":
                extra["list"] = bench_list(eh, trie, xo, info["alg_bytes"], gold)
            elif leg == "order":
                extra["order"] = bench_order(eh)
            elif leg == "clique4":
                extra["clique4"] = bench_clique4(eh, local)
            elif leg == "batch":
                extra["batch"] = bench_batch(eh, local)
            elif leg == "serve":
                extra["serve"] = bench_serve(eh, local, args.serve_queries)

    if rank == 0:
        cfg = headline_config(g["n"], m, world)
        cfg.update({"tau": tau, "cta_warps": warps, "light_max": light_max, "gallop_ratio": ratio, "pair_warps": pw})
        if fixed:
            cfg["tuning"] = "fixed"
        line = {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
                "scaling": "weak" if world == 1 else "strong", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic", "config": cfg, "count": count, "exact": exact,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": 2 * args.steps,
                "step_ms": step_stats(step_ms)}
        if extra:
            line["exact_all"] = bool(exact and all(v.get("exact", True) for v in extra.values()))
        line.update(extra)
        print(json.dumps(line), flush=True)
    trie.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_eh(args)


if __name__ == "__main__":
    main()
