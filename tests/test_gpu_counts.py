"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Counts are exact integers, so every comparison is bit-exact.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from synth import workloads as W
from tests import graphs as G

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workload_counts.json")))
PATS = ("triangle", "clique4", "lollipop", "lollipop_distinct")
TAUS = (0, 1, 8, 32, 256, 0xFFFFFFFF)


@pytest.fixture(scope="module")
def eh():
    import torch
    assert torch.cuda.is_available()
    import paper_1503_02368_gb300 as m
    return m


def both(eh, n, edges, tau=32):
    s, d = G.arrays(edges)
    return eh.Trie(s, d, n, tau=tau), oracle.Graph(n, s, d)


# ------------------------------------------------------------------ trie build

@pytest.mark.parametrize("seed", range(4))
def test_trie_build_matches_oracle(eh, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 400))
    e = G.random_graph(n, float(rng.choice([0.02, 0.1, 0.4])), rng)
    tau = [0, 8, 32, 0xFFFFFFFF][seed]
    t, o = both(eh, n, e, tau)
    x = t.export(0)
    sym = t.export(1)
    new2old = x["new_to_old"]
    assert new2old.tolist() == o.degree_order().tolist()       # (degree desc, id asc)
    old2new = np.empty(n, np.int64)
    old2new[new2old] = np.arange(n)
    st = t.stats()
    assert st["n_edges"] == o.m
    for v in range(n):
        N = np.sort(old2new[o.neighbours(int(new2old[v]))]).astype(np.uint32)
        b, ln = int(sym["off"][v]), int(sym["len"][v])
        assert b % 4 == 0
        assert np.array_equal(sym["nbr"][b:b + ln], N)
        assert np.all(sym["nbr"][b + ln:int(sym["off"][v + 1])] == 0xFFFFFFFF)
        P = N[N < v]
        b, ln = int(x["off"][v]), int(x["len"][v])
        assert b % 4 == 0 and ln == len(P)
        assert np.array_equal(x["nbr"][b:b + ln], P)
        # layout rule and bitset contents
        is_bs = x["bits_nwords"][v] > 0
        assert is_bs == oracle.layout_is_bitset(P, tau)
        if is_bs:
            lo, nw, wo = int(x["bits_lo"][v]), int(x["bits_nwords"][v]), int(x["bits_off"][v])
            assert lo % 128 == 0 and nw % 4 == 0 and wo % 4 == 0
            bits = np.unpackbits(x["words"][wo:wo + nw].view(np.uint8), bitorder="little")
            assert np.array_equal(np.nonzero(bits)[0] + lo, P)


@pytest.mark.parametrize("scale", (13, 17))
def test_trie_build_id_spaces_off_byte_boundaries(eh, scale):
    # 13- and 17-bit ids: the build's re-sort on the low endpoint alone must not
    # mix in the bits of the high endpoint packed above it
    g = W.rmat_graph(scale, 1503 + scale, edge_factor=8)
    n = g["n"]
    o = oracle.Graph(n, g["src"], g["dst"])
    t = eh.Trie(g["src"], g["dst"], n, tau=32)
    x, sym = t.export(0), t.export(1)
    new2old = x["new_to_old"]
    old2new = np.empty(n, np.int64)
    old2new[new2old] = np.arange(n)
    rng = np.random.default_rng(scale)
    for v in sorted(set(range(64)) | set(rng.choice(n, 1500, replace=False).tolist())):
        N = np.sort(old2new[o.neighbours(int(new2old[v]))]).astype(np.uint32)
        b, ln = int(sym["off"][v]), int(sym["len"][v])
        assert np.array_equal(sym["nbr"][b:b + ln], N), v
        b, ln = int(x["off"][v]), int(x["len"][v])
        assert np.array_equal(x["nbr"][b:b + ln], N[N < v]), v
    for p in ("lollipop", "barbell"):
        assert t.count(p) == o.count(p, nthreads=8), p


def test_invalid_ids_rejected(eh):
    with pytest.raises(eh.EHError) as ei:
        eh.Trie(np.array([0, 5], np.uint32), np.array([1, 2], np.uint32), 5)
    assert ei.value.status == 1


def test_empty_graphs(eh):
    t = eh.Trie(np.zeros(0, np.uint32), np.zeros(0, np.uint32), 10)
    for p in PATS:
        assert t.count(p) == 0
    t0 = eh.Trie(np.zeros(0, np.uint32), np.zeros(0, np.uint32), 0)
    assert t0.count("triangle") == 0
    t1 = eh.Trie(np.array([3, 3], np.uint32), np.array([3, 3], np.uint32), 4)   # loops only
    assert t1.count("triangle") == 0 and t1.stats()["n_edges"] == 0


# ------------------------------------------------------------------ counts

@pytest.mark.parametrize("seed", range(10))
def test_random_graphs_all_patterns(eh, seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(10, 300))
    e = G.random_graph(n, float(rng.choice([0.05, 0.2, 0.5, 0.8])), rng)
    tau = TAUS[seed % len(TAUS)]
    t, o = both(eh, n, e, tau)
    for p in PATS:
        assert t.count(p) == o.count(p), (p, tau)


@pytest.mark.parametrize("n", [3, 4, 5, 17, 33, 40, 64])
def test_complete_graphs(eh, n):
    t, _ = both(eh, n, G.complete(n))
    assert t.count("triangle") == math.comb(n, 3)
    assert t.count("clique4") == math.comb(n, 4)
    assert t.count("lollipop") == n * (n - 1) * (n - 2) * (n - 1)


def test_special_graphs(eh):
    for n, e, tri, k4 in [(10, G.petersen(), 0, 0), (9, G.wheel(8), 8, 0)]:
        t, _ = both(eh, n, e)
        assert t.count("triangle") == tri and t.count("clique4") == k4
    n, e = G.complete_multipartite(2, 2, 2, 2)
    t, _ = both(eh, n, e)
    assert t.count("clique4") == 16 and t.count("triangle") == 32


@pytest.mark.parametrize("tau", TAUS)
def test_layout_independence_rmat(eh, tau):
    # Sec. 4.4: layouts change speed only; every tau gives the oracle's counts
    g = W.rmat_graph(13, 1503 + 13)
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=tau)
    for p in PATS:
        assert t.count(p) == o.count(p, nthreads=8), (p, tau)


@pytest.mark.parametrize("xo", [dict(gallop_ratio=1), dict(gallop_ratio=1000), dict(light_max=2),
                                dict(light_max=8, cta_warps=4), dict(cta_warps=16), dict(light_max=32),
                                dict(pair_warps=2), dict(pair_warps=4), dict(pair_warps=4, cta_warps=4),
                                dict(pair_warps=2, cta_warps=16, light_max=8)])
def test_exec_knobs_do_not_change_counts(eh, xo):
    g = W.rmat_graph(12, 1503 + 12)
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    for tau in (0, 32):
        t = eh.Trie(g["src"], g["dst"], g["n"], tau=tau)
        x = eh.exec_opts(**xo)
        for p in PATS:
            assert t.count(p, xopts=x) == o.count(p, nthreads=8), (p, tau, xo)


def test_hub_graph_spans_many_tiles(eh):
    # a few hubs joined to everything: long sets (many 128-element chunks, ragged tails),
    # on-chip bitmaps and sorted arrays for the large-range sets
    rng = np.random.default_rng(7)
    n = 70000
    hubs = np.arange(6, dtype=np.uint32)
    e = [(int(h), int(v)) for h in hubs for v in rng.choice(np.arange(6, n), 3000, replace=False)]
    e += [(int(a), int(b)) for a, b in rng.integers(0, n, size=(40000, 2))]
    e += [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4)]
    s, d = G.arrays(e)
    o = oracle.Graph(n, s, d)
    for tau in (0, 32, 0xFFFFFFFF):
        t = eh.Trie(s, d, n, tau=tau)
        for p in PATS:
            assert t.count(p) == o.count(p, nthreads=8), (p, tau)


@pytest.mark.parametrize("pw", [1, 2, 4])
def test_warps_per_intersection_on_hub_graphs(eh, pw):
    # pairs (u, v) with N+(v) spanning many 128-word / 256-element steps, shared by
    # 1, 2 or 4 warps: every split must give the oracle's count
    rng = np.random.default_rng(11)
    n = 40000
    e = [(int(h), int(v)) for h in range(40) for v in rng.choice(np.arange(40, n), 2500, replace=False)]
    e += [(int(a), int(b)) for a, b in rng.integers(0, 400, size=(30000, 2))]
    s, d = G.arrays(e)
    o = oracle.Graph(n, s, d)
    want = {p: o.count(p, nthreads=8) for p in ("triangle", "lollipop", "lollipop_distinct")}
    for tau in (0, 32, 1024, 0xFFFFFFFF):
        t = eh.Trie(s, d, n, tau=tau)
        for w in (4, 8, 16):
            x = eh.exec_opts(pair_warps=pw, cta_warps=w)
            for p, c in want.items():
                assert t.count(p, xopts=x) == c, (p, tau, w, pw)
        t.close()


def test_vertex_triangles_small(eh):
    rng = np.random.default_rng(3)
    n = 500
    e = G.random_graph(n, 0.05, rng)
    t, o = both(eh, n, e)
    vt = t.vertex_triangles()
    assert np.array_equal(vt, o.vertex_triangles(np.arange(n, dtype=np.uint32)))
    assert int(vt.sum()) == 3 * o.triangles()


# ------------------------------------------------------------------ workloads

def test_er_workload(eh):
    g = W.er_10k_100k()
    gold = GOLD["er_n10000_m100000"]
    t = eh.Trie(g["src"], g["dst"], g["n"])
    assert t.stats()["n_edges"] == gold["m"]
    for p in PATS:
        assert t.count(p) == gold[p], p


def test_rmat16_workload(eh):
    g = W.rmat_graph(16, 1503 + 16)
    gold = GOLD["rmat_s16_ef16"]
    from tests.golden.make_golden import fingerprint
    assert fingerprint(g) == gold["fingerprint"]
    for tau in (8, 32, 256):
        t = eh.Trie(g["src"], g["dst"], g["n"], tau=tau)
        for p in PATS:
            assert t.count(p) == gold[p], (p, tau)


def test_rmat22_full_size(eh):
    g = W.rmat22()
    gold = GOLD["rmat_s22_ef16"]
    from tests.golden.make_golden import fingerprint
    assert fingerprint(g) == gold["fingerprint"]
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    assert t.stats()["n_edges"] == gold["m"]
    assert t.count("triangle") == gold["triangle"]
    vt = t.vertex_triangles()
    for v, want in gold["vertex_triangles"].items():
        assert int(vt[int(v)]) == want, v
    assert int(vt.sum()) == 3 * gold["triangle"]
    # lollipop by the same per-vertex counts (sum_x 2 t(x) d(x)) and degrees from the trie
    sym = t.export(1)
    deg = np.zeros(g["n"], np.uint64)
    deg[sym["new_to_old"]] = sym["len"]
    assert t.count("lollipop") == int((2 * vt.astype(object) * deg.astype(object)).sum())


def test_chunglu_full_size(eh):
    g = W.chunglu_1m()
    gold = GOLD["chunglu_n1000000_g2.1"]
    from tests.golden.make_golden import fingerprint
    assert fingerprint(g) == gold["fingerprint"]
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    assert t.stats()["n_edges"] == gold["m"]
    assert t.count("triangle") == gold["triangle"]
    assert t.count("clique4") == gold["clique4"]


def test_bounded_wait_reports_timeout_and_context_survives(eh):
    # a wait on a barrier phase nothing completes gives up and reports, no fault
    import time
    t0 = time.time()
    r = eh.lib().eh_selftest_wait_timeout(20000, None)      # 20 ms limit
    assert r == 4                                            # EH_ETIMEOUT
    assert time.time() - t0 < 10
    g = W.er_10k_100k()
    t = eh.Trie(g["src"], g["dst"], g["n"])
    assert t.count("triangle") == GOLD["er_n10000_m100000"]["triangle"]


def test_device_input_build_matches_host_build(eh):
    import torch
    g = W.rmat_graph(13, 1503 + 13)
    host = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    s = torch.from_numpy(g["src"].astype(np.int32)).cuda()
    d = torch.from_numpy(g["dst"].astype(np.int32)).cuda()
    dev = eh.Trie(s, d, g["n"], tau=32)
    for p in PATS:
        assert dev.count(p) == host.count(p)
    assert dev.stats()["n_edges"] == host.stats()["n_edges"]


def test_sparse_large_id_space(eh):
    # 2^24 ids, a few thousand edges spread over the whole range (24-bit keys)
    rng = np.random.default_rng(17)
    n = 1 << 24
    ids = rng.choice(n, 3000, replace=False).astype(np.uint32)
    e = [(int(ids[i]), int(ids[j])) for i, j in rng.integers(0, 3000, size=(20000, 2))]
    e += [(int(ids[i]), int(ids[j])) for i in range(40) for j in range(i + 1, 40)]   # a 40-clique
    s, d = G.arrays(e)
    o = oracle.Graph(n, s, d)
    t = eh.Trie(s, d, n, tau=32)
    for p in PATS:
        assert t.count(p) == o.count(p), p
    S = ids[:40]
    assert t.count("clique4", subset=S) == math.comb(40, 4)


def test_star_plus_clique_skew(eh):
    # one vertex adjacent to everything (degree n-1) next to a dense core:
    # every pruned set of the core contains the hub; tests both CTA and warp paths
    n = 5000
    e = [(0, v) for v in range(1, n)] + [(i, j) for i in range(1, 60) for j in range(i + 1, 60)]
    s, d = G.arrays(e)
    o = oracle.Graph(n, s, d)
    for tau in (0, 32, 0xFFFFFFFF):
        t = eh.Trie(s, d, n, tau=tau)
        assert t.count("triangle") == math.comb(59, 2) + math.comb(59, 3)
        for p in PATS:
            assert t.count(p) == o.count(p), (p, tau)


def test_injected_allocation_failures_release_everything(eh):
    # each device allocation of a trie build, a work plan and a query batch
    # fails in turn: the call returns EH_ENOMEM and keeps nothing allocated
    import torch
    L = eh.lib()
    g = W.rmat_graph(12, 1503 + 12)
    want = oracle.Graph(g["n"], g["src"], g["dst"]).triangles()
    off, pool = synth.ego_subsets(g["n"], g["src"], g["dst"], synth.key(3, 3), 8, 0, 8, 512)
    pats = ["triangle", "clique4"] * 4
    ref_t = eh.Trie(g["src"], g["dst"], g["n"])
    ref_b, _ = ref_t.count_batch(pats, off, pool)
    ref_t.close()
    eh.trim_memory()                                 # cached pool memory is not a leak
    free0 = torch.cuda.mem_get_info()[0]
    fails = {"build": 0, "plan": 0, "batch": 0}
    try:
        for k in range(200):                         # the trie build
            L.eh_test_fail_alloc_after(k)
            try:
                t = eh.Trie(g["src"], g["dst"], g["n"])
            except eh.EHError as e:
                assert e.status == 2, str(e)
                fails["build"] += 1
                continue
            L.eh_test_fail_alloc_after(-1)
            assert t.count("triangle") == want
            t.close()
            break
        for k in range(200):                         # the work plan (first count)
            t = eh.Trie(g["src"], g["dst"], g["n"])
            L.eh_test_fail_alloc_after(k)
            try:
                c = t.count("triangle")
            except eh.EHError as e:
                assert e.status == 2, str(e)
                fails["plan"] += 1
                L.eh_test_fail_alloc_after(-1)
                assert t.count("triangle") == want   # the plan builds on the next call
                t.close()
                continue
            L.eh_test_fail_alloc_after(-1)
            assert c == want
            t.close()
            break
        t = eh.Trie(g["src"], g["dst"], g["n"])
        for k in range(300):                         # a query batch
            L.eh_test_fail_alloc_after(k)
            cb, sb = t.count_batch(pats, off, pool)
            L.eh_test_fail_alloc_after(-1)
            if sb.any():
                assert set(sb.tolist()) == {2}
                fails["batch"] += 1
                continue
            assert np.array_equal(cb, ref_b)
            break
        t.close()
    finally:
        L.eh_test_fail_alloc_after(-1)
    assert fails["build"] > 10 and fails["plan"] > 2 and fails["batch"] > 10, fails
    eh.trim_memory()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < (64 << 20), (free0, free1)


# ------------------------------------------------------------------ barbell (two-node GHD plan)

@pytest.mark.parametrize("seed", range(4))
def test_barbell_random_graphs(eh, seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(10, 300))
    e = G.random_graph(n, float(rng.choice([0.05, 0.2, 0.5])), rng)
    for tau in (0, 32, 0xFFFFFFFF):
        t, o = both(eh, n, e, tau)
        assert t.count("barbell") == o.count("barbell"), tau


def test_barbell_closed_forms_and_workloads(eh):
    e = [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5), (0, 3)]
    t, _ = both(eh, 6, e)
    assert t.count("barbell") == 4 * 14
    t, _ = both(eh, 7, G.complete(7))
    assert t.count("barbell") == 7 * 6 * (2 * math.comb(6, 2)) ** 2
    g = W.rmat_graph(16, 1503 + 16)
    t = eh.Trie(g["src"], g["dst"], g["n"])
    assert t.count("barbell") == GOLD["rmat_s16_ef16"]["barbell"]


def test_barbell_is_whole_graph_only(eh):
    t, _ = both(eh, 7, G.complete(7))
    with pytest.raises(eh.EHError) as ei:
        t.count("barbell", subset=np.arange(5, dtype=np.uint32))
    assert ei.value.status == 1
    c, s = t.count_batch(["barbell", "barbell"], np.array([0, 0, 3], np.uint64), np.arange(3, dtype=np.uint32))
    assert s[0] == 0 and int(c[0]) == 7 * 6 * (2 * math.comb(6, 2)) ** 2   # whole graph in a batch
    assert s[1] == 1                                                        # with a subset: refused


def test_trie_stats_match_their_definitions(eh):
    # the statistics the build reduces on the device, recomputed from the oracle's
    # degrees and the exported trie
    for scale, tau in ((12, 32), (14, 256)):
        g = W.rmat_graph(scale, 1503 + scale)
        o = oracle.Graph(g["n"], g["src"], g["dst"])
        t = eh.Trie(g["src"], g["dst"], g["n"], tau=tau)
        st = t.stats()
        deg = o.degrees().astype(np.float64)
        x = t.export(0)
        assert st["n_active"] == int((deg > 0).sum())
        assert st["max_out_degree"] == int(x["len"].max())
        assert st["n_nonempty_sets"] == int((x["len"] > 0).sum())
        assert st["n_bitset_sets"] == int((x["bits_nwords"] > 0).sum())
        assert st["max_degree"] == int(deg.max())
        mean, sd = deg.mean(), deg.std()
        mode = int(np.bincount(deg.astype(np.int64)).argmax())
        assert st["density_skew"] == pytest.approx(3 * (mean - mode) / sd, rel=1e-9)


def test_pinned_host_input_read_in_place(eh):
    # pinned host edge lists are read by the device in place; the trie must be the
    # one built from the same edges in pageable memory
    import torch
    g = W.rmat_graph(14, 1503 + 14)
    s_p = torch.from_numpy(g["src"]).pin_memory()
    d_p = torch.from_numpy(g["dst"]).pin_memory()
    assert s_p.is_pinned()
    a = eh.Trie(s_p.numpy(), d_p.numpy(), g["n"], tau=32)
    b = eh.Trie(g["src"].copy(), g["dst"].copy(), g["n"], tau=32)
    xa, xb = a.export(0), b.export(0)
    for k in ("new_to_old", "off", "len", "nbr", "bits_nwords"):
        assert np.array_equal(xa[k], xb[k]), k
    assert a.count("clique4") == b.count("clique4")
