"""Induced-subgraph counts and query batches (CUDA path vs the oracle)."""
import math

import numpy as np
import pytest

import oracle
import synth
from synth import workloads as W
from tests import graphs as G

pytestmark = pytest.mark.gpu
PATS = ("triangle", "clique4", "lollipop", "lollipop_distinct")


@pytest.fixture(scope="module")
def eh():
    import torch
    assert torch.cuda.is_available()
    import paper_1503_02368_gb300 as m
    return m


@pytest.fixture(scope="module")
def rmat12():
    g = W.rmat_graph(12, 1503 + 12)
    return g, oracle.Graph(g["n"], g["src"], g["dst"])


def test_single_subset_counts(eh, rmat12):
    g, o = rmat12
    rng = np.random.default_rng(5)
    for tau in (0, 32, 0xFFFFFFFF):
        t = eh.Trie(g["src"], g["dst"], g["n"], tau=tau)
        for trial in range(4):
            S = rng.choice(g["n"], size=int(rng.integers(5, 2000)), replace=False).astype(np.uint32)
            S = np.concatenate([S, S[: len(S) // 5]])          # repeats and any order are allowed
            rng.shuffle(S)
            sub = o.induced(S)
            for p in PATS:
                assert t.count(p, subset=S) == sub.count(p), (p, tau, trial)


def test_subset_whole_graph_and_clique(eh):
    n = 60
    rng = np.random.default_rng(2)
    e = G.random_graph(n, 0.2, rng) + [(i, j) for i in range(40, 52) for j in range(i + 1, 52)]
    s, d = G.arrays(e)
    t = eh.Trie(s, d, n)
    o = oracle.Graph(n, s, d)
    allv = np.arange(n, dtype=np.uint32)
    for p in PATS:
        assert t.count(p, subset=allv) == o.count(p)
    K = np.arange(40, 52, dtype=np.uint32)
    assert t.count("triangle", subset=K) == math.comb(12, 3)
    assert t.count("clique4", subset=K) == math.comb(12, 4)
    assert t.count("triangle", subset=np.array([7], np.uint32)) == 0


def test_batch_mixed_patterns_and_errors(eh, rmat12):
    g, o = rmat12
    rng = np.random.default_rng(9)
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    sets, pats = [], []
    for i in range(40):
        sets.append(rng.choice(g["n"], size=int(rng.integers(1, 3000)), replace=False).astype(np.uint32))
        pats.append(PATS[i % 4])
    sets[7] = np.array([1, 2, g["n"] + 5], np.uint32)      # an invalid id fails only its own query
    sets[11] = np.zeros(0, np.uint32)                       # empty subset = the whole graph
    off = np.zeros(len(sets) + 1, np.uint64)
    off[1:] = np.cumsum([len(x) for x in sets])
    pool = np.concatenate(sets)
    c0, s0 = t.count_batch(pats, off, pool, mode=0)
    c1, s1 = t.count_batch(pats, off, pool, mode=1)
    assert s0[7] == 1 and s1[7] == 1
    assert np.all(np.delete(s0, 7) == 0) and np.all(np.delete(s1, 7) == 0)
    assert np.array_equal(c0, c1)
    for i in range(len(sets)):
        if i == 7:
            continue
        want = o.count(pats[i]) if len(sets[i]) == 0 else o.induced(sets[i]).count(pats[i])
        assert int(c0[i]) == want, (i, pats[i])


def test_ego_batch_matches_oracle(eh):
    g = W.rmat_graph(14, 1503 + 14)
    off, pool = synth.ego_subsets(g["n"], g["src"], g["dst"], synth.key(1503, 14, 1), 96, 0, 16, 4096)
    pats = ["triangle" if q % 2 == 0 else "clique4" for q in range(96)]
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    c0, s0 = t.count_batch(pats, off, pool, mode=0)
    c1, s1 = t.count_batch(pats, off, pool, mode=1)
    assert not s0.any() and not s1.any()
    assert np.array_equal(c0, c1)
    for q in range(96):
        assert int(c0[q]) == o.induced(pool[off[q]:off[q + 1]]).count(pats[q]), q


def test_batch_knobs_do_not_change_counts(eh, rmat12):
    g, o = rmat12
    off, pool = synth.ego_subsets(g["n"], g["src"], g["dst"], synth.key(7, 7), 32, 0, 8, 2048)
    pats = [PATS[q % 4] for q in range(32)]
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=8)
    ref, _ = t.count_batch(pats, off, pool)
    for xo in (dict(light_max=2), dict(cta_warps=4), dict(cta_warps=16, gallop_ratio=1)):
        c, st = t.count_batch(pats, off, pool, xopts=eh.exec_opts(**xo))
        assert not st.any() and np.array_equal(c, ref), xo
    for q in range(32):
        assert int(ref[q]) == o.induced(pool[off[q]:off[q + 1]]).count(pats[q])


def test_rmat20_ego4096_workload(eh):
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workload_counts.json")))
    gold = gold["rmat_s20_ego4096"]
    g = W.rmat20_ego_batch()
    from tests.golden.make_golden import fingerprint
    assert fingerprint(g) == gold["fingerprint"]
    off, pool, pq = g["offsets"], g["pool"], g["patterns"]
    pats = ["clique4" if p else "triangle" for p in pq]
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    c0, s0 = t.count_batch(pats, off, pool, mode=0)
    assert not s0.any()
    for q, rec in gold["queries"].items():       # oracle counts of a sample, incl. the 4 largest
        assert pats[int(q)] == rec["pattern"]
        assert int(c0[int(q)]) == rec["count"], (q, rec)


def test_batch_count_graph_is_reused_across_calls(eh, rmat12):
    # each device batch's count phase is a CUDA graph; after the first, the
    # calling thread's executable graph is updated in place and relaunched
    g, o = rmat12
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    off, pool = synth.ego_subsets(g["n"], g["src"], g["dst"], synth.key(3, 3), 8, 0, 16, 400)
    pats = ["triangle", "clique4"] * 4
    c0, s0 = t.count_batch(pats, off, pool)                   # instantiates (or reuses) the graph
    c1, s1 = t.count_batch(pats, off, pool, mode=1)           # one device batch per query
    prof = eh.batch_profile()
    assert prof["batches"] == 8 and prof["graph_reuses"] >= 7
    assert not s0.any() and not s1.any() and np.array_equal(c0, c1)
    for q in range(8):
        assert int(c1[q]) == o.induced(pool[off[q]:off[q + 1]]).count(pats[q])
    t.close()
