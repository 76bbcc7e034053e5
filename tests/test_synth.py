"""The seeded input generators: determinism and recipe checks."""
import json
import os

import numpy as np
import pytest

import synth
from synth import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "workload_counts.json")


def test_rng_counter_based():
    k = synth.key(1503, 1)
    assert synth.rng(k, 5) == synth.rng(k, 5)
    assert synth.rng(k, 5) != synth.rng(k, 6)
    assert synth.key(1503, 1) != synth.key(1503, 2)


def test_det_log_exp_accuracy():
    L = synth.lib()
    for x in [1e-3, 0.5, 1.0, 2.0, 49.7, 1e6 + 49.7]:
        assert abs(L.synth_det_log(x) - np.log(x)) < 1e-13 * max(1, abs(np.log(x)))
    for y in [-20.0, -1.0, 0.0, 0.3, 5.0, 12.0]:
        assert abs(L.synth_det_exp(y) - np.exp(y)) <= 1e-14 * np.exp(y)


def test_er_exact_distinct():
    s, d = synth.er(300, 5000, synth.key(7))
    pairs = {(min(a, b), max(a, b)) for a, b in zip(s.tolist(), d.tolist())}
    assert len(pairs) == 5000 and all(a != b for a, b in pairs)
    assert max(max(p) for p in pairs) < 300
    with pytest.raises(ValueError):
        synth.er(10, 46, synth.key(7))
    s2, d2 = synth.er(10, 45, synth.key(7))     # the complete graph
    assert len({(min(a, b), max(a, b)) for a, b in zip(s2.tolist(), d2.tolist())}) == 45


def test_rmat_thread_independent_and_skewed():
    k = synth.key(1, 2)
    s1, d1 = synth.rmat(12, 40000, k, nthreads=1)
    s4, d4 = synth.rmat(12, 40000, k, nthreads=4)
    assert np.array_equal(s1, s4) and np.array_equal(d1, d4)
    assert s1.max() < 4096 and d1.max() < 4096
    # top bit of src is 1 with probability c + d = 0.24
    frac = ((s1 >> 11) & 1).mean()
    assert abs(frac - 0.24) < 0.01


def test_chunglu_recipe():
    w0 = synth.chunglu_weight(0)
    assert abs(w0 - 50000.0) < 1e-6 * 50000
    i = np.arange(0, 1_000_000, 997)
    w = np.array([synth.chunglu_weight(int(x)) for x in i])
    assert np.all(np.diff(w) < 0)
    # sum of expected degrees = 4e7 (mean 40) up to the rounding of i0
    total = sum(synth.chunglu_weight(x) for x in range(1_000_000))
    assert abs(total - 4e7) < 1e-4 * 4e7
    k = synth.key(3)
    s1, d1 = synth.chunglu(1000, 20000, k, nthreads=1)
    s2, d2 = synth.chunglu(1000, 20000, k, nthreads=3)
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)
    assert np.bincount(s1, minlength=1000)[0] > np.bincount(s1, minlength=1000)[999]


def test_ego_subsets_are_bfs_prefixes():
    s, d = synth.rmat(12, 16 * 4096, synth.key(4, 4))
    off, pool = synth.ego_subsets(4096, s, d, synth.key(4, 5), 64, 0, 8, 512, nthreads=2)
    adj = [set() for _ in range(4096)]
    for a, b in zip(s.tolist(), d.tolist()):
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    for q in range(64):
        S = pool[off[q]:off[q + 1]].tolist()
        assert len(S) == len(set(S)) and len(S) <= 512
        assert len(adj[S[0]]) > 0
        seen = {S[0]}
        for v in S[1:]:                       # every later vertex touches an earlier one
            assert adj[v] & seen
            seen.add(v)
    off2, pool2 = synth.ego_subsets(4096, s, d, synth.key(4, 5), 64, 0, 8, 512, nthreads=5)
    assert np.array_equal(off, off2) and np.array_equal(pool, pool2)
    # mode 1: induced-edge targets
    off3, pool3 = synth.ego_subsets(4096, s, d, synth.key(4, 6), 16, 1, 10, 1000, nthreads=2)
    for q in range(16):
        S = set(pool3[off3[q]:off3[q + 1]].tolist())
        ind = sum(1 for v in S for w in adj[v] if w in S and w > v)
        assert ind >= 10 or len(S) < 4096


@pytest.mark.parametrize("name,fn", [("er_n10000_m100000", W.er_10k_100k),
                                     ("rmat_s16_ef16", lambda: W.rmat_graph(16, 1503 + 16))])
def test_workload_fingerprints(name, fn):
    from tests.golden.make_golden import fingerprint
    gold = json.load(open(GOLD))[name]
    g = fn()
    assert fingerprint(g) == gold["fingerprint"]
