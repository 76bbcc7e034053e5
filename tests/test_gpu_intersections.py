"""One intersection at a time, through the whole count path.

With the identity ordering a graph can pin one pair exactly: u = n-1 is
joined to v = n-2 and to every a in A, and v to every b in B (all of A, B
below v).  Then N+(u) = A + {v}, N+(v) = B, no other pair meets, and the
triangle count is |A ∩ B|.  The cases cover size ratios from 1:1 to 1:10^4,
empty, singleton, disjoint, identical and adjacent sets, sets starting at
id 0 and ending just below v, ranges that are not whole 32-bit words, dense
sets (bitset layouts), a range too wide for the on-chip bitmap and sets too
long for on-chip staging, each on the light (|N+(u)| <= 32) and heavy paths
and at several layout thresholds.  The CPU test checks every construction
against the oracle and against numpy's sorted-set intersection; the GPU
test compares the count path with both.
"""
import numpy as np
import pytest

import oracle


def _cases():
    rng = np.random.default_rng(1503)
    cases = []

    def add(name, n, A, B):
        A = np.unique(np.asarray(A, np.int64))
        B = np.unique(np.asarray(B, np.int64))
        assert A.size == 0 or (A.min() >= 0 and A.max() < n - 2)
        assert B.size == 0 or (B.min() >= 0 and B.max() < n - 2)
        cases.append((name, n, A, B))

    n = 4096
    add("empty A", n, [], rng.choice(n - 2, 50, replace=False))
    add("empty B", n, rng.choice(n - 2, 50, replace=False), [])
    add("singleton meet", n, [7], [3, 7, 11])
    add("disjoint interleaved", n, np.arange(0, 2000, 2), np.arange(1, 2000, 2))
    add("identical", n, np.arange(100, 1100), np.arange(100, 1100))
    add("adjacent ranges", n, np.arange(0, 500), np.arange(500, 1000))
    add("from id 0, ragged words", n, np.arange(0, 45), np.arange(0, 77, 3))
    add("up to v-1", n, np.arange(n - 40, n - 2), np.arange(n - 100, n - 2, 2))
    add("light, 5 of 31", n, rng.choice(n - 2, 31, replace=False), rng.choice(n - 2, 300, replace=False))
    for ratio in (1, 10, 100, 1000, 10000):
        nn = max(4096, 3 * 10 * ratio)
        small = rng.choice(nn - 2, 10, replace=False)
        big = np.union1d(rng.choice(nn - 2, 10 * ratio, replace=False), small[::2])
        add("ratio 1:%d (A small)" % ratio, nn, small, big)
        add("ratio 1:%d (B small)" % ratio, nn, big, small)
    n = 1 << 14
    add("dense both", n, np.arange(1000, 5000), np.arange(0, 8000, 3))
    add("dense A, sparse B", n, np.arange(2000, 6000), rng.choice(n - 2, 200, replace=False))
    n = 1 << 21
    wide = np.sort(rng.choice(n - 2, 3000, replace=False))
    add("range wider than the on-chip bitmap", n, wide, np.union1d(wide[::3], rng.choice(n - 2, 2000, replace=False)))
    longA = np.sort(rng.choice(n - 2, 9000, replace=False))
    add("A longer than on-chip staging", n, longA, np.union1d(longA[1::4], rng.choice(n - 2, 5000, replace=False)))
    return cases


CASES = _cases()
TAUS = (0, 8, 32, 256, 0xFFFFFFFF)


def graph(n, A, B):
    u, v = n - 1, n - 2
    src = np.concatenate([[u], np.full(A.size, u), np.full(B.size, v)]).astype(np.uint32)
    dst = np.concatenate([[v], A, B]).astype(np.uint32)
    return src, dst


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_construction_pins_one_intersection(case):
    _, n, A, B = case
    s, d = graph(n, A, B)
    want = int(np.intersect1d(A, B).size)
    o = oracle.Graph(n, s, d)
    assert o.triangles() == want
    # identity order: N+(u) = A + {v}, N+(v) = B
    assert o.vertex_order("identity", 0).tolist() == list(range(n))


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_count_path_one_intersection(case):
    import torch
    assert torch.cuda.is_available()
    import paper_1503_02368_gb300 as eh
    _, n, A, B = case
    s, d = graph(n, A, B)
    want = int(np.intersect1d(A, B).size)
    for tau in TAUS:
        t = eh.Trie(s, d, n, tau=tau, ordering="identity")
        assert t.count("triangle") == want, tau
        assert t.count("triangle", xopts=eh.exec_opts(light_max=8)) == want, tau
        t.close()
