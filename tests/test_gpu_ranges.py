"""Partitioned whole-graph counts (eh_count_range) and the algorithmic byte
counts the roofline divides by (eh_count_info_get).

Range counts: the parts' results must sum to the oracle's count for every
splittable pattern and any number of parts.  Byte counts: recomputed here on
the host from the exported trie by each definition's rule, element by
element, and compared exactly.
"""
import json
import os

import numpy as np
import pytest

import oracle
from synth import workloads as W
from tests import graphs as G

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workload_counts.json")))
SPLIT_PATS = ("triangle", "clique4", "lollipop", "lollipop_distinct")


@pytest.fixture(scope="module")
def eh():
    import torch
    assert torch.cuda.is_available()
    import paper_1503_02368_gb300 as m
    return m


def hub_graph(n=3000, seed=0):
    # a few hubs joined to most vertices plus a random background: long pruned
    # sets (heavy CTA items) and many short ones (light warp items)
    rng = np.random.default_rng(seed)
    e = [(h, int(v)) for h in range(6) for v in rng.choice(n, n // 2, replace=False) if v != h]
    e += [tuple(map(int, rng.integers(0, n, 2))) for _ in range(15 * n)]
    return n, e


@pytest.mark.parametrize("nparts", [1, 2, 3, 8])
@pytest.mark.parametrize("tau", [0, 32, 0xFFFFFFFF])
def test_parts_sum_to_the_oracle_count(eh, nparts, tau):
    n, e = hub_graph(seed=tau & 7)
    s, d = G.arrays(e)
    o = oracle.Graph(n, s, d)
    t = eh.Trie(s, d, n, tau=tau)
    for p in SPLIT_PATS:
        want = o.count(p, nthreads=4)
        parts = [t.count_range(p, k, nparts) for k in range(nparts)]
        assert sum(parts) == want, (p, parts, want)
        assert t.count(p) == want
    t.close()


@pytest.mark.parametrize("nparts", [2, 3, 8])
def test_parts_sum_on_rmat16(eh, nparts):
    g = W.rmat_graph(16, 1503 + 16)
    gold = GOLD["rmat_s16_ef16"]
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    for p in SPLIT_PATS:
        assert sum(t.count_range(p, k, nparts) for k in range(nparts)) == gold[p]
    t.close()


def test_parts_are_balanced_and_all_busy(eh):
    g = W.rmat_graph(16, 1503 + 16)
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    parts = [t.count_range("triangle", k, 4) for k in range(4)]
    assert all(c > 0 for c in parts)
    t.close()


def test_async_range_matches_and_block_layout_uses_set_kernel(eh):
    import torch
    g = W.rmat_graph(14, 1503 + 14)
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    want = o.count("triangle", nthreads=4)
    for blocks in (False, True):
        t = eh.Trie(g["src"], g["dst"], g["n"], tau=256, block_layout=blocks)
        out = torch.zeros(3, dtype=torch.int64, device="cuda")
        tot = 0
        for k in range(3):
            t.count_range_async("triangle", k, 3, out[k].data_ptr())
            t.status()
        tot = int(out.sum().item())
        assert tot == want
        t.close()


def test_range_rejects_bad_arguments(eh):
    n, e = hub_graph(500)
    s, d = G.arrays(e)
    t = eh.Trie(s, d, n)
    for args in (("barbell", 0, 2), ("triangle", 2, 2), ("triangle", 0, 0)):
        with pytest.raises(eh.EHError) as ei:
            t.count_range(*args)
        assert ei.value.status == 1
    assert t.count_range("triangle", 0, 1) == t.count("triangle")
    t.close()


def test_empty_graph_and_more_parts_than_items(eh):
    t = eh.Trie(np.zeros(0, np.uint32), np.zeros(0, np.uint32), 10)
    assert [t.count_range("triangle", k, 4) for k in range(4)] == [0, 0, 0, 0]
    t.close()
    s, d = G.arrays(G.complete(5))
    t = eh.Trie(s, d, 5)
    assert sum(t.count_range("clique4", k, 64) for k in range(64)) == 5
    assert sum(t.count_range("triangle", k, 64) for k in range(64)) == 10
    t.close()


# ------------------------------------------------------------ byte counts

def _exported(t):
    x = t.export(0)
    n = len(x["len"])
    sets = [x["nbr"][int(x["off"][v]):int(x["off"][v]) + int(x["len"][v])].astype(np.int64) for v in range(n)]
    return x, sets


def _pair_bytes(nz, nwz, loz, r, p_lo, p_hi, ratio=32):
    # the lower-bound reading for one pair (P on chip, r elements, words
    # [p_lo, p_hi)) against B = N+(z): uint array, galloping cap, bitset words
    bb = 4 * nz
    if nz > ratio * r and 32 * r < bb:
        bb = 32 * r
    if nwz:
        lo, hi = max(p_lo, loz), min(p_hi, loz + nwz)
        wb = 4 * (hi - lo) if hi > lo else 0
        wb = min(wb, 32 * r)
        bb = min(bb, wb)
    return bb


def host_alg_bytes(x, sets, m, ratio=32):
    """Triangle pass, lower bound (the definition eh_count_info_get's alg_bytes states)."""
    nw, lw = x["bits_nwords"].astype(np.int64), (x["bits_lo"].astype(np.int64) // 32)
    b = 8 * m
    for u, A in enumerate(sets):
        if len(A) < 2:
            continue
        a_lo, a_hi = (int(A[0]) >> 7) << 2, (int(A[-1]) >> 5) + 1
        for j in range(1, len(A)):
            v = int(A[j])
            if len(sets[v]) == 0:
                continue
            b += _pair_bytes(len(sets[v]), int(nw[v]), int(lw[v]), j, a_lo, a_hi, ratio)
        b += 4 * int(nw[u]) if nw[u] and nw[u] < len(A) else 4 * len(A)
    return b


def host_alg_bytes_stored(x, sets, m, ratio=32):
    """Triangle pass with every set at its stored layout's size."""
    nw = x["bits_nwords"].astype(np.int64)
    size = [4 * int(nw[v]) if nw[v] else 4 * len(sets[v]) for v in range(len(sets))]
    b = 8 * m
    for u, A in enumerate(sets):
        for v in A:
            v = int(v)
            bb = size[v]
            if len(sets[v]) > ratio * len(A) and 32 * len(A) < bb:
                bb = 32 * len(A)
            b += bb
        b += size[u]
    return b


def _pair_bytes_vec(nz, nwz, loz, r, p_lo, p_hi, ratio=32):
    # _pair_bytes over arrays (int64): one entry per pair
    bb = 4 * nz
    gal = (nz > ratio * r) & (32 * r < bb)
    bb = np.where(gal, 32 * r, bb)
    lo, hi = np.maximum(p_lo, loz), np.minimum(p_hi, loz + nwz)
    wb = np.minimum(np.where(hi > lo, 4 * (hi - lo), 0), 32 * r)
    return np.where(nwz > 0, np.minimum(bb, wb), bb)


def host_alg_bytes_k4(x, sets, m, ratio=32, s_cap=512):
    """4-clique pass: A once, level 1 pairs (A_<y, N+(y)), level 2 pairs
    (S_<z, N+(z)), spills of S longer than the on-chip buffer."""
    nw, lw = x["bits_nwords"].astype(np.int64), (x["bits_lo"].astype(np.int64) // 32)
    ln = np.array([len(q) for q in sets], np.int64)
    b = 8 * m
    for xv, A in enumerate(sets):
        if len(A) < 3:
            continue
        a_lo, a_hi = (int(A[0]) >> 7) << 2, (int(A[-1]) >> 5) + 1
        b += 4 * int(nw[xv]) if nw[xv] and nw[xv] < len(A) else 4 * len(A)
        for j in range(2, len(A)):
            y = int(A[j])
            By = sets[y]
            if len(By) < 2:
                continue
            b += _pair_bytes(len(By), int(nw[y]), int(lw[y]), j, a_lo, a_hi, ratio)
            S = By[np.isin(By, A)]
            if len(S) >= 2:
                z, r, prev = S[1:], np.arange(1, len(S), dtype=np.int64), S[:-1]
                keep = ln[z] > 0
                pb = _pair_bytes_vec(ln[z], nw[z], lw[z], r, (int(S[0]) >> 7) << 2, (prev >> 5) + 1, ratio)
                b += int(pb[keep].sum())
            if len(S) > s_cap:
                b += 8 * len(S)
    return b


@pytest.mark.parametrize("tau", [0, 32, 1024, 0xFFFFFFFF])
def test_algorithmic_bytes_match_host_recomputation(eh, tau):
    n, e = hub_graph(800, seed=3)
    s, d = G.arrays(e)
    t = eh.Trie(s, d, n, tau=tau)
    m = t.stats()["n_edges"]
    x, sets = _exported(t)
    tri = t.info("triangle")
    assert tri["alg_bytes"] == host_alg_bytes(x, sets, m)
    assert tri["alg_bytes_stored"] == host_alg_bytes_stored(x, sets, m)
    k4 = t.info("clique4")
    assert k4["alg_bytes"] == host_alg_bytes_k4(x, sets, m)
    assert k4["alg_bytes_stored"] == 0
    t.close()


def test_k4_bytes_count_spills_of_long_intermediate_sets(eh):
    # a 560-clique: S sets of up to 558 elements exceed the 512-element buffer
    n = 1400
    s, d = G.arrays(G.complete(560) + [(560 + i, i % 560) for i in range(800)])
    t = eh.Trie(s, d, n, tau=32)
    m = t.stats()["n_edges"]
    x, sets = _exported(t)
    got = t.info("clique4")["alg_bytes"]
    assert got == host_alg_bytes_k4(x, sets, m)
    assert got > host_alg_bytes_k4(x, sets, m, s_cap=10 ** 9)       # the spill term is present
    t.close()
