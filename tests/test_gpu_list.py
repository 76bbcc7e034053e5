"""Parity of triangle / 4-clique listing (eh_list) with the oracle.

The row order of eh_list is unspecified, so rows are compared as sets: both
sides sorted lexicographically, then equal element by element (ids are exact
integers: bit-exact).  At full size, where the oracle cannot list everything
in seconds, the listing is checked by properties that together fix the set:
the row count equals the oracle's count, every row is a clique of the input
edge list (looked up with plain torch searches), no row repeats, and the rows
at sampled vertices equal the oracle's rows at those vertices.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from synth import workloads as W
from tests import graphs as G

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workload_counts.json")))
WIDTH = {"triangle": 3, "clique4": 4}


@pytest.fixture(scope="module")
def eh():
    import torch
    assert torch.cuda.is_available()
    import paper_1503_02368_gb300 as m
    return m


def lexsorted(rows):
    rows = np.ascontiguousarray(rows, np.uint32)
    if len(rows) == 0:
        return rows
    return rows[np.lexsort(rows.T[::-1])]


def gpu_rows(t, pattern, xopts=None):
    return lexsorted(t.list(pattern, xopts=xopts).cpu().numpy().view(np.uint32))


def check_small(eh, n, edges, taus=(0, 32, 0xFFFFFFFF), patterns=("triangle", "clique4"), xopts=None):
    s, d = G.arrays(edges)
    o = oracle.Graph(n, s, d)
    for tau in taus:
        t = eh.Trie(s, d, n, tau=tau)
        for p in patterns:
            got = gpu_rows(t, p, xopts)
            want = lexsorted(o.list(p))
            assert got.shape == want.shape, (p, tau, got.shape, want.shape)
            assert np.array_equal(got, want), (p, tau)


# ------------------------------------------------------------ small graphs

@pytest.mark.parametrize("seed", range(8))
def test_random_graphs_list_like_oracle(eh, seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(10, 300))
    e = G.random_graph(n, float(rng.choice([0.05, 0.2, 0.5])), rng)
    check_small(eh, n, e)


@pytest.mark.parametrize("n", [3, 4, 5, 33, 40, 64])
def test_complete_graphs_list_every_subset(eh, n):
    import itertools
    s, d = G.arrays(G.complete(n))
    t = eh.Trie(s, d, n, tau=32)
    assert gpu_rows(t, "triangle").tolist() == [list(q) for q in itertools.combinations(range(n), 3)]
    k4 = gpu_rows(t, "clique4")
    assert len(k4) == math.comb(n, 4)
    if n <= 40:
        assert k4.tolist() == [list(q) for q in itertools.combinations(range(n), 4)]


def test_empty_and_triangle_free(eh):
    for n, e in ((5, []), (10, G.petersen()), (50, G.star(50)), (9, G.cycle(9))):
        s, d = G.arrays(e)
        t = eh.Trie(s, d, n, tau=32)
        assert tuple(t.list("triangle").shape) == (0, 3)
        assert tuple(t.list("clique4").shape) == (0, 4)
        assert t.list_into("triangle", 0, 0) == 0


@pytest.mark.parametrize("xo", [dict(gallop_ratio=1), dict(gallop_ratio=1000), dict(light_max=2),
                                dict(light_max=8), dict(flags=1), dict(flags=2), dict(flags=1, gallop_ratio=1)])
def test_exec_knobs_and_staging_forms(eh, xo):
    # flags 1 / 2: A kept as a sorted array / read from device memory instead of the on-chip bitmap
    g = W.rmat_graph(12, 1503 + 12)
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    want = {p: lexsorted(o.list(p)) for p in WIDTH}
    for tau in (0, 32):
        t = eh.Trie(g["src"], g["dst"], g["n"], tau=tau)
        for p in WIDTH:
            assert np.array_equal(gpu_rows(t, p, eh.exec_opts(**xo)), want[p]), (p, tau, xo)


def test_hub_graph_long_sets(eh):
    # hubs joined to thousands of vertices: many 128-element rounds with ragged tails
    rng = np.random.default_rng(7)
    n = 70000
    e = [(int(h), int(v)) for h in range(6) for v in rng.choice(np.arange(6, n), 3000, replace=False)]
    e += [(int(a), int(b)) for a, b in rng.integers(0, n, size=(40000, 2))]
    e += [(i, j) for i in range(6) for j in range(i + 1, 6)]
    check_small(eh, n, e, taus=(0, 32))


def test_large_value_ranges_stage_sorted_arrays(eh):
    # 300,000 vertices of similar degree (~70): the out-sets of low-ranked vertices span
    # more than 262,144 new ids, beyond the on-chip bitmap, so A is staged as a sorted array
    import synth
    n, m = 300_000, 10_500_000
    src, dst = synth.er(n, m, synth.key(1503, 90))
    o = oracle.Graph(n, src, dst)
    t = eh.Trie(src, dst, n, tau=32)
    assert t.stats()["max_out_degree"] > 32
    for p in WIDTH:
        got = gpu_rows(t, p, eh.exec_opts(light_max=16))
        assert np.array_equal(got, lexsorted(o.list(p))), p


def test_buffer_too_small_and_bad_arguments(eh):
    import torch
    s, d = G.arrays(G.complete(10))
    t = eh.Trie(s, d, 10, tau=32)
    buf = torch.full((119, 3), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(eh.EHError) as ei:
        t.list_into("triangle", buf.data_ptr(), 119)
    assert ei.value.status == 7                                  # EH_ECAPACITY, nothing written
    assert bool((buf == -1).all())
    assert t.list_into("triangle", 0, 0) == 120                  # the size query
    with pytest.raises(eh.EHError) as ei:
        t.list_into("lollipop", buf.data_ptr(), 119)
    assert ei.value.status == 1
    k4 = torch.zeros(211 * 4 + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(eh.EHError) as ei:                        # 4-clique rows need 16-byte alignment
        t.list_into("clique4", k4.data_ptr() + 4, 210)
    assert ei.value.status == 1
    assert t.list_into("clique4", k4.data_ptr(), 210) == 210


# ------------------------------------------------------------ workloads

def test_er_workload_lists_like_oracle(eh):
    g = W.er_10k_100k()
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    rows = gpu_rows(t, "triangle")
    assert len(rows) == GOLD["er_n10000_m100000"]["triangle"]
    assert np.array_equal(rows, lexsorted(o.list("triangle")))


def test_rmat16_triangles_list_like_oracle(eh):
    g = W.rmat_graph(16, 1503 + 16)
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    for tau in (8, 256):
        t = eh.Trie(g["src"], g["dst"], g["n"], tau=tau)
        rows = t.list("triangle").cpu().numpy().view(np.uint32).astype(np.uint64)
        assert len(rows) == GOLD["rmat_s16_ef16"]["triangle"]
        got = np.sort((rows[:, 0] << 32) | (rows[:, 1] << 16) | rows[:, 2])   # ids < 2^16
        want = o.list("triangle").astype(np.uint64)
        assert np.array_equal(got, np.sort((want[:, 0] << 32) | (want[:, 1] << 16) | want[:, 2])), tau


def edge_keys(g):
    """Sorted int64 keys a * 2^32 + b of the simple undirected edges (a < b), from the oracle's canon."""
    import torch
    a, b = oracle.canon(g["src"], g["dst"], g["n"])
    k = torch.from_numpy(a.astype(np.int64) * (1 << 32) + b.astype(np.int64)).cuda()
    return torch.sort(k).values


def assert_rows_are_cliques(rows, keys, chunk=1 << 24):
    """Every pair of ids of every row is an edge of the input (rows ascending within)."""
    import torch
    w = rows.shape[1]
    for c0 in range(0, rows.shape[0], chunk):
        r = rows[c0:c0 + chunk].to(torch.int64)
        assert bool((r[:, 1:] > r[:, :-1]).all())
        for i in range(w):
            for j in range(i + 1, w):
                q = r[:, i] * (1 << 32) + r[:, j]
                pos = torch.searchsorted(keys, q).clamp_(max=keys.numel() - 1)
                assert bool((keys[pos] == q).all())


def assert_unique_triangles(rows, bits):
    """No row repeats (ids < 2^bits, bits <= 22).  The rows are split by the
    high bits of their last id; inside a part, (x, y, low bits of z) packs into
    64 bits, so a sort puts equal rows next to each other."""
    import torch
    low = 64 - 2 * bits
    for part in range(1 << max(0, bits - low)):
        r = rows[(rows[:, 2].to(torch.int64) >> low) == part]
        key = r[:, 0].to(torch.int64) << (bits + low)
        key |= r[:, 1].to(torch.int64) << low
        key |= r[:, 2].to(torch.int64) & ((1 << low) - 1)
        del r
        key = torch.sort(key).values
        assert not bool((key[1:] == key[:-1]).any())
        del key


def test_rmat16_clique4_full_set_by_properties(eh):
    # 290 M rows: the count, every row a 4-clique of the input, no repeats
    import torch
    g = W.rmat_graph(16, 1503 + 16)
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    rows = t.list("clique4")
    assert rows.shape[0] == GOLD["rmat_s16_ef16"]["clique4"]
    assert_rows_are_cliques(rows, edge_keys(g))
    r = rows.to(torch.int64)
    key = ((r[:, 0] * (1 << 16) + r[:, 1]) * (1 << 16) + r[:, 2]) * (1 << 16) + r[:, 3]   # ids < 2^16: 64 bits
    del r
    key = torch.sort(key).values
    assert not bool((key[1:] == key[:-1]).any())


def test_rmat22_triangles_full_size(eh):
    # 2.11 G rows (25 GB) in the benchmark's launch configuration (tau 1024, 8 warps, light 32)
    import torch
    g = W.rmat22()
    gold = GOLD["rmat_s22_ef16"]
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=1024)
    rows = t.list("triangle", xopts=eh.exec_opts(gallop_ratio=32, light_max=32, cta_warps=8))
    assert rows.shape[0] == gold["triangle"]
    assert_rows_are_cliques(rows, edge_keys(g))
    # the rows at sampled vertices, against the oracle's triangles at those vertices
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    for v in list(gold["vertex_triangles"])[:24]:
        v = int(v)
        if gold["vertex_triangles"][str(v)] > 2_000_000:
            continue
        mask = (rows == v).any(dim=1)
        got = lexsorted(rows[mask].cpu().numpy().view(np.uint32))
        assert np.array_equal(got, lexsorted(o.list_triangles_at(v))), v
    assert_unique_triangles(rows, 22)


def test_chunglu_triangles_full_size(eh):
    # 332 M rows (4 GB): the oracle's count, every row a triangle of the input, no repeats
    # (ids < 2^20: a row packs into one 64-bit key), rows at sampled vertices as the oracle's
    import torch
    g = W.chunglu_1m()
    gold = GOLD["chunglu_n1000000_g2.1"]
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    rows = t.list("triangle")
    assert rows.shape[0] == gold["triangle"]
    assert_rows_are_cliques(rows, edge_keys(g))
    r = rows.to(torch.int64)
    key = torch.sort((r[:, 0] << 40) | (r[:, 1] << 20) | r[:, 2]).values
    del r
    assert not bool((key[1:] == key[:-1]).any())
    del key
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    deg = o.degrees()
    for v in [int(x) for x in np.nonzero((deg >= 40) & (deg <= 200))[0][::50000][:8]]:
        got = lexsorted(rows[(rows == v).any(dim=1)].cpu().numpy().view(np.uint32))
        assert np.array_equal(got, lexsorted(o.list_triangles_at(v))), v
