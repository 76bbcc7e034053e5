"""Pins of the CPU oracle against facts that do not come from the oracle.

Each check is chosen so that a plausible slip in the oracle (a dropped set in
an intersection, a wrong orientation test, a missing factor, a transposed
operand) breaks at least one of them: brute force on dense matrices,
textbook closed forms, the symmetric-data multiples of App. A.1.2, the AGM
bound of Sec. 2.1, and invariance under relabelling.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests import graphs as G


def og(n, edges):
    s, d = G.arrays(edges)
    return oracle.Graph(n, s, d)


# ------------------------------------------------------------ triangles

@pytest.mark.parametrize("seed", range(12))
def test_triangles_vs_trace_a3(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 64))
    p = float(rng.choice([0.05, 0.2, 0.5, 0.9]))
    e = G.random_graph(n, p, rng)
    A = G.adjacency(n, e)
    g = og(n, e)
    assert g.triangles() == G.bf_triangles(A)
    assert g.triangles(nthreads=4) == G.bf_triangles(A)


@pytest.mark.parametrize("n", range(1, 14))
def test_triangles_complete(n):
    assert og(n, G.complete(n)).triangles() == math.comb(n, 3)


def test_triangles_zero_families():
    rng = np.random.default_rng(7)
    n, e = G.complete_multipartite(5, 7)                      # bipartite K_{5,7}
    assert og(n, e).triangles() == 0
    assert og(20, G.star(20)).triangles() == 0
    assert og(40, G.random_tree(40, rng)).triangles() == 0
    for k in (4, 6, 10, 5, 7):                                # even and odd cycles > 3
        assert og(k, G.cycle(k)).triangles() == 0
    assert og(10, G.petersen()).triangles() == 0
    assert og(3, G.cycle(3)).triangles() == 1


@pytest.mark.parametrize("n", [4, 5, 8, 13])
def test_triangles_wheel(n):
    assert og(n + 1, G.wheel(n)).triangles() == n


@pytest.mark.parametrize("parts", [(1, 1, 1), (2, 2, 2), (2, 3, 4), (5, 1, 3)])
def test_triangles_tripartite(parts):
    n, e = G.complete_multipartite(*parts)
    assert og(n, e).triangles() == parts[0] * parts[1] * parts[2]


@pytest.mark.parametrize("seed", range(6))
def test_symmetric_multiple_and_agm(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(10, 60))
    e = G.random_graph(n, 0.3, rng)
    g = og(n, e)
    t = g.triangles()
    assert g.triangles(pruned=False) == 6 * t            # App. A.1.2: symmetric data gives a multiple
    assert g.clique4(pruned=False) == 24 * g.clique4()
    assert t <= g.m ** 1.5                               # Sec. 2.1: |out| <= N^{3/2}


def test_agm_tight_on_complete():
    # Sec. 2.1 example: K_sqrt(N) has Theta(N^{3/2}) triangles
    for k in (10, 20, 40):
        g = og(k, G.complete(k))
        assert g.triangles() == math.comb(k, 3)
        assert g.triangles() >= 0.1 * g.m ** 1.5


# ------------------------------------------------------------ 4-cliques

@pytest.mark.parametrize("seed", range(8))
def test_clique4_vs_subset_enumeration(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(6, 30))
    e = G.random_graph(n, float(rng.choice([0.3, 0.6, 0.85])), rng)
    A = G.adjacency(n, e)
    g = og(n, e)
    assert g.clique4() == G.bf_clique4(A)
    assert g.clique4(nthreads=3) == G.bf_clique4(A)


@pytest.mark.parametrize("n", range(1, 12))
def test_clique4_complete(n):
    assert og(n, G.complete(n)).clique4() == math.comb(n, 4)


@pytest.mark.parametrize("parts", [(2, 2, 2, 2), (1, 2, 3, 4), (3, 3, 1, 2)])
def test_clique4_multipartite(parts):
    n, e = G.complete_multipartite(*parts)
    assert og(n, e).clique4() == int(np.prod(parts))


def test_clique4_zero():
    n, e = G.complete_multipartite(2, 2, 2)   # octahedron: triangles, no K4
    g = og(n, e)
    assert g.triangles() == 8 and g.clique4() == 0
    assert og(10, G.petersen()).clique4() == 0


# ------------------------------------------------------------ lollipop

@pytest.mark.parametrize("seed", range(6))
def test_lollipop_vs_literal_join(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(4, 16))
    e = G.random_graph(n, 0.5, rng)
    A = G.adjacency(n, e)
    g = og(n, e)
    assert g.lollipop() == G.bf_lollipop(A)
    # closed form through per-vertex triangle counts: sum_x 2 t(x) d(x)
    t = G.bf_vertex_triangles(A)
    assert g.lollipop() == int((2 * t * A.sum(1)).sum())
    assert g.lollipop_distinct() == G.bf_lollipop_distinct(A)
    assert g.lollipop_distinct() == int((t * (A.sum(1) - 2)).sum())


@pytest.mark.parametrize("n", range(3, 10))
def test_lollipop_complete(n):
    g = og(n, G.complete(n))
    assert g.lollipop() == n * (n - 1) * (n - 2) * (n - 1)
    assert g.lollipop_distinct() == n * math.comb(n - 1, 2) * (n - 3)


def test_vertex_triangles():
    rng = np.random.default_rng(5)
    n = 40
    e = G.random_graph(n, 0.4, rng)
    A = G.adjacency(n, e)
    g = og(n, e)
    verts = np.arange(n, dtype=np.uint32)
    assert np.array_equal(g.vertex_triangles(verts), G.bf_vertex_triangles(A).astype(np.uint64))


# ------------------------------------------------------------ induced subgraphs

def test_induced_subgraph():
    rng = np.random.default_rng(11)
    n = 50
    e = G.random_graph(n, 0.3, rng)
    A = G.adjacency(n, e)
    g = og(n, e)
    full = g.induced(np.arange(n, dtype=np.uint32))
    assert full.triangles() == g.triangles() and full.clique4() == g.clique4()
    for trial in range(5):
        S = rng.choice(n, size=int(rng.integers(3, n)), replace=False)
        sub = g.induced(np.concatenate([S, S[:3]]).astype(np.uint32))   # repeats are harmless
        As = A[np.ix_(np.sort(S), np.sort(S))]
        assert sub.triangles() == G.bf_triangles(As)
        assert sub.clique4() == G.bf_clique4(As)
        assert sub.lollipop() == G.bf_lollipop(As)
    # a planted clique's vertex set
    kk = n - 40
    e2 = e + [(40 + i, 40 + j) for i in range(kk) for j in range(i + 1, kk)]
    g2 = og(n, e2)
    sub = g2.induced(np.arange(40, n, dtype=np.uint32))
    assert sub.triangles() == math.comb(kk, 3) and sub.clique4() == math.comb(kk, 4)


def test_induced_rejects_bad_id():
    g = og(5, G.complete(5))
    with pytest.raises(ValueError):
        g.induced(np.array([1, 7], np.uint32))


# ------------------------------------------------------------ invariances

@pytest.mark.parametrize("seed", range(4))
def test_relabel_invariance(seed):
    rng = np.random.default_rng(400 + seed)
    n = 45
    e = G.random_graph(n, 0.35, rng)
    perm = rng.permutation(n)
    e2 = [(int(perm[a]), int(perm[b])) for a, b in e]
    g1, g2 = og(n, e), og(n, e2)
    for pat in ("triangle", "clique4", "lollipop", "lollipop_distinct"):
        assert g1.count(pat) == g2.count(pat)


def test_direction_loops_duplicates_ignored():
    e = G.complete(6)
    noisy = e + [(b, a) for a, b in e] + [(v, v) for v in range(6)] + e[:4]
    assert og(6, noisy).triangles() == 20 and og(6, noisy).m == 15


# ------------------------------------------------------------ canonical relation, order, layout

def test_canon_matches_set_semantics():
    rng = np.random.default_rng(9)
    n = 300
    s = rng.integers(0, n, 5000).astype(np.uint32)
    d = rng.integers(0, n, 5000).astype(np.uint32)
    a, b = oracle.canon(s, d, n)
    ref = sorted({(min(x, y), max(x, y)) for x, y in zip(s.tolist(), d.tolist()) if x != y})
    assert list(zip(a.tolist(), b.tolist())) == ref
    with pytest.raises(ValueError):
        oracle.canon(np.array([0, 300], np.uint32), np.array([1, 2], np.uint32), n)


def test_degree_order():
    rng = np.random.default_rng(3)
    n = 80
    e = G.random_graph(n, 0.1, rng)
    A = G.adjacency(n, e)
    deg = A.sum(1)
    want = sorted(range(n), key=lambda v: (-deg[v], v))
    assert og(n, e).degree_order().tolist() == want


def test_layout_rule():
    # Sec. 4.4: bitset when range <= tau * |S|
    assert oracle.layout_is_bitset(np.arange(100, 356), 1)          # range 256, |S| 256
    assert not oracle.layout_is_bitset(np.array([0, 1000]), 256)     # range 1001 > 512
    assert oracle.layout_is_bitset(np.array([0, 511]), 256)          # range 512 <= 512
    assert not oracle.layout_is_bitset(np.array([0, 512]), 256)      # range 513 > 512
    assert not oracle.layout_is_bitset(np.arange(10), 0)             # tau 0: all uint
    assert oracle.layout_is_bitset(np.array([0, 4_000_000_000]), 0xFFFFFFFF)
    assert not oracle.layout_is_bitset(np.array([], np.uint32), 0xFFFFFFFF)


def test_empty_graph():
    g = og(5, [])
    assert g.m == 0 and g.triangles() == 0 and g.clique4() == 0 and g.lollipop() == 0
    g0 = oracle.Graph(0, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert g0.triangles() == 0


def test_outer_sample_sums_to_whole():
    rng = np.random.default_rng(21)
    n = 60
    e = G.random_graph(n, 0.3, rng)
    g = og(n, e)
    verts = np.arange(n, dtype=np.uint32)
    half = verts[::2], verts[1::2]
    c0, e0 = g.triangles_outer(half[0], nthreads=2)
    c1, e1 = g.triangles_outer(half[1])
    assert c0 + c1 == g.triangles() == G.bf_triangles(G.adjacency(n, e))
    assert e0 + e1 == g.m


# ------------------------------------------------------------ barbell

@pytest.mark.parametrize("seed", range(6))
def test_barbell_vs_literal_join_and_matrix_form(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(4, 14))
    e = G.random_graph(n, 0.5, rng)
    A = G.adjacency(n, e)
    g = og(n, e)
    want = G.bf_barbell(A)
    assert g.barbell() == want
    d3 = np.diag(A @ A @ A)                     # ordered (y, z) pairs closing a triangle at x
    assert want == int((A * np.outer(d3, d3)).sum())


def test_barbell_closed_forms():
    # two triangles joined by one edge: 2 ordered edge directions x (2*1)*(2*1) at the bridge ends
    e = [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5), (0, 3)]
    g = og(6, e)
    # t = 1 on every vertex; B = sum over ordered edges of 4 t(x) t(x') = 4 * 14
    assert g.barbell() == 4 * 14
    # K_n: every ordered edge (n(n-1)) times (2 C(n-1,2))^2
    for n in (3, 4, 6):
        assert og(n, G.complete(n)).barbell() == n * (n - 1) * (2 * math.comb(n - 1, 2)) ** 2
    assert og(10, G.petersen()).barbell() == 0


# ------------------------------------------------------------ listing

def _rows(t):
    return [tuple(int(v) for v in r) for r in t]


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("pattern,k", [("triangle", 3), ("clique4", 4)])
def test_listing_vs_subset_enumeration(seed, pattern, k):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(5, 22))
    e = G.random_graph(n, float(rng.choice([0.2, 0.5, 0.8])), rng)
    A = G.adjacency(n, e)
    g = og(n, e)
    rows = g.list(pattern)
    assert rows.shape == (g.count(pattern), k)
    assert all(list(r) == sorted(r) and len(set(r)) == k for r in _rows(rows))   # ascending ids
    assert sorted(_rows(rows)) == G.bf_list(A, k)                                # same set, no repeats


def test_listing_closed_forms():
    for n in (3, 5, 8):
        g = og(n, G.complete(n))
        assert sorted(_rows(g.list("triangle"))) == list(itertools.combinations(range(n), 3))
        assert sorted(_rows(g.list("clique4"))) == list(itertools.combinations(range(n), 4))
    assert og(10, G.petersen()).list("triangle").shape == (0, 3)
    assert og(9, G.cycle(9)).list("clique4").shape == (0, 4)
    # wheel W_n (n >= 4): the n triangles through the hub, no 4-clique
    rows = sorted(_rows(og(8, G.wheel(7)).list("triangle")))
    assert rows == sorted(tuple(sorted((0, i, i % 7 + 1))) for i in range(1, 8))


def test_listing_loop_order_and_capacity():
    import ctypes
    g = og(6, G.complete(6))
    rows = g.list("triangle")
    # loop order of the nest: largest id (x) slowest, then y, then z
    keys = [(r[2], r[1], r[0]) for r in _rows(rows)]
    assert keys == sorted(keys)
    # a buffer smaller than the result: the full size is returned, only `cap` rows written
    buf = np.full((4, 3), 7, np.uint32)
    k = oracle.lib().oracle_list_triangles(g._h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), 2)
    assert k == 20
    assert _rows(buf[:2]) == _rows(rows[:2]) and (buf[2:] == 7).all()


@pytest.mark.parametrize("seed", range(4))
def test_listing_at_vertex(seed):
    rng = np.random.default_rng(800 + seed)
    n = int(rng.integers(6, 24))
    e = G.random_graph(n, 0.5, rng)
    A = G.adjacency(n, e)
    g = og(n, e)
    bf = G.bf_list(A, 3)
    t = G.bf_vertex_triangles(A)
    for x in range(n):
        rows = g.list_triangles_at(x)
        assert len(rows) == t[x]
        assert sorted(_rows(rows)) == [q for q in bf if x in q]


# ------------------------------------------------------------ node orderings

# Two hubs (0 and 4) joined by the path 0-3-7-8-4; hub 0 has leaves 5, 6 and
# hub 4 has leaves 1, 2.  The orders below were worked out by hand from the
# definitions (App. "Node Ordering"; BFS from the highest-degree vertex,
# neighbours in ascending id; hybrid = BFS re-sorted stably by degree).
HUBS = [(0, 5), (0, 6), (0, 3), (3, 7), (7, 8), (8, 4), (4, 1), (4, 2)]
HUBS_ORDERS = {
    "degree": [0, 4, 3, 7, 8, 1, 2, 5, 6],
    "rev_degree": [1, 2, 5, 6, 3, 7, 8, 0, 4],
    "bfs": [0, 3, 5, 6, 7, 8, 4, 1, 2],
    "strong_runs": [0, 3, 5, 6, 4, 1, 2, 8, 7],
    "hybrid": [0, 4, 3, 7, 8, 5, 6, 1, 2],
    "identity": list(range(9)),
}


@pytest.mark.parametrize("ordering", sorted(HUBS_ORDERS))
def test_orderings_by_hand(ordering):
    assert og(9, HUBS).vertex_order(ordering).tolist() == HUBS_ORDERS[ordering]


def test_bfs_orders_unreached_vertices_by_degree():
    # component {0..5} searched from 3 (the only degree-3 vertex); 6-7 and the
    # isolated 8 are not reached and follow in degree order
    e = [(0, 1), (0, 2), (1, 3), (2, 3), (3, 4), (4, 5), (6, 7)]
    g = og(9, e)
    assert g.vertex_order("bfs").tolist() == [3, 1, 2, 4, 0, 5, 6, 7, 8]
    assert g.vertex_order("strong_runs").tolist() == [3, 1, 2, 4, 0, 5, 6, 7, 8]
    assert g.vertex_order("rev_degree").tolist() == [8, 5, 6, 7, 0, 1, 2, 4, 3]


@pytest.mark.parametrize("seed", range(4))
def test_orderings_are_permutations_and_seeded(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(20, 200))
    g = og(n, G.random_graph(n, 0.05, rng))
    for o in g.ORDERINGS:
        assert sorted(g.vertex_order(o, seed).tolist()) == list(range(n)), o
    assert g.vertex_order("random", 1).tolist() != g.vertex_order("random", 2).tolist()
    assert g.vertex_order("random", 5).tolist() == g.vertex_order("random", 5).tolist()


def test_shingle_puts_twins_together():
    # vertices with equal neighbourhoods share their min-hash shingle, so they
    # are consecutive (ties by id)
    e = [(0, 10), (0, 11), (1, 10), (1, 11), (2, 10), (2, 11),     # 0, 1, 2 twins
         (3, 12), (4, 12), (5, 12), (6, 13), (7, 14), (8, 15)]     # 3, 4, 5 twins
    for seed in range(5):
        o = og(16, e).vertex_order("shingle", seed).tolist()
        i = o.index(0)
        assert o[i:i + 3] == [0, 1, 2]
        j = o.index(3)
        assert o[j:j + 3] == [3, 4, 5]
        assert o.index(9) == 15                     # no neighbours: last (of the ties at all ones, largest id)



# ------------------------------------------------------------ selections

@pytest.mark.parametrize("seed", range(5))
def test_selection_queries_vs_tuple_enumeration(seed):
    rng = np.random.default_rng(1200 + seed)
    n = int(rng.integers(5, 11))
    e = G.random_graph(n, 0.6, rng)
    A = G.adjacency(n, e)
    g = og(n, e)
    for node in range(n):
        assert g.count_selected("clique4", node) == G.bf_sk4(A, node)
        assert g.count_selected("barbell", node) == G.bf_sbarbell(A, node)
        d3 = np.diag(A @ A @ A)                      # 2 t(x)
        assert g.count_selected("barbell", node) == int(A[node] @ d3) ** 2


def test_selection_closed_forms():
    for n in (4, 5, 7):
        g = og(n, G.complete(n))
        for node in (0, n - 1):
            assert g.count_selected("clique4", node) == (n - 1) ** 2 * (n - 2) * (n - 3)
            assert g.count_selected("barbell", node) == (n - 1) ** 4 * (n - 2) ** 2
    g = og(10, G.petersen())                         # triangle-free
    assert g.count_selected("clique4", 0) == 0 and g.count_selected("barbell", 0) == 0
    g = og(6, [(0, 1), (1, 2), (0, 2), (3, 4)])      # node 5 isolated, node 3 next to no triangle
    assert g.count_selected("barbell", 5) == 0 and g.count_selected("barbell", 3) == 0
    assert g.count_selected("barbell", 0) == (2 + 2) ** 2



# ------------------------------------------------------------ composite layout

def test_block_layout_rule():
    # block 0 holds 1 value, block 1 holds 2, block 3 all 256
    S = np.array([1, 300, 301] + list(range(768, 1024)), np.uint32)
    ids, kind = oracle.block_layout(S, 32)
    assert ids.tolist() == [0, 1, 3] and kind.tolist() == [False, False, True]
    ids, kind = oracle.block_layout(S, 128)              # 2 * 128 >= 256 in block 1
    assert kind.tolist() == [False, True, True]
    assert oracle.block_layout(S, 256)[1].tolist() == [True, True, True]
    assert oracle.block_layout(S, 0)[1].tolist() == [False, False, False]
    assert oracle.block_layout(S, 0xFFFFFFFF)[1].tolist() == [True, True, True]
    assert oracle.block_layout(S, 1)[1].tolist() == [False, False, True]   # only a full block at tau 1
    assert oracle.block_layout(np.zeros(0, np.uint32), 32)[0].tolist() == []


def test_block_layout_vs_per_block_set_rule():
    # each block's kind is the set-level rule applied to the block's values with range 256
    rng = np.random.default_rng(5)
    for _ in range(20):
        S = np.unique(rng.integers(0, 5000, size=int(rng.integers(1, 600)))).astype(np.uint32)
        tau = int(rng.choice([1, 8, 32, 100, 256]))
        ids, kind = oracle.block_layout(S, tau)
        assert ids.tolist() == sorted(set((S // 256).tolist()))
        for b, k in zip(ids, kind):
            c = int(((S // 256) == b).sum())
            assert k == (256 <= tau * c)
