"""Node orderings of the trie build (App. "Node Ordering") against the oracle.

The permutation from original ids to trie ids must equal the oracle's
sequential definition exactly (integers: bit-exact), the trie built under it
must hold the oracle's sets, and every pattern count must stay the oracle's
count (the ordering changes the pruned sets, never the answer).
"""
import numpy as np
import pytest

import oracle
from synth import workloads as W
from tests import graphs as G

pytestmark = pytest.mark.gpu

ORDERINGS = ("degree", "rev_degree", "random", "bfs", "strong_runs", "shingle", "hybrid", "identity")
PATS = ("triangle", "clique4", "lollipop", "lollipop_distinct", "barbell")


@pytest.fixture(scope="module")
def eh():
    import torch
    assert torch.cuda.is_available()
    import paper_1503_02368_gb300 as m
    return m


def check_order(eh, n, s, d, ordering, seed=0, tau=32, patterns=PATS):
    o = oracle.Graph(n, s, d)
    t = eh.Trie(s, d, n, tau=tau, ordering=ordering, order_seed=seed)
    new2old = t.export(0)["new_to_old"]
    assert new2old.tolist() == o.vertex_order(ordering, seed).tolist(), ordering
    for p in patterns:
        assert t.count(p) == o.count(p), (ordering, p)
    return t, o


@pytest.mark.parametrize("ordering", ORDERINGS)
@pytest.mark.parametrize("seed", range(3))
def test_small_graphs(eh, ordering, seed):
    # several components and isolated vertices
    rng = np.random.default_rng(1100 + seed)
    n = int(rng.integers(30, 400))
    e = G.random_graph(n, float(rng.choice([0.01, 0.04, 0.2])), rng)
    s, d = G.arrays(e)
    check_order(eh, n, s, d, ordering, seed=seed)


@pytest.mark.parametrize("ordering", ORDERINGS)
def test_rmat14_orders_and_counts(eh, ordering):
    g = W.rmat_graph(14, 1503 + 14)
    check_order(eh, g["n"], g["src"], g["dst"], ordering, seed=3, patterns=("triangle", "clique4"))


@pytest.mark.parametrize("ordering", ("bfs", "hybrid", "strong_runs"))
def test_trie_sets_under_an_ordering(eh, ordering):
    rng = np.random.default_rng(77)
    n = 600
    s, d = G.arrays(G.random_graph(n, 0.03, rng))
    t, o = check_order(eh, n, s, d, ordering, patterns=("triangle",))
    x = t.export(0)
    new2old = x["new_to_old"]
    old2new = np.empty(n, np.int64)
    old2new[new2old] = np.arange(n)
    for v in range(n):
        N = np.sort(old2new[o.neighbours(int(new2old[v]))])
        P = N[N < v].astype(np.uint32)
        b, ln = int(x["off"][v]), int(x["len"][v])
        assert ln == len(P) and np.array_equal(x["nbr"][b:b + ln], P)


def test_chunglu_bfs_many_levels(eh):
    import synth
    n = 200_000
    s, d = synth.chunglu(n, 600_000, synth.key(1503, 91), gamma=2.5)
    for ordering in ("bfs", "hybrid", "shingle"):
        check_order(eh, n, s, d, ordering, seed=1, patterns=("triangle",))


def test_unknown_ordering_rejected(eh):
    with pytest.raises(eh.EHError) as ei:
        eh.Trie(np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), 3, ordering=8)
    assert ei.value.status == 1


# ------------------------------------------------------------ selection queries (Sec. 5.3)

@pytest.mark.parametrize("seed", range(4))
def test_selection_queries_random_graphs(eh, seed):
    rng = np.random.default_rng(1300 + seed)
    n = int(rng.integers(40, 300))
    s, d = G.arrays(G.random_graph(n, float(rng.choice([0.05, 0.2, 0.4])), rng))
    o = oracle.Graph(n, s, d)
    for tau in (0, 32):
        t = eh.Trie(s, d, n, tau=tau)
        for node in rng.choice(n, 6, replace=False):
            node = int(node)
            for p in ("clique4", "barbell"):
                assert t.count_selected(p, node) == o.count_selected(p, node), (p, node, tau)


def test_selection_queries_rmat_hubs_and_knobs(eh):
    # the top hubs as selected vertices: neighbours with hundreds of neighbours (CTA path)
    g = W.rmat_graph(12, 1503 + 12)
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    deg = o.degrees()
    rank = np.argsort(-deg.astype(np.int64))
    nodes = [int(rank[0]), int(rank[1]), int(rank[50]), int(np.argmax(deg == 5))]
    want = {v: (o.count_selected("clique4", v), o.count_selected("barbell", v)) for v in nodes}
    for tau in (0, 32):
        t = eh.Trie(g["src"], g["dst"], g["n"], tau=tau)
        for node in nodes:
            assert t.count_selected("clique4", node) == want[node][0], (node, tau)
            assert t.count_selected("clique4", node, xopts=eh.exec_opts(light_max=8, flags=1)) == want[node][0]
            assert t.count_selected("barbell", node) == want[node][1], node


def test_selection_closed_forms_and_errors(eh):
    n = 40
    s, d = G.arrays(G.complete(n))
    t = eh.Trie(s, d, n, tau=32)
    assert t.count_selected("clique4", 7) == (n - 1) ** 2 * (n - 2) * (n - 3)
    assert t.count_selected("barbell", 7) == (n - 1) ** 4 * (n - 2) ** 2
    with pytest.raises(eh.EHError) as ei:
        t.count_selected("clique4", n)
    assert ei.value.status == 1
