"""The composite (block-level) layout of Sec. 4.3 on the device.

The directory of every pruned set must describe exactly the set's values,
each block in the kind the layout rule gives it (checked against the
oracle's rule), and the triangle count over the directories must equal the
oracle's count at every threshold.  Other patterns of a block-layout trie
use the uint arrays and must stay exact too.
"""
import numpy as np
import pytest

import oracle
from synth import workloads as W
from tests import graphs as G

pytestmark = pytest.mark.gpu

TAUS = (0, 1, 8, 32, 256, 0xFFFFFFFF)


@pytest.fixture(scope="module")
def eh():
    import torch
    assert torch.cuda.is_available()
    import paper_1503_02368_gb300 as m
    return m


def check_directories(t, tau):
    x = t.export(0)
    off, d, w = t.export_blocks()
    for v in range(t.n):
        b, ln = int(x["off"][v]), int(x["len"][v])
        S = x["nbr"][b:b + ln]
        ids, kinds = oracle.block_layout(S, tau)
        ent = d[int(off[v]):int(off[v + 1])]
        assert ent[:, 0].tolist() == ids.tolist(), v
        vals = []
        for (bid, info), k in zip(ent.tolist(), kinds.tolist()):
            if info & 0x80000000:
                assert k, (v, bid)
                bits = np.unpackbits(w[info & 0x7FFFFFFF].view(np.uint8), bitorder="little")
                vals += (np.nonzero(bits)[0] + 256 * bid).tolist()
            else:
                assert not k, (v, bid)
                st, n = info & 0x7FFFFF, ((info >> 23) & 255) + 1
                assert all(int(y) // 256 == bid for y in S[st:st + n])
                vals += S[st:st + n].tolist()
        assert vals == S.tolist(), v


@pytest.mark.parametrize("seed", range(4))
def test_random_graphs_directories_and_triangles(eh, seed):
    rng = np.random.default_rng(1400 + seed)
    n = int(rng.integers(100, 1500))
    s, d = G.arrays(G.random_graph(n, float(rng.choice([0.01, 0.05, 0.3])), rng))
    o = oracle.Graph(n, s, d)
    want = o.triangles()
    for tau in TAUS:
        t = eh.Trie(s, d, n, tau=tau, block_layout=True)
        check_directories(t, tau)
        assert t.count("triangle") == want, tau


def test_rmat_block_layout_all_patterns(eh):
    g = W.rmat_graph(13, 1503 + 13)
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    for tau in (8, 256):
        t = eh.Trie(g["src"], g["dst"], g["n"], tau=tau, block_layout=True)
        assert t.stats()["n_bitset_sets"] == 0            # no set-level bitsets in this layout
        for p in ("triangle", "clique4", "lollipop", "barbell"):
            assert t.count(p) == o.count(p, nthreads=8), (p, tau)


@pytest.mark.parametrize("ordering", ("random", "rev_degree"))
def test_block_layout_under_other_orderings(eh, ordering):
    g = W.rmat_graph(12, 1503 + 12)
    want = oracle.Graph(g["n"], g["src"], g["dst"]).triangles()
    t = eh.Trie(g["src"], g["dst"], g["n"], tau=32, block_layout=True, ordering=ordering, order_seed=2)
    assert t.count("triangle") == want


@pytest.mark.parametrize("ordering", ("random", "degree"))
def test_block_layout_long_directories(eh, ordering):
    # Chung-Lu hubs over 1,024 block ids.  Under a random order some pruned sets
    # touch more than 512 blocks (more than a warp stages in shared memory), and
    # light u's meet hub v's whose directories are over 8x longer than theirs
    # and over 256 entries (searched rather than walked).
    import synth
    n = 1 << 18
    s, d = synth.chunglu(n, 1_500_000, synth.key(1503, 95), gamma=2.1)
    want = oracle.Graph(n, s, d).triangles()
    for tau in (1, 256):
        t = eh.Trie(s, d, n, tau=tau, ordering=ordering, order_seed=3, block_layout=True)
        assert t.count("triangle") == want, tau
    x = t.export(0)
    off, _, _ = t.export_blocks()
    na = np.diff(off.astype(np.int64))
    u = np.repeat(np.arange(n), x["len"].astype(np.int64))
    v = np.concatenate([x["nbr"][int(b):int(b) + int(ln)] for b, ln in zip(x["off"], x["len"])]).astype(np.int64)
    skew = int(((na[v] > 8 * na[u]) & (na[v] > 256)).sum())
    if ordering == "random":
        assert na.max() > 512 and skew > 0, (na.max(), skew)


def test_export_blocks_needs_the_layout(eh):
    s, d = G.arrays(G.complete(5))
    t = eh.Trie(s, d, 5, tau=32)
    with pytest.raises(eh.EHError) as ei:
        t.export_blocks()
    assert ei.value.status == 1
