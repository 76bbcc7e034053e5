"""The serving loop: admission, continuous batching, results equal alone and in the mix."""
import random
import threading
import time

import numpy as np
import pytest

import oracle
import synth
from synth import workloads as W

pytestmark = pytest.mark.gpu
PATS = ("triangle", "clique4", "lollipop", "lollipop_distinct")


@pytest.fixture(scope="module")
def eh():
    import torch
    assert torch.cuda.is_available()
    import paper_1503_02368_gb300 as m
    return m


@pytest.fixture(scope="module")
def setup(eh):
    g = W.rmat_graph(14, 1503 + 41)
    off, pool = synth.ego_subsets(g["n"], g["src"], g["dst"], synth.key(1503, 41), 160, 1, 10, 20000)
    trie = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    return g, off, pool, trie


def test_results_same_alone_and_in_the_mix(eh, setup):
    g, off, pool, trie = setup
    nq = len(off) - 1
    pats = [PATS[q % 4] for q in range(nq)]
    subsets = [pool[off[q]:off[q + 1]] for q in range(nq)]
    alone = [trie.count(pats[q], subset=subsets[q]) for q in range(nq)]
    srv = eh.Server(trie, memory_budget_bytes=8 << 30, max_batch=16, max_inflight=3)
    tickets = [None] * nq
    order = list(range(nq))
    random.Random(3).shuffle(order)

    def client(idx):
        rnd = random.Random(idx)
        for q in order[idx::4]:
            while True:
                t = srv.submit(pats[q], subsets[q])
                if t is not None:
                    break
                time.sleep(0.001)
            tickets[q] = t
            time.sleep(rnd.random() * 0.002)

    th = [threading.Thread(target=client, args=(i,)) for i in range(4)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    got = [srv.wait(tickets[q], timeout_ms=120000) for q in range(nq)]
    assert all(st == 0 for _, st in got)
    assert [c for c, _ in got] == alone
    st = srv.stats()
    assert st["completed"] == nq and st["submitted"] == nq and st["bytes_in_use"] == 0
    assert st["batches"] < nq and st["mean_batch"] > 1.0          # queries were batched
    assert all(srv.latency(t) >= 0 for t in tickets)
    srv.close()
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    for q in range(0, nq, 16):
        assert alone[q] == o.induced(subsets[q]).count(pats[q])


def test_admission_rejects_what_does_not_fit(eh, setup):
    g, off, pool, trie = setup
    srv = eh.Server(trie, memory_budget_bytes=1 << 16, max_batch=4, max_inflight=1)
    assert srv.submit("triangle", pool[off[0]:off[1]]) is None       # EH_EBUSY
    assert srv.stats()["rejected"] == 1
    srv.close()
    srv = eh.Server(trie, memory_budget_bytes=1 << 34, max_batch=4, max_inflight=2)
    t = srv.submit("triangle", pool[off[0]:off[1]])
    c, s = srv.wait(t, timeout_ms=60000)
    assert s == 0 and c == trie.count("triangle", subset=pool[off[0]:off[1]])
    with pytest.raises(eh.EHError):
        srv.wait(t + 1000)                                            # unknown ticket
    srv.close()


def test_invalid_query_fails_alone(eh, setup):
    g, off, pool, trie = setup
    srv = eh.Server(trie, memory_budget_bytes=1 << 34, max_batch=8, max_inflight=1)
    good = srv.submit("triangle", pool[off[1]:off[2]])
    bad = srv.submit("triangle", np.array([1, g["n"] + 3], np.uint32))
    cg, sg = srv.wait(good, timeout_ms=60000)
    cb, sb = srv.wait(bad, timeout_ms=60000)
    assert sg == 0 and cg == trie.count("triangle", subset=pool[off[1]:off[2]])
    assert sb == 1
    srv.close()
