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


def test_rmat24_serving_workload_matches_oracle(eh):
    # the serving configuration itself: R-MAT scale 24 resident, ego nets with
    # induced edges log-uniform in [100, 1e6], patterns triangle / 4-clique /
    # lollipop; the oracle's counts of a sample of 24 queries (8 per pattern)
    import json
    import os
    from tests.golden.make_golden import fingerprint
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workload_counts.json")))
    gold = gold["rmat_s24_serve"]
    g = W.rmat24_serve(n_queries=gold["n_queries"])
    assert fingerprint(g) == gold["fingerprint"]
    names = ("triangle", "clique4", "lollipop")
    off, pool = g["offsets"], g["pool"]
    trie = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    srv = eh.Server(trie, memory_budget_bytes=48 << 30, max_batch=32, max_inflight=3)
    tickets = {}
    for q in range(gold["n_queries"]):               # every query of the sample run, in the mix
        while True:
            t = srv.submit(names[g["patterns"][q]], pool[off[q]:off[q + 1]])
            if t is not None:
                break
            time.sleep(0.001)
        tickets[q] = t
    for q, rec in gold["queries"].items():
        c, st = srv.wait(tickets[int(q)], timeout_ms=600000)
        assert st == 0 and rec["pattern"] == names[g["patterns"][int(q)]]
        assert c == rec["count"], (q, rec)
    for q in list(gold["queries"])[:6]:               # and alone
        assert trie.count(gold["queries"][q]["pattern"], subset=pool[off[int(q)]:off[int(q) + 1]]) == \
            gold["queries"][q]["count"]
    srv.close()
