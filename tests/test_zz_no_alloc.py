"""eh_count_noalloc: whole-graph counts that allocate no device memory.

Some callers cannot allocate device memory while they count: a process that
has handed its device memory to a fixed pool or budget, or code where an
allocation could block or fail at the wrong moment.  eh_count_noalloc serves
them by keeping the count kernels' scratch in a static device array.  These
checks call it through the C ABI and compare it with eh_count, twice in a row
(the array keeps the previous call's contents).  The file sorts last so that
a run stopping at its first failure has run every other test already.
"""
import ctypes
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from synth import workloads as W

pytestmark = pytest.mark.gpu
PATS = ("triangle", "clique4", "lollipop", "lollipop_distinct")


@pytest.fixture(scope="module")
def eh():
    import torch
    assert torch.cuda.is_available()
    import paper_1503_02368_gb300 as m
    return m


def noalloc(eh, trie, pattern):
    """One eh_count_noalloc call with the library's allocation-failure hook
    armed (any device allocation the call made would fail it) and the
    device's free memory compared before and after."""
    import torch
    L = eh.lib()
    out = ctypes.c_uint64(0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    L.eh_test_fail_alloc_after(0)
    try:
        r = L.eh_count_noalloc(trie.handle, eh.PATTERNS[pattern], None, ctypes.byref(out))
    finally:
        L.eh_test_fail_alloc_after(-1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    if r != 0:
        raise eh.EHError(r, L.eh_last_error().decode())
    return int(out.value)


def clique_edges(k, extra=0, n=None, seed=0):
    i, j = np.triu_indices(k, 1)
    s, d = i.astype(np.uint32), j.astype(np.uint32)
    if extra:
        rng = np.random.default_rng(seed)
        e = rng.integers(0, n, size=(extra, 2)).astype(np.uint32)
        s, d = np.concatenate([s, e[:, 0]]), np.concatenate([d, e[:, 1]])
    return s, d


def test_matches_eh_count_on_two_calls(eh):
    g = W.rmat_graph(14, 1503 + 14)
    trie = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
    for p in PATS:
        want = trie.count(p)              # also builds the work plan
        assert noalloc(eh, trie, p) == want
        assert noalloc(eh, trie, p) == want


def test_clique4_through_the_static_spill_arena(eh):
    # a 1,100-clique: out-degrees up to 1,099 exceed the per-warp shared buffer
    n = 3000
    s, d = clique_edges(1100, extra=20000, n=n, seed=1)
    trie = eh.Trie(s, d, n, tau=32)
    assert trie.stats()["max_out_degree"] > 1024
    want = trie.count("clique4")
    assert want >= math.comb(1100, 4)
    assert noalloc(eh, trie, "clique4") == want
    assert noalloc(eh, trie, "clique4") == want
    assert noalloc(eh, trie, "triangle") == trie.count("triangle")


def test_rejects_what_it_cannot_hold(eh):
    g = W.er_10k_100k()
    fresh = eh.Trie(g["src"], g["dst"], g["n"])
    with pytest.raises(eh.EHError) as ei:                 # no work plan yet
        noalloc(eh, fresh, "triangle")
    assert ei.value.status == 1
    fresh.info("triangle")
    assert noalloc(eh, fresh, "triangle") == fresh.count("triangle")
    s, d = clique_edges(6000)                             # needs far more arena than the array holds
    big = eh.Trie(s, d, 6000, tau=32)
    big.info("clique4")
    with pytest.raises(eh.EHError) as ei:
        noalloc(eh, big, "clique4")
    assert ei.value.status == 1 and "arena" in str(ei.value)


def test_matches_the_oracle_directly(eh):
    import oracle
    g = W.rmat_graph(13, 1503 + 13)
    o = oracle.Graph(g["n"], g["src"], g["dst"])
    trie = eh.Trie(g["src"], g["dst"], g["n"], tau=256)
    trie.info("triangle")
    for p in PATS:
        want = o.count(p, nthreads=4)
        assert noalloc(eh, trie, p) == want
        assert noalloc(eh, trie, p) == want


def test_block_layout_trie_and_barbell_rejection(eh):
    g = W.rmat_graph(13, 1503 + 13)
    blk = eh.Trie(g["src"], g["dst"], g["n"], tau=256, block_layout=True)
    want = blk.count("triangle")                          # the block-layout kernel; also builds the plan
    assert noalloc(eh, blk, "triangle") == want            # the set-level kernel, same count
    assert noalloc(eh, blk, "clique4") == blk.count("clique4")
    with pytest.raises(eh.EHError) as ei:
        noalloc(eh, blk, "barbell")
    assert ei.value.status == 1


_FRESH = r"""
import ctypes, sys
sys.path.insert(0, sys.argv[1])
import torch
import paper_1503_02368_gb300 as eh
from synth import workloads as W
torch.cuda.init()
g = W.rmat_graph(12, 1503 + 12)
t = eh.Trie(g["src"], g["dst"], g["n"], tau=32)
t.info("triangle")
L = eh.lib()
res = []
for p in ("triangle", "clique4", "lollipop"):
    torch.cuda.synchronize()
    f0 = torch.cuda.mem_get_info()[0]
    out = ctypes.c_uint64(0)
    L.eh_test_fail_alloc_after(0)
    r = L.eh_count_noalloc(t.handle, eh.PATTERNS[p], None, ctypes.byref(out))
    L.eh_test_fail_alloc_after(-1)
    torch.cuda.synchronize()
    f1 = torch.cuda.mem_get_info()[0]
    res.append((p, r, f0 - f1, int(out.value), t.count(p)))
print(repr(res))
"""


def test_first_call_in_a_fresh_process_allocates_nothing(eh):
    # the first noalloc call of a process (after a trie build and its work
    # plan, but no count) must not change the device's free memory
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = eval(r.stdout.strip().splitlines()[-1])
    for p, status, used, got, want in res:
        assert status == 0 and used == 0 and got == want, (p, status, used, got, want)
