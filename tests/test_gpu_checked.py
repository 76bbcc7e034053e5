"""The checked build (libeh_check.so): the count kernels with every global
load verified against the extent of the array it reads (sets, bitset words,
degrees, descriptors, work lists, bulk-copy sources).  A load outside them
is not made and the call returns EH_ECUDA with a message.  These cases run
small graphs through every dispatch path of the count kernels under it, in a
subprocess bound to that library, and require both the oracle's counts and a
clean status: no load of these runs leaves its array."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CASES = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import paper_1503_02368_gb300 as eh
import oracle
from synth import workloads as W
from tests import graphs as G
assert eh.library_path().endswith("libeh_check.so"), eh.library_path()
PATS = ("triangle", "clique4", "lollipop", "lollipop_distinct", "barbell")
done = 0

def check(n, s, d, taus, xos=(None,), pats=PATS, blocks=False):
    global done
    o = oracle.Graph(n, s, d)
    want = {p: o.count(p, nthreads=8) for p in pats}
    for tau in taus:
        t = eh.Trie(s, d, n, tau=tau, block_layout=blocks)
        for xo in xos:
            x = eh.exec_opts(**xo) if xo else None
            for p in pats:
                got = t.count(p, xopts=x)
                assert got == want[p], (p, tau, xo, got, want[p])
                done += 1
        t.close()

rng = np.random.default_rng(5)
for k in range(4):
    n = int(rng.integers(50, 600))
    s, d = G.arrays(G.random_graph(n, float(rng.choice([0.02, 0.1, 0.3])), rng))
    check(n, s, d, (0, 8, 32, 256, 0xFFFFFFFF))
# hubs: heavy CTA items with on-chip bitmaps and sorted arrays, long sets
n = 30000
e = [(int(h), int(v)) for h in range(24) for v in rng.choice(np.arange(24, n), 2500, replace=False)]
e += [(int(a), int(b)) for a, b in rng.integers(0, 600, size=(20000, 2))]
s, d = G.arrays(e)
check(n, s, d, (0, 32, 1024, 0xFFFFFFFF),
      xos=(None, dict(pair_warps=2), dict(pair_warps=4, cta_warps=16), dict(cta_warps=4, light_max=8),
           dict(gallop_ratio=1), dict(gallop_ratio=1000)))
check(n, s, d, (256,), pats=("triangle",), blocks=True)
# a 1,100-clique: 4-clique sets S beyond the shared buffer, in the spill arena
s, d = G.arrays(G.complete(1100) + [(1100 + i, i) for i in range(300)])
check(1400, s, d, (32,), pats=("triangle", "clique4"))
# R-MAT: whole graph, range parts and an ego-net batch
g = W.rmat_graph(13, 1503 + 13)
o = oracle.Graph(g["n"], g["src"], g["dst"])
t = eh.Trie(g["src"], g["dst"], g["n"], tau=256)
for p in ("triangle", "clique4", "lollipop"):
    want = o.count(p, nthreads=8)
    assert t.count(p) == want
    assert sum(t.count_range(p, k, 3) for k in range(3)) == want
import synth
off, pool = synth.ego_subsets(g["n"], g["src"], g["dst"], synth.key(7, 7), 24, 0, 16, 1024)
pats = ["triangle", "clique4", "lollipop"] * 8
c, st = t.count_batch(pats, off, pool)
assert not st.any()
for q in range(24):
    assert int(c[q]) == o.induced(pool[off[q]:off[q + 1]]).count(pats[q], nthreads=4), q
t.close()
print("checked ok", done)
"""


def test_checked_build_runs_every_count_path_in_bounds():
    lib = os.path.join(ROOT, "paper_1503_02368_gb300", "libeh_check.so")
    assert os.path.exists(lib), "libeh_check.so is built by __graft_entry__.build()"
    env = dict(os.environ, EH_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", _CASES, ROOT], capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "checked ok" in r.stdout
