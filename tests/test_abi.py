"""The C-ABI library loads and exports every function include/eh.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_1503_02368_gb300 as eh
from paper_1503_02368_gb300 import eh as ehmod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(eh_\w+)\s*\(", src, flags=re.M):
                names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    L = eh.lib()
    names = declared_functions()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(ehmod.EXPORTED) <= names


# the boundary calls the pattern-count engine is built around: the trie
# build, the counts, the batch, statistics, release and errors
BOUNDARY = ["eh_build_trie", "eh_count", "eh_count_batch", "eh_trie_stats", "eh_free_trie", "eh_last_error"]


def test_boundary_names_exported_and_declared():
    L = eh.lib()
    names = declared_functions()
    for n in BOUNDARY + ["eh_count_range", "eh_count_range_async", "eh_range_bounds"]:
        assert n in names, n
        assert hasattr(L, n), n


def test_every_declaration_cites_a_passage_or_says_it_has_none():
    # each function declaration of the header is preceded by a comment that
    # names a passage of the paper (Sec., Table, Algorithm, App.) or states
    # that the paper has no counterpart
    src = open(os.path.join(ROOT, "include", "eh.h")).read()
    missing = []
    for name in BOUNDARY + ["eh_count_range", "eh_count_noalloc"]:
        i = src.index(" " + name + "(")
        j = src.rindex("/*", 0, i)
        comment = src[j:src.index("*/", j)]
        if not re.search(r"Sec\. |Table \d|Algorithm \d|App\. |no counterpart|not in the paper", comment):
            missing.append(name)
    assert not missing, missing


def test_range_bounds_cover_every_item_once_without_gpu():
    import numpy as np
    rng = np.random.default_rng(3)
    for n in (0, 1, 7, 1000):
        cost = rng.integers(0, 1000, size=n).astype(np.uint64)
        if n > 3:
            cost[-3:] = 0                                   # zero-cost tail goes to the last part
        total = int(cost.sum())
        for nparts in (1, 2, 3, 8, 13):
            parts = [eh.range_bounds(cost, p, nparts) for p in range(nparts)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            for (a, b), (c, d) in zip(parts, parts[1:]):
                assert b == c and a <= b
            mx = int(cost.max()) if n else 0
            for a, b in parts:
                assert abs(int(cost[a:b].sum()) - total / nparts) <= mx + 1e-9


def test_range_bounds_rejects_bad_parts_without_gpu():
    import numpy as np
    with pytest.raises(eh.EHError):
        eh.range_bounds(np.ones(4, np.uint64), 2, 2)
    with pytest.raises(eh.EHError):
        eh.range_bounds(np.ones(4, np.uint64), 0, 0)


def test_checked_build_exports_the_same_symbols():
    # libeh_check.so: the same library with the count kernels' loads range-checked
    lib = os.path.join(ROOT, "paper_1503_02368_gb300", "libeh_check.so")
    assert os.path.exists(lib)
    L = ctypes.CDLL(lib)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_last_error_is_callable_without_gpu():
    L = eh.lib()
    assert isinstance(L.eh_last_error(), bytes)


def test_null_arguments_rejected_without_device_work():
    L = eh.lib()
    out = ctypes.c_uint64(0)
    assert L.eh_count(None, 0, None, 0, None, ctypes.byref(out)) == 1
    assert L.eh_count_async(None, 0, None, None, None) == 1
    assert L.eh_build_trie(None, None, 0, 0, None, None, None) == 1
    assert L.eh_trie_stats_get(None, None) == 1


def test_structs_match_header_sizes(tmp_path):
    # the sizes the C compiler gives the header's structs, against the binding's
    import subprocess
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "eh.h"\nint main(void) { printf("%zu %zu %zu %zu %zu %zu %zu\\n", '
                   'sizeof(eh_build_opts), sizeof(eh_exec_opts), sizeof(eh_query), sizeof(eh_trie_stats_t), '
                   'sizeof(eh_count_info), sizeof(eh_server_stats), sizeof(eh_batch_profile)); return 0; }\n')
    exe = tmp_path / "sizes"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-I", inc, str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == [ctypes.sizeof(ehmod.BuildOpts), ctypes.sizeof(ehmod.ExecOpts), ctypes.sizeof(ehmod.Query),
                   ctypes.sizeof(ehmod.TrieStats), ctypes.sizeof(ehmod.CountInfo),
                   ctypes.sizeof(ehmod.ServerStats), ctypes.sizeof(ehmod.BatchProfile)]


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(ehmod, "_lib", None)
    monkeypatch.setattr(ehmod, "_LIB_PATH", "/nonexistent/libeh.so")
    with pytest.raises(RuntimeError):
        ehmod.lib()
