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
    src.write_text('#include <stdio.h>\n#include "eh.h"\nint main(void) { printf("%zu %zu %zu %zu %zu %zu\\n", '
                   'sizeof(eh_build_opts), sizeof(eh_exec_opts), sizeof(eh_query), sizeof(eh_trie_stats), '
                   'sizeof(eh_count_info), sizeof(eh_server_stats)); return 0; }\n')
    exe = tmp_path / "sizes"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-I", inc, str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == [ctypes.sizeof(ehmod.BuildOpts), ctypes.sizeof(ehmod.ExecOpts), ctypes.sizeof(ehmod.Query),
                   ctypes.sizeof(ehmod.TrieStats), ctypes.sizeof(ehmod.CountInfo),
                   ctypes.sizeof(ehmod.ServerStats)]


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(ehmod, "_lib", None)
    monkeypatch.setattr(ehmod, "_LIB_PATH", "/nonexistent/libeh.so")
    with pytest.raises(RuntimeError):
        ehmod.lib()
