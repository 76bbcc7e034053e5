"""CPU oracle for the pattern COUNT(*) queries (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product path never does.  The C source
(``eh_oracle.c``) is a plain nested-loop generic join with scalar merges.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eh_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        ip = ctypes.POINTER(ctypes.c_int)
        vp = ctypes.c_void_p
        L.oracle_canon.restype = ctypes.c_int64
        L.oracle_canon.argtypes = [u32p, u32p, ctypes.c_uint64, ctypes.c_uint32, u32p, u32p]
        L.oracle_graph_new.restype = vp
        L.oracle_graph_new.argtypes = [ctypes.c_uint32, u32p, u32p, ctypes.c_uint64]
        L.oracle_graph_free.argtypes = [vp]
        L.oracle_graph_n.restype = ctypes.c_uint32
        L.oracle_graph_n.argtypes = [vp]
        L.oracle_graph_m.restype = ctypes.c_uint64
        L.oracle_graph_m.argtypes = [vp]
        L.oracle_neighbours.restype = ctypes.c_uint64
        L.oracle_neighbours.argtypes = [vp, ctypes.c_uint32, u32p]
        for f in (L.oracle_triangles, L.oracle_clique4):
            f.restype = ctypes.c_uint64
            f.argtypes = [vp, ctypes.c_int, ctypes.c_int, ip]
        for f in (L.oracle_lollipop, L.oracle_lollipop_distinct):
            f.restype = ctypes.c_uint64
            f.argtypes = [vp, ctypes.c_int, ip]
        L.oracle_vertex_triangles.argtypes = [vp, u32p, ctypes.c_uint64, u64p]
        L.oracle_barbell.restype = ctypes.c_uint64
        L.oracle_barbell.argtypes = [vp, ip]
        L.oracle_triangles_outer.restype = ctypes.c_uint64
        L.oracle_triangles_outer.argtypes = [vp, u32p, ctypes.c_uint64, ctypes.c_int, u64p, ip]
        L.oracle_list_triangles_at.restype = ctypes.c_uint64
        L.oracle_list_triangles_at.argtypes = [vp, ctypes.c_uint32, u32p, ctypes.c_uint64]
        for f in (L.oracle_list_triangles, L.oracle_list_clique4):
            f.restype = ctypes.c_uint64
            f.argtypes = [vp, u32p, ctypes.c_uint64]
        L.oracle_induced.restype = vp
        L.oracle_induced.argtypes = [vp, u32p, ctypes.c_uint64]
        L.oracle_block_layout.restype = ctypes.c_uint64
        L.oracle_block_layout.argtypes = [u32p, ctypes.c_uint64, ctypes.c_uint32, u32p,
                                          ctypes.POINTER(ctypes.c_uint8)]
        L.oracle_layout_is_bitset.restype = ctypes.c_int
        L.oracle_layout_is_bitset.argtypes = [u32p, ctypes.c_uint64, ctypes.c_uint32]
        L.oracle_degree_order.argtypes = [vp, u32p]
        L.oracle_count_selected.restype = ctypes.c_uint64
        L.oracle_count_selected.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, ip]
        L.oracle_vertex_order.restype = ctypes.c_int
        L.oracle_vertex_order.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, u32p]
        _lib = L
    return _lib


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _threads(t):
    return int(t) if t else 1


class OverflowError64(ArithmeticError):
    pass


def canon(src, dst, n):
    """Canonical simple undirected edge set (a<b), sorted, unique."""
    src = np.ascontiguousarray(src, np.uint32)
    dst = np.ascontiguousarray(dst, np.uint32)
    a = np.empty(len(src), np.uint32)
    b = np.empty(len(src), np.uint32)
    m = lib().oracle_canon(_u32p(src), _u32p(dst), len(src), n, _u32p(a), _u32p(b))
    if m == -1:
        raise ValueError("vertex id >= n")
    if m < 0:
        raise MemoryError("oracle_canon")
    return a[:m].copy(), b[:m].copy()


class Graph:
    """Simple undirected graph as a two-level trie (oracle side)."""

    def __init__(self, n, src=None, dst=None, _handle=None):
        if _handle is not None:
            self._h = _handle
            return
        a, b = canon(src, dst, n)
        self._h = lib().oracle_graph_new(n, _u32p(a), _u32p(b), len(a))
        if not self._h:
            raise MemoryError("oracle graph")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_graph_free(h)
            self._h = None

    @property
    def n(self):
        return int(lib().oracle_graph_n(self._h))

    @property
    def m(self):
        return int(lib().oracle_graph_m(self._h))

    def neighbours(self, v):
        d = lib().oracle_neighbours(self._h, v, None)
        out = np.empty(d, np.uint32)
        lib().oracle_neighbours(self._h, v, _u32p(out))
        return out

    def degrees(self):
        return np.array([lib().oracle_neighbours(self._h, v, None) for v in range(self.n)], np.uint64)

    def _chk(self, val, ovf):
        if ovf.value:
            raise OverflowError64("count exceeds uint64")
        return int(val)

    def triangles(self, pruned=True, nthreads=1):
        o = ctypes.c_int(0)
        return self._chk(lib().oracle_triangles(self._h, int(pruned), _threads(nthreads), ctypes.byref(o)), o)

    def triangles_outer(self, verts, nthreads=1):
        """Pruned triangle loop nest over the listed outer vertices only:
        returns (count, pruned edges covered)."""
        verts = np.ascontiguousarray(verts, np.uint32)
        o = ctypes.c_int(0)
        e = ctypes.c_uint64(0)
        c = lib().oracle_triangles_outer(self._h, _u32p(verts), len(verts), _threads(nthreads), ctypes.byref(e),
                                         ctypes.byref(o))
        return self._chk(c, o), int(e.value)

    def clique4(self, pruned=True, nthreads=1):
        o = ctypes.c_int(0)
        return self._chk(lib().oracle_clique4(self._h, int(pruned), _threads(nthreads), ctypes.byref(o)), o)

    def lollipop(self, nthreads=1):
        o = ctypes.c_int(0)
        return self._chk(lib().oracle_lollipop(self._h, _threads(nthreads), ctypes.byref(o)), o)

    def lollipop_distinct(self, nthreads=1):
        o = ctypes.c_int(0)
        return self._chk(lib().oracle_lollipop_distinct(self._h, _threads(nthreads), ctypes.byref(o)), o)

    def barbell(self, nthreads=1):
        o = ctypes.c_int(0)
        return self._chk(lib().oracle_barbell(self._h, ctypes.byref(o)), o)

    def count(self, pattern, nthreads=1):
        """pattern: 'triangle' | 'clique4' | 'lollipop' | 'lollipop_distinct' | 'barbell'."""
        return {"triangle": self.triangles, "clique4": self.clique4, "lollipop": self.lollipop,
                "lollipop_distinct": self.lollipop_distinct, "barbell": self.barbell}[pattern](nthreads=nthreads)

    def count_selected(self, pattern, node):
        """Selection queries with attribute x bound to N(node): 'clique4' (SK4)
        or 'barbell' (SB3,1), join semantics on the symmetric relation."""
        o = ctypes.c_int(0)
        k = {"clique4": 0, "barbell": 1}[pattern]
        return self._chk(lib().oracle_count_selected(self._h, k, node, ctypes.byref(o)), o)

    def vertex_triangles(self, verts):
        verts = np.ascontiguousarray(verts, np.uint32)
        out = np.empty(len(verts), np.uint64)
        lib().oracle_vertex_triangles(self._h, _u32p(verts), len(verts),
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        return out

    def list(self, pattern):
        """Every triangle ('triangle') or 4-clique ('clique4') once, as rows of
        ascending original ids, in the oracle's loop order: uint32 [k, 3|4]."""
        fn, width = {"triangle": (lib().oracle_list_triangles, 3),
                     "clique4": (lib().oracle_list_clique4, 4)}[pattern]
        k = int(fn(self._h, None, 0))
        out = np.empty((k, width), np.uint32)
        if k:
            fn(self._h, _u32p(out), k)
        return out

    def list_triangles_at(self, x):
        """The triangles containing vertex x, rows of ascending ids: uint32 [t(x), 3]."""
        k = int(lib().oracle_list_triangles_at(self._h, x, None, 0))
        out = np.empty((k, 3), np.uint32)
        if k:
            lib().oracle_list_triangles_at(self._h, x, _u32p(out), k)
        return out

    def induced(self, subset):
        subset = np.ascontiguousarray(subset, np.uint32)
        h = lib().oracle_induced(self._h, _u32p(subset), len(subset))
        if not h:
            raise ValueError("subset id >= n")
        return Graph(0, _handle=h)

    ORDERINGS = {"degree": 0, "rev_degree": 1, "random": 2, "bfs": 3, "strong_runs": 4, "shingle": 5,
                 "hybrid": 6, "identity": 7}

    def vertex_order(self, ordering, seed=0):
        """new_to_old permutation of a node ordering (App. "Node Ordering")."""
        out = np.empty(self.n, np.uint32)
        if lib().oracle_vertex_order(self._h, self.ORDERINGS[ordering], seed, _u32p(out)) != 0:
            raise ValueError("oracle_vertex_order")
        return out

    def degree_order(self):
        out = np.empty(self.n, np.uint32)
        lib().oracle_degree_order(self._h, _u32p(out))
        return out


def layout_is_bitset(sorted_set, tau):
    s = np.ascontiguousarray(sorted_set, np.uint32)
    return bool(lib().oracle_layout_is_bitset(_u32p(s), len(s), tau))


def block_layout(sorted_set, tau):
    """Composite layout of a sorted set: (block ids, is_bitset) per 256-value block."""
    s = np.ascontiguousarray(sorted_set, np.uint32)
    ids = np.empty(max(len(s), 1), np.uint32)
    kind = np.empty(max(len(s), 1), np.uint8)
    k = int(lib().oracle_block_layout(_u32p(s), len(s), tau, _u32p(ids),
                                      kind.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
    return ids[:k].copy(), kind[:k].astype(bool)
