"""Seeded synthetic inputs: raw edge lists and ego-network vertex subsets.

This package produces inputs only (see ``synth.c``).  It holds none of the
pattern-counting method's arithmetic, and both the CPU oracle and the CUDA
path consume exactly what it emits.  Every number is drawn from a
counter-based SplitMix64 stream, so the same seed gives the same graph on any
machine and under any thread count.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

BASE_SEED = 1503


def build(force=False):
    """Compile libsynth.so in-tree (gcc, no FMA contraction, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.synth_rng.restype = ctypes.c_uint64
        L.synth_rng.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.synth_key.restype = ctypes.c_uint64
        L.synth_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        L.synth_det_log.restype = ctypes.c_double
        L.synth_det_log.argtypes = [ctypes.c_double]
        L.synth_det_exp.restype = ctypes.c_double
        L.synth_det_exp.argtypes = [ctypes.c_double]
        L.synth_er.restype = ctypes.c_int
        L.synth_er.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p]
        L.synth_rmat.restype = ctypes.c_int
        L.synth_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_uint64, u32p, u32p, ctypes.c_int]
        L.synth_chunglu.restype = ctypes.c_int
        L.synth_chunglu.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_uint64, ctypes.c_uint64, u32p, u32p, ctypes.c_int]
        L.synth_chunglu_weight.restype = ctypes.c_double
        L.synth_chunglu_weight.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.synth_graph_new.restype = ctypes.c_void_p
        L.synth_graph_new.argtypes = [ctypes.c_uint32, u32p, u32p, ctypes.c_uint64, ctypes.c_int]
        L.synth_graph_free.argtypes = [ctypes.c_void_p]
        L.synth_graph_degree.restype = ctypes.c_uint64
        L.synth_graph_degree.argtypes = [ctypes.c_void_p, ctypes.c_uint32]
        L.synth_ego_batch.restype = ctypes.c_void_p
        L.synth_ego_batch.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int, u64p]
        L.synth_ego_fetch.argtypes = [ctypes.c_void_p, u32p]
        L.synth_ego_free.argtypes = [ctypes.c_void_p]
        _lib = L
    return _lib


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def key(base, a=0, b=0):
    """Stream key from a base seed and two labels."""
    return int(lib().synth_key(base, a, b))


def rng(k, i):
    return int(lib().synth_rng(k, i))


def er(n, m, k):
    """Erdos-Renyi G(n, m): exactly m distinct unordered pairs, random direction."""
    src = np.empty(m, np.uint32)
    dst = np.empty(m, np.uint32)
    if lib().synth_er(n, m, k, _u32p(src), _u32p(dst)) != 0:
        raise ValueError("G(n,m) needs m <= n(n-1)/2")
    return src, dst


def rmat(scale, n_edges, k, a=0.57, b=0.19, c=0.19, nthreads=None):
    """R-MAT raw edge list (direction, repeats and loops as generated)."""
    src = np.empty(n_edges, np.uint32)
    dst = np.empty(n_edges, np.uint32)
    if lib().synth_rmat(scale, n_edges, a, b, c, k, _u32p(src), _u32p(dst), _threads(nthreads)) != 0:
        raise ValueError("bad R-MAT scale")
    return src, dst


def chunglu(n, n_pairs, k, gamma=2.1, i0=49.7268008, wmax=50000.0, nthreads=None):
    """Chung-Lu raw pairs with endpoints drawn proportional to w_i = c (i+i0)^(-1/(gamma-1))."""
    src = np.empty(n_pairs, np.uint32)
    dst = np.empty(n_pairs, np.uint32)
    if lib().synth_chunglu(n, gamma, i0, wmax, n_pairs, k, _u32p(src), _u32p(dst), _threads(nthreads)) != 0:
        raise ValueError("bad Chung-Lu parameters")
    return src, dst


def chunglu_weight(i, gamma=2.1, i0=49.7268008, wmax=50000.0):
    return float(lib().synth_chunglu_weight(i, gamma, i0, wmax))


def ego_subsets(n, src, dst, k, n_queries, mode, lo, hi, nthreads=None):
    """Ego-network vertex subsets (BFS prefixes) of the raw graph.

    mode 0: |S| = floor(lo (hi/lo)^U) vertices; mode 1: shortest BFS prefix whose
    induced (simple) edge count reaches floor(lo (hi/lo)^U).  Returns
    (offsets[n_queries+1] uint64, pool uint32) with subsets in BFS order."""
    L = lib()
    g = L.synth_graph_new(n, _u32p(src), _u32p(dst), len(src), _threads(nthreads))
    if not g:
        raise MemoryError("synth graph")
    try:
        off = np.zeros(n_queries + 1, np.uint64)
        res = L.synth_ego_batch(g, k, n_queries, mode, float(lo), float(hi), _threads(nthreads),
                                off.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        pool = np.empty(int(off[-1]), np.uint32)
        L.synth_ego_fetch(res, _u32p(pool))
        L.synth_ego_free(res)
    finally:
        L.synth_graph_free(g)
    return off, pool
