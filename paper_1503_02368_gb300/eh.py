"""ctypes binding of libeh.so (argument marshalling only).

Every computation happens in the library's CUDA kernels; when the library is
missing this module raises instead of falling back to anything else.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# EH_LIBRARY may name the checked build (libeh_check.so, the count kernels'
# loads range-checked); it must exist like the default library
_LIB_PATH = os.environ.get("EH_LIBRARY") or os.path.join(_HERE, "libeh.so")
_lib = None

PATTERNS = {"triangle": 0, "clique4": 1, "lollipop": 2, "lollipop_distinct": 3, "barbell": 4}
STATUS = {0: "EH_OK", 1: "EH_EINVAL", 2: "EH_ENOMEM", 3: "EH_ECUDA", 4: "EH_ETIMEOUT", 5: "EH_EOVERFLOW",
          6: "EH_EBUSY", 7: "EH_ECAPACITY"}
EH_BUILD_DEVICE_INPUT = 1
EH_BUILD_BLOCK_LAYOUT = 2


class EHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


ORDERINGS = {"degree": 0, "rev_degree": 1, "random": 2, "bfs": 3, "strong_runs": 4, "shingle": 5, "hybrid": 6,
             "identity": 7}


class BuildOpts(ctypes.Structure):
    _fields_ = [("bitset_tau", ctypes.c_uint32), ("min_bitset_len", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("ordering", ctypes.c_uint32), ("order_seed", ctypes.c_uint32)]


class ExecOpts(ctypes.Structure):
    _fields_ = [("gallop_ratio", ctypes.c_uint32), ("light_max", ctypes.c_uint32), ("cta_warps", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("pair_warps", ctypes.c_uint32)]


class TrieStats(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_uint32), ("n_active", ctypes.c_uint32), ("n_edges", ctypes.c_uint64),
                ("max_degree", ctypes.c_uint32), ("max_out_degree", ctypes.c_uint32),
                ("n_bitset_sets", ctypes.c_uint64), ("n_nonempty_sets", ctypes.c_uint64),
                ("bitset_words", ctypes.c_uint64), ("density_skew", ctypes.c_double),
                ("device_bytes", ctypes.c_uint64), ("bitset_tau", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class CountInfo(ctypes.Structure):
    _fields_ = [("alg_bytes", ctypes.c_double), ("n_heavy", ctypes.c_uint64), ("n_light", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("alg_bytes_stored", ctypes.c_double)]


class Query(ctypes.Structure):
    _fields_ = [("pattern", ctypes.c_uint32), ("subset_len", ctypes.c_uint32), ("subset_off", ctypes.c_uint64)]


class BatchProfile(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("sub_vertices", ctypes.c_uint64),
                ("sub_set_elements", ctypes.c_uint64), ("heavy_items", ctypes.c_uint64),
                ("light_items", ctypes.c_uint64), ("prepare_s", ctypes.c_double), ("count_s", ctypes.c_double),
                ("graph_reuses", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("bytes_in_use", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("mean_batch", ctypes.c_double)]


EXPORTED = ["eh_build_trie", "eh_count", "eh_count_ex", "eh_count_noalloc", "eh_count_async", "eh_count_status", "eh_count_info_get",
            "eh_count_range", "eh_count_range_async", "eh_range_bounds",
            "eh_vertex_triangles", "eh_count_batch", "eh_count_batch_ex", "eh_batch_profile_get", "eh_trie_stats",
            "eh_trie_stats_get", "eh_trie_export",
            "eh_free_trie", "eh_last_error", "eh_selftest_wait_timeout", "eh_test_fail_alloc_after", "eh_server_create", "eh_server_submit", "eh_server_poll",
            "eh_server_wait", "eh_server_latency", "eh_server_stats_get", "eh_server_destroy"]


def library_path():
    return _LIB_PATH


def lib():
    """Loads libeh.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError("libeh.so is not built (run __graft_entry__.build()); there is no fallback path")
    L = ctypes.CDLL(_LIB_PATH)
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    u32p, u64p = ctypes.POINTER(u32), ctypes.POINTER(u64)
    st = ctypes.c_int
    L.eh_last_error.restype = ctypes.c_char_p
    L.eh_last_error.argtypes = []
    L.eh_build_trie.restype = st
    L.eh_build_trie.argtypes = [vp, vp, u64, u32, ctypes.POINTER(BuildOpts), vp, ctypes.POINTER(vp)]
    L.eh_count.restype = st
    L.eh_count.argtypes = [vp, st, u32p, u32, vp, u64p]
    L.eh_count_ex.restype = st
    L.eh_count_ex.argtypes = [vp, st, u32p, u32, ctypes.POINTER(ExecOpts), vp, u64p]
    L.eh_count_noalloc.restype = st
    L.eh_count_noalloc.argtypes = [vp, st, vp, u64p]
    L.eh_count_async.restype = st
    L.eh_count_async.argtypes = [vp, st, ctypes.POINTER(ExecOpts), vp, vp]
    L.eh_count_status.restype = st
    L.eh_count_status.argtypes = [vp, vp]
    L.eh_count_range.restype = st
    L.eh_count_range.argtypes = [vp, st, u32, u32, ctypes.POINTER(ExecOpts), vp, u64p]
    L.eh_count_range_async.restype = st
    L.eh_count_range_async.argtypes = [vp, st, u32, u32, ctypes.POINTER(ExecOpts), vp, vp]
    L.eh_range_bounds.restype = st
    L.eh_range_bounds.argtypes = [u64p, u64, u32, u32, u64p, u64p]
    L.eh_trie_stats.restype = st
    L.eh_trie_stats.argtypes = [vp, ctypes.POINTER(TrieStats)]
    L.eh_count_info_get.restype = st
    L.eh_count_info_get.argtypes = [vp, st, ctypes.POINTER(ExecOpts), vp, ctypes.POINTER(CountInfo)]
    L.eh_trim_memory.restype = st
    L.eh_trim_memory.argtypes = []
    L.eh_trie_export_blocks.restype = st
    L.eh_trie_export_blocks.argtypes = [vp, u64p, u32p, u32p, u64p, u64p]
    L.eh_count_selected.restype = st
    L.eh_count_selected.argtypes = [vp, st, u32, ctypes.POINTER(ExecOpts), vp, u64p]
    L.eh_list.restype = st
    L.eh_list.argtypes = [vp, st, ctypes.POINTER(ExecOpts), vp, vp, u64, u64p]
    L.eh_vertex_triangles.restype = st
    L.eh_vertex_triangles.argtypes = [vp, vp, u64p]
    L.eh_count_batch.restype = st
    L.eh_count_batch.argtypes = [vp, ctypes.POINTER(Query), u32, u32p, u64, vp, u64p, ctypes.POINTER(ctypes.c_int)]
    L.eh_count_batch_ex.restype = st
    L.eh_count_batch_ex.argtypes = [vp, ctypes.POINTER(Query), u32, u32p, u64, ctypes.POINTER(ExecOpts), u32, vp,
                                    u64p, ctypes.POINTER(ctypes.c_int)]
    L.eh_batch_profile_get.restype = st
    L.eh_batch_profile_get.argtypes = [ctypes.POINTER(BatchProfile)]
    L.eh_trie_stats_get.restype = st
    L.eh_trie_stats_get.argtypes = [vp, ctypes.POINTER(TrieStats)]
    L.eh_trie_export.restype = st
    L.eh_trie_export.argtypes = [vp, u32, u32p, u64p, u32p, u32p, u32p, u32p, u64p, u32p]
    L.eh_test_fail_alloc_after.restype = None
    L.eh_test_fail_alloc_after.argtypes = [ctypes.c_longlong]
    L.eh_selftest_wait_timeout.restype = st
    L.eh_selftest_wait_timeout.argtypes = [u32, vp]
    L.eh_free_trie.restype = None
    L.eh_free_trie.argtypes = [vp]
    L.eh_server_create.restype = st
    L.eh_server_create.argtypes = [vp, u64, u32, u32, ctypes.POINTER(vp)]
    L.eh_server_submit.restype = st
    L.eh_server_submit.argtypes = [vp, st, u32p, u32, u64p]
    L.eh_server_poll.restype = st
    L.eh_server_poll.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_int), u64p, ctypes.POINTER(ctypes.c_int)]
    L.eh_server_wait.restype = st
    L.eh_server_wait.argtypes = [vp, u64, u32, u64p, ctypes.POINTER(ctypes.c_int)]
    L.eh_server_latency.restype = st
    L.eh_server_latency.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_double)]
    L.eh_server_stats_get.restype = st
    L.eh_server_stats_get.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.eh_server_destroy.restype = None
    L.eh_server_destroy.argtypes = [vp]
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise EHError(status, lib().eh_last_error().decode(errors="replace"))


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _stream(stream):
    """cudaStream_t handle: an int, a torch.cuda.Stream, or None (torch's current stream)."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def batch_profile():
    """Phase times of this thread's last count_batch call."""
    p = BatchProfile()
    _check(lib().eh_batch_profile_get(ctypes.byref(p)))
    return {f: getattr(p, f) for f, _ in BatchProfile._fields_}


def range_bounds(cost, part, nparts):
    """eh_range_bounds: the items [lo, hi) of part `part` of `nparts` of a list
    with per-item costs `cost` (host-only; the split eh_count_range applies)."""
    cost = np.ascontiguousarray(cost, np.uint64)
    lo, hi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().eh_range_bounds(_u64p(cost), len(cost), part, nparts, ctypes.byref(lo), ctypes.byref(hi)))
    return int(lo.value), int(hi.value)


def trim_memory():
    """Return the device temporaries cached in the default memory pool (eh_trim_memory)."""
    _check(lib().eh_trim_memory())


def build_opts(tau=32, min_bitset_len=0, flags=0, ordering="degree", order_seed=0):
    o = ORDERINGS[ordering] if isinstance(ordering, str) else int(ordering)
    return BuildOpts(tau & 0xFFFFFFFF, min_bitset_len, flags, o, order_seed)


EH_EXEC_SORTED_A = 1
EH_EXEC_GLOBAL_A = 2


def exec_opts(gallop_ratio=0, light_max=0, cta_warps=0, flags=0, pair_warps=0):
    return ExecOpts(gallop_ratio, light_max, cta_warps, flags, pair_warps)


def _pattern(p):
    return PATTERNS[p] if isinstance(p, str) else int(p)


class Trie:
    """Device-resident trie of a simple undirected graph (eh_build_trie)."""

    def __init__(self, src, dst, n_vertices, tau=32, min_bitset_len=0, stream=None, ordering="degree",
                 order_seed=0, block_layout=False):
        L = lib()
        self._h = ctypes.c_void_p(0)
        flags = 0
        if hasattr(src, "data_ptr"):          # torch tensors already on the device
            assert src.is_cuda and dst.is_cuda and src.numel() == dst.numel()
            ps, pd, ne = src.data_ptr(), dst.data_ptr(), src.numel()
            flags = EH_BUILD_DEVICE_INPUT
        else:
            src = np.ascontiguousarray(src, np.uint32)
            dst = np.ascontiguousarray(dst, np.uint32)
            assert len(src) == len(dst)
            ps, pd, ne = src.ctypes.data, dst.ctypes.data, len(src)
        if block_layout:
            flags |= EH_BUILD_BLOCK_LAYOUT
        o = build_opts(tau, min_bitset_len, flags, ordering, order_seed)
        _check(L.eh_build_trie(ctypes.c_void_p(ps), ctypes.c_void_p(pd), ne, n_vertices, ctypes.byref(o),
                               _stream(stream), ctypes.byref(self._h)))
        self.n = n_vertices
        self.tau = tau

    def close(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.eh_free_trie(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        self.close()

    @property
    def handle(self):
        return self._h

    def count(self, pattern, subset=None, xopts=None, stream=None):
        out = ctypes.c_uint64(0)
        if subset is not None:
            subset = np.ascontiguousarray(subset, np.uint32)
            sp, sl = _u32p(subset), len(subset)
        else:
            sp, sl = None, 0
        xo = ctypes.byref(xopts) if xopts is not None else None
        _check(lib().eh_count_ex(self._h, _pattern(pattern), sp, sl, xo, _stream(stream), ctypes.byref(out)))
        return int(out.value)

    def count_range(self, pattern, part, nparts, xopts=None, stream=None):
        """eh_count_range: part `part` of `nparts` of the whole-graph count."""
        out = ctypes.c_uint64(0)
        xo = ctypes.byref(xopts) if xopts is not None else None
        _check(lib().eh_count_range(self._h, _pattern(pattern), part, nparts, xo, _stream(stream),
                                    ctypes.byref(out)))
        return int(out.value)

    def count_range_async(self, pattern, part, nparts, d_out_ptr, xopts=None, stream=None):
        xo = ctypes.byref(xopts) if xopts is not None else None
        _check(lib().eh_count_range_async(self._h, _pattern(pattern), part, nparts, xo, _stream(stream),
                                          ctypes.c_void_p(d_out_ptr)))

    def count_async(self, pattern, d_out_ptr, xopts=None, stream=None):
        xo = ctypes.byref(xopts) if xopts is not None else None
        _check(lib().eh_count_async(self._h, _pattern(pattern), xo, _stream(stream), ctypes.c_void_p(d_out_ptr)))

    def status(self, stream=None):
        _check(lib().eh_count_status(self._h, _stream(stream)))

    def info(self, pattern="triangle", xopts=None, stream=None):
        ci = CountInfo()
        xo = ctypes.byref(xopts) if xopts is not None else None
        _check(lib().eh_count_info_get(self._h, _pattern(pattern), xo, _stream(stream), ctypes.byref(ci)))
        return {f: getattr(ci, f) for f, _ in CountInfo._fields_ if f != "reserved"}

    def stats(self):
        s = TrieStats()
        _check(lib().eh_trie_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in TrieStats._fields_ if f != "reserved"}

    def count_selected(self, pattern, node, xopts=None, stream=None):
        """Selection query count (eh_count_selected): 'clique4' (SK4) or
        'barbell' (SB3,1) with attribute x bound to the neighbours of `node`."""
        out = ctypes.c_uint64(0)
        xo = ctypes.byref(xopts) if xopts is not None else None
        _check(lib().eh_count_selected(self._h, {"clique4": 0, "barbell": 1}[pattern], node, xo, _stream(stream),
                                       ctypes.byref(out)))
        return int(out.value)

    def list_into(self, pattern, d_out_ptr, capacity, xopts=None, stream=None):
        """eh_list into a caller's device buffer of `capacity` rows; returns the
        number of rows of the result (EHError EH_ECAPACITY if they do not fit)."""
        n = ctypes.c_uint64(0)
        xo = ctypes.byref(xopts) if xopts is not None else None
        _check(lib().eh_list(self._h, _pattern(pattern), xo, _stream(stream),
                             ctypes.c_void_p(d_out_ptr) if d_out_ptr else None, capacity, ctypes.byref(n)))
        return int(n.value)

    def list(self, pattern="triangle", xopts=None, stream=None):
        """Every triangle ('triangle') or 4-clique ('clique4') once, as a device
        tensor [rows, 3|4] of int32 holding the uint32 original ids in ascending
        order (rows in no particular order).  The buffer is sized by a count."""
        import torch
        width = {"triangle": 3, "clique4": 4}[pattern]
        rows = self.count(pattern, xopts=xopts, stream=stream)
        out = torch.empty((max(rows, 1), width), dtype=torch.int32, device="cuda")
        got = self.list_into(pattern, out.data_ptr(), rows, xopts=xopts, stream=stream)
        assert got == rows
        return out[:rows]

    def vertex_triangles(self, stream=None):
        out = np.zeros(self.n, np.uint64)
        _check(lib().eh_vertex_triangles(self._h, _stream(stream), _u64p(out)))
        return out

    def export(self, which=0):
        """Host copy of the pruned (which=0) or symmetric (which=1) trie."""
        n = self.n
        st = self.stats()
        off = np.zeros(n + 1, np.uint64)
        L = lib()
        _check(L.eh_trie_export(self._h, which, None, _u64p(off), None, None, None, None, None, None))
        new2old = np.zeros(n, np.uint32)
        ln = np.zeros(n, np.uint32)
        nbr = np.zeros(max(int(off[-1]), 1), np.uint32)
        blo = np.zeros(n, np.uint32)
        bnw = np.zeros(n, np.uint32)
        boff = np.zeros(n, np.uint64)
        words = np.zeros(max(int(st["bitset_words"]), 1), np.uint32)
        _check(L.eh_trie_export(self._h, which, _u32p(new2old), _u64p(off), _u32p(ln), _u32p(nbr), _u32p(blo),
                                _u32p(bnw), _u64p(boff), _u32p(words)))
        return {"new_to_old": new2old, "off": off, "len": ln, "nbr": nbr, "bits_lo": blo, "bits_nwords": bnw,
                "bits_off": boff, "words": words}

    def export_blocks(self):
        """Host copy of the composite layout: (off[n+1], dir[n_blocks, 2], words[n_bit_blocks, 8])."""
        nb, nbit = ctypes.c_uint64(0), ctypes.c_uint64(0)
        L = lib()
        _check(L.eh_trie_export_blocks(self._h, None, None, None, ctypes.byref(nb), ctypes.byref(nbit)))
        off = np.zeros(self.n + 1, np.uint64)
        d = np.zeros((max(nb.value, 1), 2), np.uint32)
        w = np.zeros((max(nbit.value, 1), 8), np.uint32)
        _check(L.eh_trie_export_blocks(self._h, _u64p(off), _u32p(d), _u32p(w), ctypes.byref(nb), ctypes.byref(nbit)))
        return off, d[:nb.value], w[:nbit.value]

    def count_batch(self, patterns, offsets, pool, mode=0, xopts=None, stream=None):
        """Queries i = (patterns[i], pool[offsets[i]:offsets[i+1]]); returns (counts, statuses)."""
        nq = len(patterns)
        offsets = np.asarray(offsets, np.uint64)
        pool = np.ascontiguousarray(pool, np.uint32)
        qs = (Query * max(nq, 1))()
        for i in range(nq):
            qs[i].pattern = _pattern(patterns[i])
            qs[i].subset_off = int(offsets[i])
            qs[i].subset_len = int(offsets[i + 1] - offsets[i])
        counts = np.zeros(max(nq, 1), np.uint64)
        sts = (ctypes.c_int * max(nq, 1))()
        xo = ctypes.byref(xopts) if xopts is not None else None
        r = lib().eh_count_batch_ex(self._h, qs, nq, _u32p(pool), len(pool), xo, mode, _stream(stream),
                                    _u64p(counts), sts)
        statuses = np.array(list(sts)[:nq], np.int32)
        if r != 0 and not np.any(statuses != 0):
            _check(r)
        return counts[:nq], statuses


class Server:
    """Continuous-batching request loop over a resident trie (eh_server_*)."""

    def __init__(self, trie, memory_budget_bytes, max_batch=256, max_inflight=4):
        self._h = ctypes.c_void_p(0)
        self.trie = trie
        _check(lib().eh_server_create(trie.handle, memory_budget_bytes, max_batch, max_inflight,
                                      ctypes.byref(self._h)))

    def submit(self, pattern, subset):
        subset = np.ascontiguousarray(subset, np.uint32)
        t = ctypes.c_uint64(0)
        r = lib().eh_server_submit(self._h, _pattern(pattern), _u32p(subset), len(subset), ctypes.byref(t))
        if r == 6:
            return None
        _check(r)
        return int(t.value)

    def poll(self, ticket):
        done, cnt, st = ctypes.c_int(0), ctypes.c_uint64(0), ctypes.c_int(0)
        _check(lib().eh_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(cnt), ctypes.byref(st)))
        return bool(done.value), int(cnt.value), int(st.value)

    def wait(self, ticket, timeout_ms=0):
        cnt, st = ctypes.c_uint64(0), ctypes.c_int(0)
        _check(lib().eh_server_wait(self._h, ticket, timeout_ms, ctypes.byref(cnt), ctypes.byref(st)))
        return int(cnt.value), int(st.value)

    def latency(self, ticket):
        x = ctypes.c_double(0)
        _check(lib().eh_server_latency(self._h, ticket, ctypes.byref(x)))
        return float(x.value)

    def stats(self):
        s = ServerStats()
        _check(lib().eh_server_stats_get(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.eh_server_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        self.close()
