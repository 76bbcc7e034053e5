// eh_internal.cuh -- shared definitions of the CUDA implementation of eh.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdarg.h>
#include <string.h>

#include <mutex>
#include <vector>
#include <map>

#include "eh.h"
#include <nvtx3/nvToolsExt.h>

// NVTX range for the lifetime of a scope (visible in Nsight Systems / Compute)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// ------------------------------------------------------------------ errors

void eh_set_error(const char *fmt, ...);

#define EH_CUDA_TRY(call)                                                                       \
    do {                                                                                        \
        cudaError_t _e = (call);                                                                \
        if (_e != cudaSuccess) {                                                                \
            eh_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(_e));     \
            return _e == cudaErrorMemoryAllocation ? EH_ENOMEM : EH_ECUDA;                      \
        }                                                                                       \
    } while (0)

#define EH_TRY(call)                                   \
    do {                                               \
        eh_status _s = (call);                         \
        if (_s != EH_OK) return _s;                    \
    } while (0)

// device-side status bits (written with atomicOr, read by the host)
enum : uint32_t {
    DEV_ST_TIMEOUT = 1u,   // a bounded mbarrier wait gave up
    DEV_ST_OVERFLOW = 2u,  // an accumulator passed 2^63
    DEV_ST_INVALID = 4u,   // an input id was out of range
    DEV_ST_RANGE = 8u,     // a listing row fell outside the range its count pass gave it (not written)
    DEV_ST_BOUNDS = 16u,   // checked build (EH_CHECK_LOADS): a load outside its array (not made)
};

// Scratch layout of a whole-graph count (unsigned long long words of
// eh_trie::d_scratch, and of the static array of eh_count_noalloc): the
// accumulators the count kernels add into and their work counters.
enum {
    SC_T = 0,      // triangles
    SC_S = 1,      // sum over triangles of the three degrees (lollipop)
    SC_CNT = 2,    // 2 words: next heavy item, next light chunk (triangle kernels)
    SC_K4 = 4,     // 4-cliques (also the barbell's sum)
    SC_CNT2 = 6,   // 2 words: the 4-clique kernel's work counters
    SC_WORDS = 8   // words cleared before each count
};

// ------------------------------------------------------------ set layouts
//
// Every pruned set N+(v) is kept as a sorted uint32 array in `nbr`, starting
// on a 16-byte boundary and padded to a multiple of four elements with
// EH_PAD (never a valid id).  When the set-level rule selects the bitset
// layout, a bitset copy is kept as well: `nwords` 32-bit words starting at
// word `woff` of the bitset pool, bit b of word i standing for the value
// 32*(lo_word+i)+b.  lo_word and nwords are multiples of 4, so that two
// bitsets line up on 128-bit vectors.
#define EH_PAD 0xFFFFFFFFu

struct __align__(16) SetDesc {
    uint64_t off;      // element offset of the uint array in nbr (multiple of 4)
    uint32_t len;      // |N+(v)|
    uint32_t deg;      // d(v) in the symmetric graph
    uint64_t woff;     // word offset of the bitset in words (multiple of 4)
    uint32_t lo_word;  // first covered word, value/32 (multiple of 4)
    uint32_t nwords;   // 0 = uint layout only
};

// The device view of one pruned trie (whole graph or one induced subgraph).
struct TrieView {
    const SetDesc *desc;    // per vertex
    const uint32_t *nbr;    // uint arrays
    const uint32_t *words;  // bitset pool
    const uint32_t *deg;    // d(v), symmetric degree
    uint32_t n;
    uint64_t n_nbr = 0, n_words = 0;   // array extents (the checked build's load checks)
};

// Concatenated induced sub-tries of a batch of queries (see count.cu).
struct BatchView {
    const SetDesc *desc;    // per sub-vertex
    const uint32_t *nbr;    // sets of local ids
    const uint32_t *words;  // bitset pool
    const uint32_t *deg;    // degree in the induced subgraph
    const uint32_t *sub_q;  // query of each sub-vertex
    const uint32_t *qbase;  // first sub-vertex of each query (n_queries + 1)
    const uint32_t *qpat;   // pattern of each query
    uint64_t n_sub = 0, n_nbr = 0, n_words = 0, n_queries = 0;   // extents (checked build)
};

// per-pattern work lists (vertex ids, heaviest first)
struct WorkPlan {
    uint32_t light_max = 0;
    uint32_t *d_heavy = nullptr;   // |N+(u)| > light_max
    uint32_t n_heavy = 0;
    uint32_t *d_light = nullptr;   // 2 <= |N+(u)| <= light_max
    uint32_t n_light = 0;
    uint32_t *d_heavy_blk = nullptr;   // block layout only: the heavy list, big items first (blocks.cu)
    uint32_t n_big = 0;
    // algorithmic bytes of one pass (< 0: not computed yet; eh_plan_alg_bytes)
    double alg_bytes = -1.0;        // triangle pass, lower bound over the stored layouts
    double alg_bytes_stored = -1.0; // triangle pass, each set at its stored layout's size
    double alg_bytes_k4 = -1.0;     // 4-clique pass, lower bound (both levels, spills)
    uint64_t *d_cost = nullptr;     // per vertex: sum_{v in N+(u)} |N+(v)| (the lists' order key)
    // exclusive prefix sums of d_cost along the heavy and the light list
    // (n_heavy + 1 and n_light + 1 entries), built on the first range count
    std::vector<uint64_t> h_heavy_pre, h_light_pre;
};

struct eh_trie {
    uint32_t n = 0;         // id space
    uint32_t n_active = 0;  // vertices with degree > 0 (new ids [0, n_active))
    uint32_t nb = 1;        // bits for an id
    uint64_t m = 0;         // unique undirected edges
    uint32_t max_deg = 0, max_out = 0;
    eh_build_opts opts{};

    uint32_t *d_new2old = nullptr, *d_old2new = nullptr;
    // symmetric trie N(v)
    uint64_t *d_soff = nullptr;   // n+1 padded offsets
    uint32_t *d_snbr = nullptr;
    uint64_t snbr_len = 0;
    // pruned trie N+(v)
    SetDesc *d_desc = nullptr;    // n
    uint32_t *d_onbr = nullptr;
    uint64_t onbr_len = 0;
    uint32_t *d_words = nullptr;
    uint64_t n_words = 0;
    uint32_t *d_deg = nullptr;    // n, symmetric degree (new ids)
    uint64_t n_bitset = 0, n_nonempty = 0;
    // composite (block-level) layout, EH_BUILD_BLOCK_LAYOUT only (blocks.cu)
    uint64_t *d_boff = nullptr;   // n+1 directory offsets
    uint2 *d_bdir = nullptr;      // {block id, info}
    uint32_t *d_bwords = nullptr; // 8 words per bitset block
    uint64_t n_blocks = 0, n_bit_blocks = 0;
    double density_skew = 0;
    uint64_t device_bytes = 0;
    std::vector<uint32_t> h_out_by_old;   // |N+(v)| by original id (host; serving footprints; built on first use)

    // scratch owned by the trie: counters, accumulators, status
    unsigned long long *d_scratch = nullptr;  // 16 words
    uint32_t *d_arena = nullptr;              // 4-clique spill arena for large S sets
    uint64_t arena_words = 0;
    uint32_t *d_status = nullptr;

    std::mutex mu;        // guards plans
    std::mutex call_mu;   // serialises synchronous counts (they share d_scratch)
    std::map<uint32_t, WorkPlan> plans;   // keyed by light_max

    TrieView view() const {
        TrieView v;
        v.desc = d_desc; v.nbr = d_onbr; v.words = d_words; v.deg = d_deg; v.n = n;
        v.n_nbr = onbr_len; v.n_words = n_words;
        return v;
    }
};

// ------------------------------------------------------------- primitives

// Exclusive prefix sum of n values (in may equal out).  Returns the total in
// *total_host when non-null (synchronises the stream).
eh_status dev_exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, cudaStream_t s,
                                 uint64_t *total_host);
eh_status dev_exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t s,
                                 uint64_t *total_host);
// Stable LSD radix sort of keys on bits [0, key_bits) (bits above are ignored,
// not required to be zero); result in *keys (the two buffers may be swapped
// on return).
eh_status dev_radix_sort_u64(uint64_t **keys, uint64_t **tmp, uint64_t n, int key_bits, cudaStream_t s);

// Allocation-failure injection for tests (eh_test_fail_alloc_after): when
// armed, the countdown-th device allocation from now fails as if out of memory.
bool eh_alloc_should_fail();

// Device memory helpers (stream-ordered).
template <typename T>
eh_status dev_alloc(T **p, uint64_t count, cudaStream_t s) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (eh_alloc_should_fail()) {
        eh_set_error("device allocation of %llu bytes failed (injected)", (unsigned long long)(sizeof(T) * count));
        return EH_ENOMEM;
    }
    cudaError_t e = cudaMallocAsync((void **)p, sizeof(T) * count, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        eh_set_error("device allocation of %llu bytes failed: %s", (unsigned long long)(sizeof(T) * count),
                     cudaGetErrorString(e));
        return EH_ENOMEM;
    }
    return EH_OK;
}

template <typename T>
void dev_free(T *&p, cudaStream_t s) {
    if (p) cudaFreeAsync((void *)p, s);
    p = nullptr;
}

static inline uint32_t ceil_div_u32(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

// blocks of t threads covering n items
static inline unsigned blocks_for(uint64_t n, unsigned t = 256) { return (unsigned)((n + t - 1) / t); }

// bits to represent values in [0, n)
static inline int bits_for(uint64_t n) {
    int b = 1;
    while (b < 63 && (1ull << b) < n) ++b;
    return b;
}

int eh_num_sms();

// Count entry points shared between files.
eh_status eh_plan_get(eh_trie *t, uint32_t light_max, cudaStream_t s, WorkPlan **out);
// a plan's algorithmic bytes of one pass, computed on first use and cached:
// which = ALG_TRI (lower bound), ALG_TRI_STORED (stored layouts), ALG_K4
enum { ALG_TRI = 0, ALG_TRI_STORED = 1, ALG_K4 = 2 };
eh_status eh_plan_alg_bytes(eh_trie *t, WorkPlan *p, cudaStream_t s, int which, double *out);
// the cost prefixes of the plan's lists on the host (built on first use)
eh_status eh_plan_cost_prefix(eh_trie *t, WorkPlan *p, cudaStream_t s);
// part `part` of `nparts` contiguous ranges of a list whose items have the
// exclusive cost prefix pre[0..n]: [*lo, *hi), the items i with
// pre[i] * nparts in [part * total, (part + 1) * total) -- every item in
// exactly one part, each part within one item's cost of total / nparts
void eh_split_range(const uint64_t *pre, uint64_t n, uint32_t part, uint32_t nparts, uint64_t *lo, uint64_t *hi);
// eh_launch_triangle modes: 0 count, 1 lollipop, 2 per-vertex t (d_vt[n]),
// TRI_MODE_APEX: each work item's triangles in which it is the largest id, to
// d_vt[item] for heavy items and d_vt[n_heavy + i] for light item i
constexpr int TRI_MODE_APEX = 3;

// per-warp shared buffer of the 4-clique's materialised S = N+(x) ∩ N+(y), in
// elements, in the count and batch kernels; a set longer than this needs the
// global spill arena (512 measured faster than 1024: a smaller shared carve-out
// leaves more L1)
constexpr uint32_t K4_S_CAP = 512;
eh_status eh_launch_triangle(const eh_trie *t, const WorkPlan &plan, TrieView tv, int mode,
                             const eh_exec_opts &xo, cudaStream_t s, unsigned long long *d_acc,
                             unsigned long long *d_counters, uint32_t *d_status, unsigned long long *d_vt,
                             const uint32_t *d_qid);
eh_status eh_launch_clique4(const eh_trie *t, const WorkPlan &plan, TrieView tv, const eh_exec_opts &xo,
                            cudaStream_t s, unsigned long long *d_acc, unsigned long long *d_counters,
                            uint32_t *d_status, uint32_t *d_arena, uint64_t arena_words_per_warp);
eh_exec_opts eh_exec_defaults(const eh_exec_opts *x);
// grid_warps != NULL: only reports the warps of the launch (sizes the arena)
eh_status eh_launch_batch(const BatchView &bv, const uint32_t *heavy, uint32_t n_heavy, const uint32_t *light,
                          uint32_t n_light, const eh_exec_opts &xo, cudaStream_t s, unsigned long long *d_out,
                          unsigned long long *d_counters, uint32_t *d_status, uint32_t *arena,
                          uint64_t arena_words_per_warp, uint32_t *grid_warps);
// set-level layouts of a pruned trie given as padded uint arrays (trie_build.cu)
eh_status eh_build_layouts(const uint32_t *nbr, const uint64_t *off, const uint32_t *len, const uint32_t *deg,
                           uint32_t nv, uint32_t tau, uint32_t min_len, cudaStream_t s, SetDesc *desc_out,
                           uint32_t **words_out, uint64_t *n_words_out, uint64_t *n_bitset_out);
// node ordering of the dictionary encoding: new2old[n] from the unique pairs
// (lo << nb | hi, original ids) and the degrees (order.cu)
eh_status eh_vertex_order(uint32_t ordering, uint32_t seed, const uint64_t *ukeys, uint64_t m, uint32_t n, int nb,
                          const uint32_t *deg, uint32_t maxdeg, cudaStream_t s, uint32_t *new2old);
// composite layout: build the directories of the pruned sets; the triangle
// count over them (adds into d_acc; d_next = 2 zeroed counters) (blocks.cu)
eh_status eh_build_blocks(eh_trie *t, uint32_t tau, cudaStream_t s);
// the block-layout count's order of the heavy list (plan.d_heavy_blk, n_big)
eh_status eh_plan_blocks(eh_trie *t, WorkPlan *p, cudaStream_t s);
eh_status eh_launch_tri_blocks(eh_trie *t, const WorkPlan &plan, cudaStream_t s, unsigned long long *d_acc,
                               unsigned int *d_next);
// fills eh_trie::h_out_by_old if not yet built (trie_build.cu)
eh_status eh_host_out_degrees(eh_trie *t);
// SK4 per-x sum over the selected vertex's neighbours (list.cu)
eh_status eh_sk4_total(eh_trie *t, uint32_t node_new, const eh_exec_opts &xo, cudaStream_t s, uint64_t *total);
// the result of `pattern` from the SC_* accumulators at acc, to *out (api.cu)
eh_status eh_launch_finalize(const unsigned long long *acc, int pattern, unsigned long long *out, uint32_t *status,
                             cudaStream_t s);
// eh_count_noalloc's set-up on the current device (count.cu), once per
// device: resolves the static scratch array's device address and runs the
// kernels the call launches once on empty work lists (on `s`, synchronised),
// so that the array and the kernels are resident before the first call
eh_status eh_noalloc_setup(cudaStream_t s);
eh_status eh_enqueue_whole(eh_trie *t, eh_pattern pattern, const eh_exec_opts &xo, cudaStream_t s,
                           unsigned long long *d_out);
eh_status eh_check_status(eh_trie *t, cudaStream_t s);
