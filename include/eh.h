/*
 * eh.h -- C ABI of the GB300 pattern-count engine (libeh.so).
 *
 * The engine evaluates COUNT(*) graph pattern queries by the generic
 * worst-case optimal join (EmptyHeaded, Aberger et al., SIGMOD'16,
 * arXiv 1503.02368, Algorithm 1) over a two-level trie of sorted 32-bit
 * neighbour sets (Sec. 2.2), each set stored in a density-chosen uint or
 * bitset layout (Sec. 4.1, set-level rule of Sec. 4.4).  Its operations are
 * those of the paper's execution engine (Table 2): R[t] (the set under a
 * prefix), for-x-in-xs, and xs ∩ ys, composed for the triangle, 4-clique and
 * lollipop queries of Table 1.
 *
 * Conventions for every call:
 *   - Every function returns an eh_status and never aborts, exits or traps.
 *     On failure eh_last_error() gives a message (thread-local, valid until
 *     the next call on the same thread).
 *   - Host pointers are owned by the caller; the library copies what it
 *     needs before returning.  Device pointers are accepted only where a flag
 *     says so.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that return host results synchronise that stream before returning.
 *   - Vertex ids are uint32 in [0, n_vertices).  Direction is ignored;
 *     self-loops and repeated pairs are dropped (the graph is simple and
 *     undirected).
 *   - Counts are exact uint64.  A count that would exceed 2^64-1 returns
 *     EH_EOVERFLOW.
 *   - Device temporaries are stream-ordered allocations from the device's
 *     default memory pool.  The first eh_build_trie on a device raises that
 *     pool's release threshold for the process, so freed temporaries stay
 *     cached for the next call instead of being unmapped at every
 *     synchronisation; eh_trim_memory returns them to the driver.
 *   - Concurrency: a trie is read-only after eh_build_trie.  Batches
 *     (eh_count_batch*, subset counts, the server) own all their device state
 *     and may run concurrently on different streams.  Whole-graph counts use
 *     a small scratch area of the trie: eh_count/eh_count_ex serialise on it,
 *     while eh_count_async calls on one trie must be issued on one stream (or
 *     otherwise ordered) and not overlap an eh_count on the same trie.
 */
#ifndef EH_H
#define EH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EH_OK = 0,
    EH_EINVAL = 1,    /* bad argument: id >= n_vertices, NULL pointer, unknown pattern */
    EH_ENOMEM = 2,    /* device or host allocation failed; nothing leaked */
    EH_ECUDA = 3,     /* a CUDA runtime error (message in eh_last_error) */
    EH_ETIMEOUT = 4,  /* a bounded device-side wait ran out; the context stays usable */
    EH_EOVERFLOW = 5, /* a count exceeds uint64 */
    EH_EBUSY = 6,     /* admission refused: the query does not fit the memory budget now */
    EH_ECAPACITY = 7  /* an output buffer is smaller than the result (the size needed is returned) */
} eh_status;

/* Table 1 patterns, COUNT(*) semantics:
 *   EH_TRIANGLE  Triangle(x,y,z) :- R(x,y),S(y,z),T(x,z)          each triangle once
 *   EH_CLIQUE4   4Clique(x,y,z,w) :- R,S,T,U,V,Q (all six pairs)   each 4-clique once
 *   EH_LOLLIPOP  Lollipop(x,y,z,w) :- R(x,y),S(y,z),T(x,z),U(x,w)  on the undirected
 *                relation, datalog join semantics (ordered tuples, w unconstrained):
 *                sum_x 2 t(x) d(x), with t(x) the triangles at x and d(x) its degree
 *   EH_LOLLIPOP_DISTINCT  lollipop subgraphs (triangle + pendant edge, w outside the
 *                triangle), each once: sum_x t(x) (d(x) - 2)
 *   EH_BARBELL   Barbell(x,y,z,x',y',z') :- triangle at x, U(x,x'), triangle at x'
 *                on the undirected relation, join semantics, by the two-node GHD
 *                plan (triangles aggregated per vertex first, Sec. 3.1):
 *                sum over ordered edges (x,x') of 2 t(x) * 2 t(x').  Whole graph
 *                only (EH_EINVAL with a subset or in a batch).                    */
typedef enum {
    EH_TRIANGLE = 0,
    EH_CLIQUE4 = 1,
    EH_LOLLIPOP = 2,
    EH_LOLLIPOP_DISTINCT = 3,
    EH_BARBELL = 4
} eh_pattern;

typedef struct eh_trie eh_trie; /* opaque, device-resident, owned by the library */

/* eh_build_trie options.  Pass NULL for the defaults (tau 32, input on host,
 * degree ordering). */
typedef struct {
    /* Set-level layout rule (Sec. 4.4): a set S is stored as a bitset when its
     * range max-min+1 is at most bitset_tau bits per element (range <= tau*|S|).
     * 0 = every set uint (the paper's relation-level "-R" configuration);
     * 0xFFFFFFFF = every non-empty set bitset.  The paper's value is 256 (one
     * AVX register per element). */
    uint32_t bitset_tau;
    uint32_t min_bitset_len; /* sets shorter than this stay uint (default 0) */
    uint32_t flags;          /* EH_BUILD_* */
    uint32_t ordering;       /* eh_ordering: how original ids become trie ids (default EH_ORDER_DEGREE) */
    uint32_t order_seed;     /* seed of EH_ORDER_RANDOM and EH_ORDER_SHINGLE */
} eh_build_opts;

/* Node orderings of the dictionary encoding (App. "Node Ordering"): the
 * permutation from original ids to the trie's ids.  Pruning keeps each edge in
 * the set of its larger trie id, so the ordering decides the shape of N+(v)
 * (counts do not depend on it).  Vertices without edges take part like any
 * other.  h(v) = SplitMix64 of the counter (order_seed * 2^32 + v).
 *   EH_ORDER_DEGREE       degree descending, ties by original id
 *   EH_ORDER_REV_DEGREE   degree ascending, ties by original id
 *   EH_ORDER_RANDOM       by h(v), ties by original id
 *   EH_ORDER_BFS          breadth-first from the highest-degree vertex (first in
 *                         EH_ORDER_DEGREE), neighbours in ascending id; vertices
 *                         it does not reach follow in EH_ORDER_DEGREE order
 *   EH_ORDER_STRONG_RUNS  vertices visited in EH_ORDER_DEGREE order; each
 *                         labels itself if unlabelled, then its unlabelled
 *                         neighbours in ascending id
 *   EH_ORDER_SHINGLE      by the min-hash shingle min_{w in N(v)} h(w) (its top
 *                         64 - bits(n) bits), ties by id; no neighbours: last
 *   EH_ORDER_HYBRID       EH_ORDER_BFS positions re-sorted by degree
 *                         descending; equal degrees keep their BFS order
 *   EH_ORDER_IDENTITY     the original ids */
typedef enum {
    EH_ORDER_DEGREE = 0,
    EH_ORDER_REV_DEGREE = 1,
    EH_ORDER_RANDOM = 2,
    EH_ORDER_BFS = 3,
    EH_ORDER_STRONG_RUNS = 4,
    EH_ORDER_SHINGLE = 5,
    EH_ORDER_HYBRID = 6,
    EH_ORDER_IDENTITY = 7
} eh_ordering;

#define EH_BUILD_DEVICE_INPUT 1u /* src/dst are device pointers (read on `stream`) */
/* Composite (block-level) layout of Sec. 4.3 instead of the set-level one: the
 * value domain cut into blocks of 256 values; in each pruned set a block
 * holding c values is a 256-bit bitset when 256 <= bitset_tau * c, else its
 * run of the uint array.  Triangle counts of such a trie intersect block
 * directories (eh_trie_export_blocks); the other patterns use the uint arrays. */
#define EH_BUILD_BLOCK_LAYOUT 2u

/* Execution knobs for the intersection kernels.  NULL = defaults; a field
 * left 0 takes its default. */
typedef struct {
    uint32_t gallop_ratio;  /* uint∩uint: gallop when |large| > ratio*|small| (Sec. 4.2's 32:1); default 32 */
    uint32_t light_max;     /* vertices with |N+(u)| <= light_max run one warp each; default 32 (at most 32) */
    uint32_t cta_warps;     /* warps per CTA for heavy vertices (4, 8 or 16); default 8 */
    uint32_t flags;         /* EH_EXEC_* bits, 0 by default */
    /* warps per intersection: how many warps of a heavy vertex's CTA share one
     * pair (u, v), each taking every pair_warps-th step of N+(v) against the
     * staged N+(u) (1, 2 or 4; default 1).  Whole-graph triangle and lollipop
     * counts; the other patterns take one warp per pair.  At 1, when N+(u) is
     * staged as a bitmap, the triangle and lollipop counts give each of the
     * four pairs a warp takes at a time a quarter warp (8 lanes) for the word
     * AND pairs, and the whole warp for the others. */
    uint32_t pair_warps;
} eh_exec_opts;

/* eh_list staging of A = N+(u) for vertices taken by a whole CTA: by default
 * the kernel keeps A on chip as a bitmap when its value range fits, else as a
 * sorted array when it fits, else reads it from device memory.  These bits
 * force the later forms (same rows, other code paths; the counts ignore them). */
#define EH_EXEC_SORTED_A 1u /* never a bitmap: the sorted array (on chip when it fits) */
#define EH_EXEC_GLOBAL_A 2u /* A read from device memory, not staged */

/* Facts of a built trie.  The struct tag is the name of the call that fills
 * it (eh_trie_stats), so C and C++ code names the type `struct eh_trie_stats`
 * or `eh_trie_stats_t`. */
struct eh_trie_stats {
    uint32_t n_vertices;   /* id space */
    uint32_t n_active;     /* vertices with degree > 0 */
    uint64_t n_edges;      /* unique undirected edges m */
    uint32_t max_degree;   /* max d(v) */
    uint32_t max_out_degree; /* max |N+(v)| of the pruned (degree-oriented) relation */
    uint64_t n_bitset_sets;  /* pruned sets stored as bitsets */
    uint64_t n_nonempty_sets;
    uint64_t bitset_words;   /* 32-bit words in the bitset pool */
    double density_skew;     /* Pearson's first skewness 3(mean-mode)/sigma of the degrees (Sec. 4 footnote) */
    uint64_t device_bytes;   /* device memory held by the trie */
    uint32_t bitset_tau;
    uint32_t reserved;
};
typedef struct eh_trie_stats eh_trie_stats_t;

/* One query of a batch: pattern over the subgraph induced by
 * subset_pool[subset_off .. subset_off+subset_len) (original ids; order and
 * repeats are irrelevant).  subset_len == 0 means the whole graph. */
typedef struct {
    uint32_t pattern;   /* eh_pattern */
    uint32_t subset_len;
    uint64_t subset_off;
} eh_query;

/* eh_build_trie -- edge list to a device-resident trie (Sec. 2.2; pruning
 * and degree ordering of Sec. 5.2.1 / App. A.1.1; layout rule of Sec. 4.4).
 *   src, dst    n_edges vertex ids each (host, or device with EH_BUILD_DEVICE_INPUT)
 *   n_vertices  id space; every id must be < n_vertices, else EH_EINVAL
 *   out         receives the trie; release it with eh_free_trie.
 * Builds: the simple undirected edge set; new ids by (degree desc, original
 * id asc); the symmetric trie N(v) and the pruned trie N+(v) = {u in N(v) :
 * u < v} (new ids), each set sorted, 16-byte aligned; a bitset copy of each
 * pruned set the layout rule selects; the per-vertex work list. */
eh_status eh_build_trie(const uint32_t *src, const uint32_t *dst, uint64_t n_edges, uint32_t n_vertices,
                        const eh_build_opts *opts, void *stream, eh_trie **out);

/* eh_count -- COUNT(*) of `pattern` over the whole graph (subset == NULL or
 * subset_len == 0) or over the subgraph induced by `subset` (host array of
 * original ids, any order, repeats allowed).  Writes *out_count (host).
 * The COUNT(*) queries of Table 1, evaluated by Algorithm 1 (Generic-Join)
 * with the attribute order of the Sec. 3.3.2 loop nest on the pruned trie of
 * App. A.1.2 (x > y > z: each triangle, each 4-clique once).  The induced
 * subgraph restriction is not in the paper (a batching pattern of this
 * library, see eh_count_batch). */
eh_status eh_count(const eh_trie *trie, eh_pattern pattern, const uint32_t *subset, uint32_t subset_len,
                   void *stream, uint64_t *out_count);

/* eh_count_ex -- as eh_count with explicit execution knobs (NULL = defaults). */
eh_status eh_count_ex(const eh_trie *trie, eh_pattern pattern, const uint32_t *subset, uint32_t subset_len,
                      const eh_exec_opts *xopts, void *stream, uint64_t *out_count);

/* eh_count_async -- whole-graph count enqueued on `stream` with no host
 * synchronisation: the uint64 result is written to device memory
 * d_out_count (8 bytes, caller-owned, 8-byte aligned).  Errors found on the
 * device (a timed-out wait, an overflow) are reported by the next
 * eh_count_status call. */
eh_status eh_count_async(const eh_trie *trie, eh_pattern pattern, const eh_exec_opts *xopts, void *stream,
                         uint64_t *d_out_count);

/* eh_count_status -- synchronises `stream` and returns the device-side
 * status word of the trie's last asynchronous counts (then clears it). */
eh_status eh_count_status(const eh_trie *trie, void *stream);

/* eh_count_range -- one part of a whole-graph count split across `nparts`
 * workers, such as one process per GPU each holding a replica of the trie:
 * the sum of the results of parts 0 .. nparts-1 is eh_count's result.  Not
 * in the paper, which runs on one shared-memory node (Sec. 5.1.4); the parts
 * split the outermost loop of Algorithm 1 (the vertex x of the Sec. 3.3.2
 * loop nest), whose iterations are independent.
 *   pattern     EH_TRIANGLE, EH_CLIQUE4, EH_LOLLIPOP or EH_LOLLIPOP_DISTINCT
 *               (each a sum over the outer vertices); EH_BARBELL is EH_EINVAL
 *   part        0 .. nparts-1; nparts >= 1 (else EH_EINVAL)
 *   out_count   host uint64: this part's share.  The call synchronises `stream`.
 * The work plan's heavy and light lists (in their locality order) are each cut into
 * nparts contiguous ranges of about equal estimated cost (per vertex u,
 * sum over v in N+(u) of |N+(v)|; as eh_range_bounds); the first call on a
 * plan copies the lists' cost prefix sums to the host (8 bytes per listed
 * vertex).  A trie with the block layout is counted here with the set-level
 * kernel.  Serialised with the other synchronous counts of the trie. */
eh_status eh_count_range(const eh_trie *trie, eh_pattern pattern, uint32_t part, uint32_t nparts,
                         const eh_exec_opts *xopts, void *stream, uint64_t *out_count);

/* eh_count_range_async -- as eh_count_range with the result written to device
 * memory d_out_count (8 bytes, caller-owned) and no host synchronisation;
 * the same ordering rules as eh_count_async (device errors come back through
 * eh_count_status). */
eh_status eh_count_range_async(const eh_trie *trie, eh_pattern pattern, uint32_t part, uint32_t nparts,
                               const eh_exec_opts *xopts, void *stream, uint64_t *d_out_count);

/* eh_range_bounds -- the split eh_count_range applies to each list, on host
 * arrays (no device work): items 0 .. n-1 with costs cost[0 .. n-1] in list
 * order; part `part` of `nparts` is the items [*lo, *hi), those whose cost
 * prefix P(i) = cost[0] + ... + cost[i-1] has P(i) * nparts in
 * [part * total, (part + 1) * total) (the last part also takes the items with
 * P(i) = total).  Consecutive parts are adjacent and together cover 0 .. n-1
 * once; each part's cost is within one item's cost of total / nparts.
 * EH_EINVAL on a bad argument, EH_EOVERFLOW when the total exceeds uint64. */
eh_status eh_range_bounds(const uint64_t *cost, uint64_t n, uint32_t part, uint32_t nparts, uint64_t *lo,
                          uint64_t *hi);

/* eh_count_noalloc -- a whole-graph count (as eh_count) that allocates
 * nothing.  For callers that may not allocate device memory while they
 * count: a process that has handed its device memory to a fixed pool or
 * budget, code running where an allocation could block or fail at the wrong
 * moment.  The paper has no counterpart: this is a property of this library.
 *   trie       a trie built by eh_build_trie whose work plan exists: call
 *              eh_count_info_get (or any whole-graph count) on it once first,
 *              otherwise EH_EINVAL.
 *   pattern    EH_TRIANGLE, EH_CLIQUE4, EH_LOLLIPOP or EH_LOLLIPOP_DISTINCT;
 *              EH_BARBELL (which needs a per-vertex array) is EH_EINVAL.  A
 *              trie with the block layout is counted with the set-level
 *              kernel (same result as eh_count).
 *   out_count  host uint64, written on success.  The call synchronises `stream`.
 * Scratch (work counters, accumulators, status word and the 4-clique spill
 * arena) lives in one 32 MiB static device array that every device using the
 * library keeps until the process exits.  The first eh_build_trie on a
 * device makes it resident there: it looks up the array's device address
 * (cudaGetSymbolAddress, with that device current; this commits the array's
 * memory) and runs the kernels this call launches once on empty work lists.
 * On a device where no trie was built, the first call does that set-up
 * itself (and may then allocate); make that first call before any stream
 * capture.
 * The 4-clique pattern needs max out-degree x launch warps x 4 bytes of arena
 * when the max out-degree exceeds 512; above 32 MiB the call returns
 * EH_EINVAL with the sizes in eh_last_error, before launching anything.
 * All calls share the array (each clears its counters first): calls whose
 * work overlaps on the GPU, on any trie or stream, race and must not be
 * issued. */
eh_status eh_count_noalloc(const eh_trie *trie, eh_pattern pattern, void *stream, uint64_t *out_count);

/* eh_count_info_get -- work-plan facts of a whole-graph count (builds the
 * plan if needed): the bytes the method must move in one pass (the
 * set-intersection inner loop of Algorithm 1, where the paper finds up to
 * 95% of Generic-Join's runtime, Sec. 1), the number of heavy (CTA) and light (warp)
 * vertices, and the kernel launches one eh_count_async enqueues.
 *   alg_bytes  a lower bound over the stored layouts (Sec. 4.1): the staged
 *              set once per vertex in its cheaper form; per intersection the
 *              cheapest way to read what of the other set can meet the
 *              staged prefix (its uint array, the bitset words overlapping
 *              the staged set's range, or at most 32 bytes per probe); 8
 *              bytes per edge of offsets.  Triangle family (also the lollipop
 *              and barbell): the pairs (N+(u)_<v, N+(v)).  EH_CLIQUE4: level 1
 *              as the triangle, level 2 the pairs (S_<z, N+(z)) of every
 *              S = N+(x) ∩ N+(y), plus 8 bytes per element of S when S is
 *              longer than the kernel's 512-element on-chip buffer.
 *   alg_bytes_stored  triangle family only (0 for EH_CLIQUE4): every set at
 *              its stored layout's size (4|S| uint, 4 x words bitset), N+(u)
 *              once per u, N+(v) once per pair unless |N+(v)| > 32 |N+(u)|,
 *              then at most 32 bytes per element of N+(u); 8 bytes per edge.
 * Each figure is computed by a device pass on the first call for a plan and
 * cached; the call synchronises `stream`. */
typedef struct {
    double alg_bytes;
    uint64_t n_heavy;
    uint64_t n_light;
    uint32_t kernel_launches;
    uint32_t reserved;
    double alg_bytes_stored;
} eh_count_info;

eh_status eh_count_info_get(const eh_trie *trie, eh_pattern pattern, const eh_exec_opts *xopts, void *stream,
                            eh_count_info *out);

/* eh_vertex_triangles -- t(x), the number of triangles containing x, for
 * every original id x (host array of n_vertices uint64). */
eh_status eh_vertex_triangles(const eh_trie *trie, void *stream, uint64_t *out_t);

/* eh_list -- the rows of Triangle(x,y,z) or 4Clique(x,y,z,w) (Table 1 with
 * the head variables kept instead of COUNT(*)) over the whole graph, written
 * to a device buffer.
 *   pattern   EH_TRIANGLE (rows of 3 ids) or EH_CLIQUE4 (rows of 4); any
 *             other pattern is EH_EINVAL.
 *   d_out     device buffer of `capacity` rows, uint32, row-major; 4-byte
 *             aligned for triangles, 16-byte aligned for 4-cliques.  Owned by
 *             the caller.  NULL with capacity 0: only the size is computed.
 *   out_n     host; receives the number of rows of the result (equal to
 *             eh_count of the same pattern), also when the buffer is too small.
 * Each triangle (4-clique) is one row holding its vertices' original ids in
 * ascending order; the order of the rows is unspecified.  When the result has
 * more rows than `capacity` the call writes nothing and returns EH_ECAPACITY
 * (size the buffer with eh_count, or with a first call with d_out NULL).  The
 * call synchronises `stream`; whole-graph counts of the same trie wait for it.
 * Temporary device memory: 16 bytes per vertex with |N+(v)| >= 2, plus for
 * 4-cliques whose max out-degree exceeds 512, max out-degree x 4 bytes per
 * resident warp. */
eh_status eh_list(const eh_trie *trie, eh_pattern pattern, const eh_exec_opts *xopts, void *stream,
                  uint32_t *d_out, uint64_t capacity, uint64_t *out_n);

/* Selection queries (Sec. 5.3): a pattern with one attribute bound to a given
 * vertex, on the undirected relation with join semantics (ordered tuples),
 * the selection pushed below the rest of the plan.
 *   EH_SEL_CLIQUE4  S4Clique(x,y,z,w) :- 4Clique(x,y,z,w), P(x,node):
 *                   sum over x in N(node) of the ordered (y,z,w) closing a
 *                   4-clique with x = 6 x (4-cliques containing x), each x's
 *                   4-cliques counted as the triangles of G[N(x)]
 *   EH_SEL_BARBELL  SBarbell(x,y,z,x',y',z') :- triangle(x,y,z), U(x,node),
 *                   V(node,x'), triangle(x',y',z'):
 *                   (sum over x in N(node) of 2 t(x))^2                      */
typedef enum {
    EH_SEL_CLIQUE4 = 0,
    EH_SEL_BARBELL = 1
} eh_sel_pattern;

/* eh_count_selected -- the count of a selection query for the selected vertex
 * `node` (original id; EH_EINVAL if >= n_vertices).  Writes *out_count (host)
 * and synchronises `stream`.  EH_EOVERFLOW above 2^64 - 1.  Serialised with
 * the other synchronous counts of the trie. */
eh_status eh_count_selected(const eh_trie *trie, eh_sel_pattern pattern, uint32_t node, const eh_exec_opts *xopts,
                            void *stream, uint64_t *out_count);

/* eh_trim_memory -- waits for the current device, then returns the device
 * temporaries cached in its default memory pool to the driver. */
eh_status eh_trim_memory(void);

/* eh_trie_export_blocks -- host copy of the composite layout of a trie built
 * with EH_BUILD_BLOCK_LAYOUT (EH_EINVAL otherwise).  *n_blocks and
 * *n_bit_blocks are always written; each array is written when non-NULL:
 *   off    n_vertices + 1 uint64: the directory of pruned set v (trie id) is
 *          entries off[v] .. off[v+1]-1
 *   dir    2 * n_blocks uint32, entry {block id (value / 256), info}: info bit 31
 *          set = bitset block whose 8 words start at words[8 * (info & 0x7FFFFFFF)];
 *          clear = uint block, the run of (info >> 23 & 255) + 1 values starting at
 *          position info & 0x7FFFFF of the set's uint array (eh_trie_export)
 *   words  8 * n_bit_blocks uint32, bit b of word i of a block = value 256 * id + 32 i + b */
eh_status eh_trie_export_blocks(const eh_trie *trie, uint64_t *off, uint32_t *dir, uint32_t *words,
                                uint64_t *n_blocks, uint64_t *n_bit_blocks);

/* eh_count_batch -- not in the paper (a batching pattern of this library;
 * each query is one Table 1 COUNT(*) over an induced subgraph, evaluated as
 * eh_count does).  n_queries independent queries in one persistent launch.
 * Each query's count goes to out_counts[i] and its status to out_status[i]
 * (a failing query does not fail the others; the call returns the first
 * non-OK status, or EH_OK).  subset_pool is a host array of pool_len ids. */
eh_status eh_count_batch(const eh_trie *trie, const eh_query *queries, uint32_t n_queries,
                         const uint32_t *subset_pool, uint64_t pool_len, void *stream, uint64_t *out_counts,
                         eh_status *out_status);

/* eh_count_batch_ex -- as eh_count_batch with explicit knobs; `mode` 0 runs
 * the batch as one persistent launch, 1 runs it one query at a time (the
 * one-launch-per-query baseline, same kernels, same results). */
eh_status eh_count_batch_ex(const eh_trie *trie, const eh_query *queries, uint32_t n_queries,
                            const uint32_t *subset_pool, uint64_t pool_len, const eh_exec_opts *xopts,
                            uint32_t mode, void *stream, uint64_t *out_counts, eh_status *out_status);

/* Where the calling thread's last eh_count_batch / eh_count_batch_ex spent
 * its time, summed over its device batches: prepare = subsets to device,
 * sort, membership bitmaps, induced sub-tries, layouts, work lists (host wall
 * clock, stream synchronised); count = the persistent count launch (a CUDA
 * graph) and the result copy.  graph_reuses = device batches whose count
 * graph was launched by updating the calling thread's executable graph in
 * place instead of instantiating a new one. */
typedef struct {
    uint64_t queries, batches;
    uint64_t sub_vertices;      /* distinct (query, vertex) pairs */
    uint64_t sub_set_elements;  /* padded elements of the induced pruned sets */
    uint64_t heavy_items, light_items;
    double prepare_s, count_s;
    uint64_t graph_reuses;
} eh_batch_profile;

eh_status eh_batch_profile_get(eh_batch_profile *out);

/* eh_trie_stats -- facts of a built trie (host struct, no device work):
 * sizes, max degree and out-degree, how many pruned sets the layout rule of
 * Sec. 4.4 made bitsets, device bytes held, and the density skew of the
 * degree distribution as the paper measures it (Pearson's first skewness
 * coefficient, Sec. 4 footnote).  EH_EINVAL on NULL. */
eh_status eh_trie_stats(const eh_trie *trie, eh_trie_stats_t *out);
/* the same call under its earlier name */
eh_status eh_trie_stats_get(const eh_trie *trie, eh_trie_stats_t *out);

/* eh_trie_export -- copies the trie to host arrays for inspection (tests).
 * Any output pointer may be NULL.  Sizes: new_to_old[n], out_off[n+1]
 * (element offsets into out_nbr, 16-byte aligned sets), out_len[n],
 * out_nbr[out_off[n]], bits_lo[n] (first value covered by the bitset, or
 * 0xFFFFFFFF for uint sets), bits_nwords[n], bits_off[n] (word offsets into
 * out_words), out_words[total bitset words].  `which` 0 = pruned trie N+,
 * 1 = symmetric trie N (no bitsets). */
eh_status eh_trie_export(const eh_trie *trie, uint32_t which, uint32_t *new_to_old, uint64_t *out_off,
                         uint32_t *out_len, uint32_t *out_nbr, uint32_t *bits_lo, uint32_t *bits_nwords,
                         uint64_t *bits_off, uint32_t *out_words);

/* eh_free_trie -- no counterpart in the paper (resource release of this
 * library).  Waits for the device, then releases every array of the trie
 * (NULL is ignored).  Servers created on the trie must be destroyed first. */
void eh_free_trie(eh_trie *trie);

/* eh_test_fail_alloc_after -- failure injection for tests: the n-th device
 * allocation the library makes from now on (n = 0: the next one) fails as if
 * the device were out of memory; n < 0 disarms.  Calls then return
 * EH_ENOMEM and release what they had allocated. */
void eh_test_fail_alloc_after(long long n);

/* eh_selftest_wait_timeout -- runs one kernel that waits, with the bounded
 * wait every count kernel uses for its bulk copies, on a barrier phase that
 * nothing completes.  The wait gives up after limit_us microseconds and the
 * kernel reports it through its status word: the call returns EH_ETIMEOUT
 * (the expected result) and the CUDA context stays usable.  For tests of
 * the failure path; no GPU fault is involved. */
eh_status eh_selftest_wait_timeout(uint32_t limit_us, void *stream);

/* eh_last_error -- no counterpart in the paper (error reporting of this
 * library): the calling thread's message of its last failed call, valid until
 * the thread's next call; never NULL. */
const char *eh_last_error(void);

/* ---------------------------------------------------------------- serving
 * A request loop over a resident trie: submit() admits a query when its
 * estimated device footprint fits the memory budget (else EH_EBUSY), queued
 * queries are batched onto the device as they arrive and slots free up
 * (continuous batching, several batches in flight on separate streams), and
 * poll()/wait() return each query's result. */
typedef struct eh_server eh_server;

typedef struct {
    uint64_t submitted, completed, rejected;
    uint64_t batches;        /* device batches launched */
    uint64_t bytes_in_use;   /* admitted footprint not yet released */
    uint64_t peak_bytes;
    double mean_batch;       /* queries per batch */
} eh_server_stats;

eh_status eh_server_create(const eh_trie *trie, uint64_t memory_budget_bytes, uint32_t max_batch,
                           uint32_t max_inflight, eh_server **out);
/* Copies subset[0..subset_len) and queues the query; *ticket identifies it.
 * EH_EBUSY when the query's estimated device footprint does not fit the
 * budget next to the queries admitted and not yet finished. */
eh_status eh_server_submit(eh_server *s, eh_pattern pattern, const uint32_t *subset, uint32_t subset_len,
                           uint64_t *ticket);
/* *done = 1 when the result is ready (then in *count, *status; results stay
 * available until eh_server_destroy), 0 while pending; EH_EINVAL for an
 * unknown ticket. */
eh_status eh_server_poll(eh_server *s, uint64_t ticket, int *done, uint64_t *count, eh_status *status);
/* Blocks up to timeout_ms (0 = no limit) for the ticket; EH_ETIMEOUT when
 * the limit passes first. */
eh_status eh_server_wait(eh_server *s, uint64_t ticket, uint32_t timeout_ms, uint64_t *count,
                         eh_status *status);
/* Seconds from the ticket's submit() to its result reaching the host
 * (measured by the server; EH_EINVAL while the ticket is not complete). */
eh_status eh_server_latency(eh_server *s, uint64_t ticket, double *seconds);
eh_status eh_server_stats_get(eh_server *s, eh_server_stats *out);
void eh_server_destroy(eh_server *s);

#ifdef __cplusplus
}
#endif
#endif /* EH_H */
