/*
 * eh_oracle.c -- the CPU oracle for pattern COUNT(*) queries by generic join.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  The product path (the
 * CUDA library) never links, loads or calls it, and it shares no code with
 * it: no headers, helpers, tables or generated constants.
 *
 * What it computes, and from which passage of the paper (EmptyHeaded,
 * Aberger et al., SIGMOD'16, arXiv 1503.02368):
 *   - the input relation: dictionary-encoded 32-bit vertex ids (Sec. 2.2),
 *     read as a simple undirected graph: direction ignored, self-loops and
 *     repeated pairs dropped (the reading stated for the synthetic inputs);
 *   - pruning for symmetric queries (Sec. 5.2.1 / App. A.1.2): each undirected
 *     edge is kept once, in the set of its larger endpoint.  The oracle ranks
 *     vertices by their ORIGINAL id (the accelerated path ranks by degree);
 *     counts do not depend on the rank, so agreement also checks that;
 *   - Generic-Join (Algorithm 1), unrolled for the triangle as in the loop
 *     nest of Sec. 3.3.2, for the 4-clique and lollipop of Table 1;
 *   - the lollipop's tail atom U(x,w) aggregated early as the count d(x) of
 *     its w values (the COUNT(*) aggregation of Sec. 3.1, Table 1);
 *   - listing (the same joins with the head variables kept, Table 1 without
 *     COUNT): each triangle or 4-clique written once as a tuple of ids;
 *   - the set-level layout rule of Sec. 4.4 (bitset iff the set's range, in
 *     bits, is at most tau bits per element).
 *
 * Every set intersection is a scalar two-pointer merge: slow and plainly
 * correct.  Counts are uint64 with explicit overflow detection.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* --------------------------------------------------- parallel-for (plain) */

typedef void (*orc_fn)(void *ctx, int64_t i, int tid);
typedef struct { orc_fn fn; void *ctx; int64_t n; int64_t next; } orc_pf;
typedef struct { orc_pf *pf; int tid; } orc_arg;

static void *orc_worker(void *p) {
    orc_arg *a = (orc_arg *)p;
    for (;;) {
        int64_t lo = __atomic_fetch_add(&a->pf->next, 64, __ATOMIC_RELAXED);
        if (lo >= a->pf->n) break;
        int64_t hi = lo + 64 < a->pf->n ? lo + 64 : a->pf->n;
        for (int64_t i = lo; i < hi; ++i) a->pf->fn(a->pf->ctx, i, a->tid);
    }
    return NULL;
}

#define ORC_MAXT 256
static void orc_for(int nthreads, int64_t n, orc_fn fn, void *ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ORC_MAXT) nthreads = ORC_MAXT;
    orc_pf pf = {fn, ctx, n, 0};
    pthread_t th[ORC_MAXT];
    orc_arg args[ORC_MAXT];
    for (int t = 0; t < nthreads; ++t) { args[t].pf = &pf; args[t].tid = t; }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_worker, &args[t]);
    orc_worker(&args[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* per-thread uint64 accumulators with overflow flags, padded apart */
typedef struct { uint64_t sum; int ovf; char pad[52]; } orc_acc;

static uint64_t acc_total(orc_acc *acc, int nthreads, int *overflow) {
    uint64_t s = 0;
    int o = 0;
    for (int t = 0; t < nthreads; ++t) {
        o |= acc[t].ovf;
        if (__builtin_add_overflow(s, acc[t].sum, &s)) o = 1;
    }
    if (overflow) *overflow = o;
    return s;
}

static void acc_add(orc_acc *a, uint64_t x) {
    if (__builtin_add_overflow(a->sum, x, &a->sum)) a->ovf = 1;
}

/* ------------------------------------------------ canonical edge relation */

static int cmp_u64(const void *x, const void *y) {
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return a < b ? -1 : a > b;
}

/* Canonical simple undirected edge set: pairs (a<b), sorted, unique.
 * Returns m, or -1 if an id is >= n (invalid input), -2 on allocation failure. */
int64_t oracle_canon(const uint32_t *src, const uint32_t *dst, uint64_t n_edges, uint32_t n,
                     uint32_t *out_a, uint32_t *out_b) {
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (n_edges ? n_edges : 1));
    if (!key) return -2;
    uint64_t k = 0;
    for (uint64_t i = 0; i < n_edges; ++i) {
        uint32_t s = src[i], t = dst[i];
        if (s >= n || t >= n) { free(key); return -1; }
        if (s == t) continue;
        uint32_t lo = s < t ? s : t, hi = s < t ? t : s;
        key[k++] = ((uint64_t)lo << 32) | hi;
    }
    qsort(key, k, sizeof(uint64_t), cmp_u64);
    int64_t m = 0;
    for (uint64_t i = 0; i < k; ++i) {
        if (i > 0 && key[i] == key[i - 1]) continue;
        out_a[m] = (uint32_t)(key[i] >> 32);
        out_b[m] = (uint32_t)key[i];
        ++m;
    }
    free(key);
    return m;
}

/* ----------------------------------------------------- the graph (a trie)
 * Two-level trie of the symmetric edge relation: level 1 = vertex, level 2 =
 * N(v) sorted ascending (Sec. 2.2, both index orders stored).  Because N(v)
 * is sorted, the pruned set N+(v) = {u in N(v) : u < v} is a prefix of it. */

typedef struct {
    uint32_t n;
    uint64_t m;
    uint64_t *off;    /* n+1 */
    uint32_t *adj;    /* 2m  */
    uint32_t *nless;  /* |N+(v)| */
} oracle_graph;

void *oracle_graph_new(uint32_t n, const uint32_t *a, const uint32_t *b, uint64_t m) {
    oracle_graph *g = (oracle_graph *)calloc(1, sizeof(oracle_graph));
    if (!g) return NULL;
    g->n = n;
    g->m = m;
    g->off = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    g->adj = (uint32_t *)malloc(sizeof(uint32_t) * (2 * m + 1));
    g->nless = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    if (!g->off || !g->adj || !g->nless || !fill) {
        free(g->off); free(g->adj); free(g->nless); free(fill); free(g);
        return NULL;
    }
    for (uint64_t i = 0; i < m; ++i) { g->off[a[i] + 1]++; g->off[b[i] + 1]++; }
    for (uint32_t v = 0; v < n; ++v) g->off[v + 1] += g->off[v];
    memcpy(fill, g->off, sizeof(uint64_t) * ((size_t)n + 1));
    /* edges arrive sorted by (a,b) with a<b: appending b to N(a) and a to N(b)
     * in this order leaves every N(v) sorted ascending (all a < v come first,
     * in increasing a; then all b > v in increasing b). */
    for (uint64_t i = 0; i < m; ++i) g->adj[fill[b[i]]++] = a[i];
    for (uint64_t i = 0; i < m; ++i) g->adj[fill[a[i]]++] = b[i];
    for (uint32_t v = 0; v < n; ++v) {
        uint32_t c = 0;
        for (uint64_t i = g->off[v]; i < g->off[v + 1] && g->adj[i] < v; ++i) ++c;
        g->nless[v] = c;
    }
    free(fill);
    return g;
}

void oracle_graph_free(void *h) {
    oracle_graph *g = (oracle_graph *)h;
    if (!g) return;
    free(g->off); free(g->adj); free(g->nless); free(g);
}

uint32_t oracle_graph_n(void *h) { return ((oracle_graph *)h)->n; }
uint64_t oracle_graph_m(void *h) { return ((oracle_graph *)h)->m; }

/* copies N(v) (sorted) to out; returns d(v) */
uint64_t oracle_neighbours(void *h, uint32_t v, uint32_t *out) {
    oracle_graph *g = (oracle_graph *)h;
    uint64_t d = g->off[v + 1] - g->off[v];
    if (out) memcpy(out, g->adj + g->off[v], sizeof(uint32_t) * d);
    return d;
}

/* the set R[t] of Table 2 for the pruned or the symmetric relation */
static inline const uint32_t *set_of(const oracle_graph *g, uint32_t v, int pruned, uint64_t *len) {
    *len = pruned ? g->nless[v] : g->off[v + 1] - g->off[v];
    return g->adj + g->off[v];
}

/* |xs ∩ ys| by the scalar two-pointer merge */
static uint64_t merge_count(const uint32_t *x, uint64_t nx, const uint32_t *y, uint64_t ny) {
    uint64_t i = 0, j = 0, c = 0;
    while (i < nx && j < ny) {
        if (x[i] < y[j]) ++i;
        else if (x[i] > y[j]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

/* xs ∩ ys materialised (sorted); returns its length */
static uint64_t merge_into(const uint32_t *x, uint64_t nx, const uint32_t *y, uint64_t ny, uint32_t *out) {
    uint64_t i = 0, j = 0, c = 0;
    while (i < nx && j < ny) {
        if (x[i] < y[j]) ++i;
        else if (x[i] > y[j]) ++j;
        else { out[c++] = x[i]; ++i; ++j; }
    }
    return c;
}

/* ------------------------------------------------------------ triangle
 * Loop nest of Sec. 3.3.2 with R = S = T = the (pruned or symmetric) edge
 * relation:  for x; for y in R[x]; count |S[y] ∩ T[x]|.
 * Pruned: each triangle once.  Symmetric: every ordered triple, 6 per
 * triangle (App. A.1.2, the multiple for symmetric data). */

typedef struct { const oracle_graph *g; int pruned; orc_acc *acc; } tri_ctx;

static void tri_one(void *p, int64_t xi, int tid) {
    tri_ctx *c = (tri_ctx *)p;
    uint32_t x = (uint32_t)xi;
    uint64_t nx;
    const uint32_t *Nx = set_of(c->g, x, c->pruned, &nx);
    for (uint64_t i = 0; i < nx; ++i) {
        uint64_t ny;
        const uint32_t *Ny = set_of(c->g, Nx[i], c->pruned, &ny);
        acc_add(&c->acc[tid], merge_count(Nx, nx, Ny, ny));
    }
}

uint64_t oracle_triangles(void *h, int pruned, int nthreads, int *overflow) {
    orc_acc acc[ORC_MAXT];
    memset(acc, 0, sizeof(acc));
    tri_ctx c = {(oracle_graph *)h, pruned, acc};
    orc_for(nthreads, ((oracle_graph *)h)->n, tri_one, &c);
    return acc_total(acc, nthreads < 1 ? 1 : nthreads > ORC_MAXT ? ORC_MAXT : nthreads, overflow);
}

/* The same loop nest restricted to the listed outer vertices x (a sample of
 * the outer loop, used to time the oracle on a bounded share of a large
 * graph).  *edges gets the number of pruned edges (x, y) the sample covers. */
typedef struct { const oracle_graph *g; const uint32_t *verts; orc_acc *acc; orc_acc *edges; } tri_s_ctx;

static void tri_sample_one(void *p, int64_t i, int tid) {
    tri_s_ctx *c = (tri_s_ctx *)p;
    uint32_t x = c->verts[i];
    uint64_t nx;
    const uint32_t *Nx = set_of(c->g, x, 1, &nx);
    acc_add(&c->edges[tid], nx);
    for (uint64_t k = 0; k < nx; ++k) {
        uint64_t ny;
        const uint32_t *Ny = set_of(c->g, Nx[k], 1, &ny);
        acc_add(&c->acc[tid], merge_count(Nx, nx, Ny, ny));
    }
}

uint64_t oracle_triangles_outer(void *h, const uint32_t *verts, uint64_t k, int nthreads, uint64_t *edges,
                                int *overflow) {
    orc_acc acc[ORC_MAXT], ed[ORC_MAXT];
    memset(acc, 0, sizeof(acc));
    memset(ed, 0, sizeof(ed));
    tri_s_ctx c = {(oracle_graph *)h, verts, acc, ed};
    orc_for(nthreads, (int64_t)k, tri_sample_one, &c);
    int nt = nthreads < 1 ? 1 : nthreads > ORC_MAXT ? ORC_MAXT : nthreads;
    if (edges) *edges = acc_total(ed, nt, NULL);
    return acc_total(acc, nt, overflow);
}

/* ------------------------------------------------------------ 4-clique
 * Table 1's 4Clique(x,y,z,w) on the pruned relation, attribute order
 * x > y > z > w (single-node GHD, Sec. 5.2.2): for x; for y in N+(x);
 * S = N+(x) ∩ N+(y) materialised; for z in S: count |S ∩ N+(z)|.
 * Symmetric relation: every ordered 4-tuple, 24 per 4-clique. */

typedef struct { const oracle_graph *g; int pruned; orc_acc *acc; uint32_t **buf; } k4_ctx;

static void k4_one(void *p, int64_t xi, int tid) {
    k4_ctx *c = (k4_ctx *)p;
    uint32_t x = (uint32_t)xi;
    uint64_t nx;
    const uint32_t *Nx = set_of(c->g, x, c->pruned, &nx);
    uint32_t *S = c->buf[tid];
    for (uint64_t i = 0; i < nx; ++i) {
        uint64_t ny;
        const uint32_t *Ny = set_of(c->g, Nx[i], c->pruned, &ny);
        uint64_t ns = merge_into(Nx, nx, Ny, ny, S);
        for (uint64_t k = 0; k < ns; ++k) {
            uint64_t nz;
            const uint32_t *Nz = set_of(c->g, S[k], c->pruned, &nz);
            acc_add(&c->acc[tid], merge_count(S, ns, Nz, nz));
        }
    }
}

uint64_t oracle_clique4(void *h, int pruned, int nthreads, int *overflow) {
    oracle_graph *g = (oracle_graph *)h;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ORC_MAXT) nthreads = ORC_MAXT;
    uint64_t dmax = 0;
    for (uint32_t v = 0; v < g->n; ++v)
        if (g->off[v + 1] - g->off[v] > dmax) dmax = g->off[v + 1] - g->off[v];
    orc_acc acc[ORC_MAXT];
    memset(acc, 0, sizeof(acc));
    uint32_t *buf[ORC_MAXT];
    for (int t = 0; t < nthreads; ++t) buf[t] = (uint32_t *)malloc(sizeof(uint32_t) * (dmax + 1));
    k4_ctx c = {g, pruned, acc, buf};
    orc_for(nthreads, g->n, k4_one, &c);
    for (int t = 0; t < nthreads; ++t) free(buf[t]);
    return acc_total(acc, nthreads, overflow);
}

/* ------------------------------------------------------------ lollipop
 * Table 1's Lollipop(x,y,z,w) :- R(x,y),S(y,z),T(x,z),U(x,w) on the
 * symmetric relation (Sec. 5.2.2 runs it on undirected data), COUNT(*) under
 * join semantics (w is not required to differ from y or z).  Generic-Join
 * with the order x, y, z, w; the innermost attribute w appears only in U, so
 * its loop is the count |U[x]| = d(x), aggregated early:
 *   L = sum_x sum_{y in N(x)} sum_{z in N(x) ∩ N(y)} d(x). */

typedef struct { const oracle_graph *g; orc_acc *acc; int distinct; } lol_ctx;

static void lol_one(void *p, int64_t xi, int tid) {
    lol_ctx *c = (lol_ctx *)p;
    uint32_t x = (uint32_t)xi;
    uint64_t nx;
    const uint32_t *Nx = set_of(c->g, x, 0, &nx);
    for (uint64_t i = 0; i < nx; ++i) {
        uint64_t ny;
        const uint32_t *Ny = set_of(c->g, Nx[i], 0, &ny);
        uint64_t nz = merge_count(Nx, nx, Ny, ny);
        if (!c->distinct) {
            for (uint64_t k = 0; k < nz; ++k) acc_add(&c->acc[tid], nx);
        } else {
            /* distinct form: w outside {y, z}, so d(x) - 2 tails (a triangle
             * at x implies d(x) >= 2); the caller halves for (y,z) vs (z,y) */
            for (uint64_t k = 0; k < nz; ++k) acc_add(&c->acc[tid], nx - 2);
        }
    }
}

uint64_t oracle_lollipop(void *h, int nthreads, int *overflow) {
    orc_acc acc[ORC_MAXT];
    memset(acc, 0, sizeof(acc));
    lol_ctx c = {(oracle_graph *)h, acc, 0};
    orc_for(nthreads, ((oracle_graph *)h)->n, lol_one, &c);
    return acc_total(acc, nthreads < 1 ? 1 : nthreads > ORC_MAXT ? ORC_MAXT : nthreads, overflow);
}

/* Distinct-vertex lollipops counted once per (unordered triangle, x, w):
 * sum over ordered (x,y,z) of (d(x) - 2), halved for the (y,z) symmetry. */
uint64_t oracle_lollipop_distinct(void *h, int nthreads, int *overflow) {
    orc_acc acc[ORC_MAXT];
    memset(acc, 0, sizeof(acc));
    lol_ctx c = {(oracle_graph *)h, acc, 1};
    orc_for(nthreads, ((oracle_graph *)h)->n, lol_one, &c);
    uint64_t s = acc_total(acc, nthreads < 1 ? 1 : nthreads > ORC_MAXT ? ORC_MAXT : nthreads, overflow);
    return s / 2;
}

/* t(x) = number of triangles containing x = (1/2) sum_{y in N(x)} |N(x) ∩ N(y)|,
 * for the listed vertices one by one. */
void oracle_vertex_triangles(void *h, const uint32_t *verts, uint64_t k, uint64_t *out) {
    oracle_graph *g = (oracle_graph *)h;
    for (uint64_t j = 0; j < k; ++j) {
        uint32_t x = verts[j];
        uint64_t nx, s = 0;
        const uint32_t *Nx = set_of(g, x, 0, &nx);
        for (uint64_t i = 0; i < nx; ++i) {
            uint64_t ny;
            const uint32_t *Ny = set_of(g, Nx[i], 0, &ny);
            s += merge_count(Nx, nx, Ny, ny);
        }
        out[j] = s / 2;
    }
}

/* ------------------------------------------------------------- barbell
 * Table 1's Barbell(x,y,z,x',y',z') :- R(x,y),S(y,z),T(x,z),U(x,x'),
 * R'(x',y'),S'(y',z'),T'(x',z') on the symmetric relation, COUNT(*) with join
 * semantics, by the two-node GHD plan of Sec. 3.1 (Fig. barbell GHD): each
 * triangle node is aggregated first (the ordered (y,z) pairs at x number
 * 2 t(x)), then the root node joins U(x,x') on the aggregates:
 *   B = sum_x sum_{x' in N(x)} (2 t(x)) (2 t(x')). */
uint64_t oracle_barbell(void *h, int *overflow) {
    oracle_graph *g = (oracle_graph *)h;
    uint64_t *t = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)g->n + 1));
    uint32_t *all = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)g->n + 1));
    if (!t || !all) { free(t); free(all); if (overflow) *overflow = 1; return 0; }
    for (uint32_t v = 0; v < g->n; ++v) all[v] = v;
    oracle_vertex_triangles(h, all, g->n, t);
    uint64_t b = 0;
    int o = 0;
    for (uint32_t x = 0; x < g->n; ++x) {
        for (uint64_t i = g->off[x]; i < g->off[x + 1]; ++i) {
            uint64_t term;
            if (__builtin_mul_overflow(2 * t[x], 2 * t[g->adj[i]], &term)) o = 1;
            if (__builtin_add_overflow(b, term, &b)) o = 1;
        }
    }
    free(t);
    free(all);
    if (overflow) *overflow = o;
    return b;
}

/* --------------------------------------------------------- listing
 * The same joins with the head variables kept (Table 1's queries without the
 * COUNT aggregation): every match of the innermost level becomes one tuple.
 * The pruned loop nests bind x > y > z (> w) in original ids, so each
 * triangle (4-clique) appears exactly once; it is written with its ids in
 * ascending order, (z, y, x) (and (w, z, y, x)).  Tuples are produced in the
 * loop order.  At most `cap` tuples are written; the return value is the
 * number of tuples of the result. */
uint64_t oracle_list_triangles(void *h, uint32_t *out, uint64_t cap) {
    oracle_graph *g = (oracle_graph *)h;
    uint64_t k = 0;
    for (uint32_t x = 0; x < g->n; ++x) {
        uint64_t nx;
        const uint32_t *Nx = set_of(g, x, 1, &nx);
        for (uint64_t i = 0; i < nx; ++i) {
            const uint32_t y = Nx[i];
            uint64_t ny;
            const uint32_t *Ny = set_of(g, y, 1, &ny);
            uint64_t a = 0, b = 0;   /* two-pointer merge of N+(x) and N+(y) */
            while (a < nx && b < ny) {
                if (Nx[a] < Ny[b]) ++a;
                else if (Nx[a] > Ny[b]) ++b;
                else {
                    if (k < cap) { out[3 * k] = Nx[a]; out[3 * k + 1] = y; out[3 * k + 2] = x; }
                    ++k; ++a; ++b;
                }
            }
        }
    }
    return k;
}

uint64_t oracle_list_clique4(void *h, uint32_t *out, uint64_t cap) {
    oracle_graph *g = (oracle_graph *)h;
    uint64_t dmax = 0, k = 0;
    for (uint32_t v = 0; v < g->n; ++v)
        if (g->nless[v] > dmax) dmax = g->nless[v];
    uint32_t *S = (uint32_t *)malloc(sizeof(uint32_t) * (dmax + 1));
    if (!S) return 0;
    for (uint32_t x = 0; x < g->n; ++x) {
        uint64_t nx;
        const uint32_t *Nx = set_of(g, x, 1, &nx);
        for (uint64_t i = 0; i < nx; ++i) {
            const uint32_t y = Nx[i];
            uint64_t ny;
            const uint32_t *Ny = set_of(g, y, 1, &ny);
            uint64_t ns = merge_into(Nx, nx, Ny, ny, S);
            for (uint64_t j = 0; j < ns; ++j) {
                const uint32_t z = S[j];
                uint64_t nz;
                const uint32_t *Nz = set_of(g, z, 1, &nz);
                uint64_t a = 0, b = 0;   /* S ∩ N+(z) */
                while (a < ns && b < nz) {
                    if (S[a] < Nz[b]) ++a;
                    else if (S[a] > Nz[b]) ++b;
                    else {
                        if (k < cap) {
                            out[4 * k] = S[a]; out[4 * k + 1] = z; out[4 * k + 2] = y; out[4 * k + 3] = x;
                        }
                        ++k; ++a; ++b;
                    }
                }
            }
        }
    }
    free(S);
    return k;
}

/* The triangles containing x, from the symmetric sets: for y in N(x), for
 * z in N(x) ∩ N(y) with y < z, the row of {x, y, z} in ascending order.  At
 * most `cap` rows are written; returns t(x). */
uint64_t oracle_list_triangles_at(void *h, uint32_t x, uint32_t *out, uint64_t cap) {
    oracle_graph *g = (oracle_graph *)h;
    uint64_t nx, k = 0;
    const uint32_t *Nx = set_of(g, x, 0, &nx);
    for (uint64_t i = 0; i < nx; ++i) {
        const uint32_t y = Nx[i];
        uint64_t ny;
        const uint32_t *Ny = set_of(g, y, 0, &ny);
        uint64_t a = 0, b = 0;
        while (a < nx && b < ny) {
            if (Nx[a] < Ny[b]) ++a;
            else if (Nx[a] > Ny[b]) ++b;
            else {
                const uint32_t z = Nx[a];
                if (y < z) {
                    if (k < cap) {
                        uint32_t r0 = x, r1 = y, r2 = z, t;   /* y < z; place x */
                        if (r0 > r1) { t = r0; r0 = r1; r1 = t; }
                        if (r1 > r2) { t = r1; r1 = r2; r2 = t; }
                        out[3 * k] = r0; out[3 * k + 1] = r1; out[3 * k + 2] = r2;
                    }
                    ++k;
                }
                ++a; ++b;
            }
        }
    }
    return k;
}

/* ------------------------------------------------- induced subgraph G[S]
 * The query restricted to a vertex subset: keep the edges whose both ends
 * lie in S (ids keep their meaning; S may be unsorted or repeat ids).
 * Returns a new graph handle, or NULL if an id of S is >= n. */
void *oracle_induced(void *h, const uint32_t *subset, uint64_t len) {
    oracle_graph *g = (oracle_graph *)h;
    uint8_t *in = (uint8_t *)calloc((size_t)g->n + 1, 1);
    if (!in) return NULL;
    for (uint64_t i = 0; i < len; ++i) {
        if (subset[i] >= g->n) { free(in); return NULL; }
        in[subset[i]] = 1;
    }
    uint64_t m = 0;
    for (uint32_t v = 0; v < g->n; ++v)
        if (in[v])
            for (uint64_t i = g->off[v]; i < g->off[v] + g->nless[v]; ++i) m += in[g->adj[i]];
    uint32_t *a = (uint32_t *)malloc(sizeof(uint32_t) * (m + 1));
    uint32_t *b = (uint32_t *)malloc(sizeof(uint32_t) * (m + 1));
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (m + 1));
    uint64_t k = 0;
    for (uint32_t v = 0; v < g->n; ++v)
        if (in[v])
            for (uint64_t i = g->off[v]; i < g->off[v] + g->nless[v]; ++i)
                if (in[g->adj[i]]) key[k++] = ((uint64_t)g->adj[i] << 32) | v;
    qsort(key, k, sizeof(uint64_t), cmp_u64);
    for (uint64_t i = 0; i < k; ++i) { a[i] = (uint32_t)(key[i] >> 32); b[i] = (uint32_t)key[i]; }
    void *r = oracle_graph_new(g->n, a, b, k);
    free(a); free(b); free(key); free(in);
    return r;
}

/* ------------------------------------------------------ layout & order */

/* Set-level layout rule of Sec. 4.4: the bitset layout is chosen when each
 * value costs at most tau bits, i.e. range = max - min + 1 <= tau * |S|.
 * tau = 0 means always uint; tau = UINT32_MAX means always bitset.
 * Returns 1 for bitset, 0 for uint.  `set` is sorted ascending. */
int oracle_layout_is_bitset(const uint32_t *set, uint64_t len, uint32_t tau) {
    if (len == 0 || tau == 0) return 0;
    if (tau == 0xFFFFFFFFu) return 1;
    uint64_t range = (uint64_t)set[len - 1] - set[0] + 1;
    return range <= (uint64_t)tau * len;
}

/* Composite (block-level) layout of Sec. 4.3: the value domain cut into
 * blocks of 256 values; a block holding c values of the set is a 256-bit
 * bitset when 256 <= tau * c (the set-level rule applied to the block's
 * fixed range), else its values stay a uint run.  tau = 0: every block uint;
 * tau = UINT32_MAX: every block bitset.  Writes, per block present (ascending
 * block id = value / 256), its id and kind (1 = bitset); returns the count. */
uint64_t oracle_block_layout(const uint32_t *set, uint64_t len, uint32_t tau, uint32_t *block_id,
                             uint8_t *is_bitset) {
    uint64_t nb = 0, i = 0;
    while (i < len) {
        uint32_t b = set[i] / 256;
        uint64_t c = 0;
        while (i < len && set[i] / 256 == b) { ++c; ++i; }
        block_id[nb] = b;
        is_bitset[nb] = tau == 0xFFFFFFFFu ? 1 : (tau != 0 && (uint64_t)tau * c >= 256);
        ++nb;
    }
    return nb;
}

typedef struct { uint64_t d; uint32_t id; } deg_id;
static int cmp_deg(const void *x, const void *y) {
    const deg_id *a = (const deg_id *)x, *b = (const deg_id *)y;
    if (a->d != b->d) return a->d > b->d ? -1 : 1;
    return a->id < b->id ? -1 : a->id > b->id;
}

/* Degree ordering (App. A.1.1 "Degree"): new id 0 = highest degree, ties by
 * ascending original id.  Writes new_to_old[n]. */
void oracle_degree_order(void *h, uint32_t *new_to_old) {
    oracle_graph *g = (oracle_graph *)h;
    deg_id *t = (deg_id *)malloc(sizeof(deg_id) * ((size_t)g->n + 1));
    for (uint32_t v = 0; v < g->n; ++v) { t[v].d = g->off[v + 1] - g->off[v]; t[v].id = v; }
    qsort(t, g->n, sizeof(deg_id), cmp_deg);
    for (uint32_t i = 0; i < g->n; ++i) new_to_old[i] = t[i].id;
    free(t);
}

/* ---------------------------------------------------- selection queries
 * Sec. 5.3's selection queries on the symmetric relation, join semantics,
 * the selected attribute bound first (a selection pushed down):
 *   kind 0  S4Clique(x,y,z,w) :- 4Clique(x,y,z,w), P(x,node): for x in N(node),
 *           y in N(x), z in N(x) ∩ N(y), w in N(x) ∩ N(y) ∩ N(z): +1
 *   kind 1  SBarbell(x,y,z,x',y',z') :- triangle(x,y,z), U(x,node), V(node,x'),
 *           triangle(x',y',z'): the triangle nodes aggregated to the ordered
 *           (y,z) pairs at x, 2 t(x); then (sum over x in N(node) of 2 t(x))^2 */
uint64_t oracle_count_selected(void *h, int kind, uint32_t node, int *overflow) {
    oracle_graph *g = (oracle_graph *)h;
    int o = 0;
    uint64_t r = 0;
    uint64_t nn;
    const uint32_t *Nn = set_of(g, node, 0, &nn);
    if (kind == 0) {
        uint64_t dmax = 0;
        for (uint32_t v = 0; v < g->n; ++v)
            if (g->off[v + 1] - g->off[v] > dmax) dmax = g->off[v + 1] - g->off[v];
        uint32_t *S = (uint32_t *)malloc(sizeof(uint32_t) * (dmax + 1));
        if (!S) { if (overflow) *overflow = 1; return 0; }
        for (uint64_t a = 0; a < nn; ++a) {
            uint64_t nx;
            const uint32_t *Nx = set_of(g, Nn[a], 0, &nx);
            for (uint64_t b = 0; b < nx; ++b) {
                uint64_t ny;
                const uint32_t *Ny = set_of(g, Nx[b], 0, &ny);
                uint64_t ns = merge_into(Nx, nx, Ny, ny, S);
                for (uint64_t c = 0; c < ns; ++c) {
                    uint64_t nz;
                    const uint32_t *Nz = set_of(g, S[c], 0, &nz);
                    if (__builtin_add_overflow(r, merge_count(S, ns, Nz, nz), &r)) o = 1;
                }
            }
        }
        free(S);
    } else {
        uint64_t *t = (uint64_t *)malloc(sizeof(uint64_t) * (nn + 1));
        if (!t) { if (overflow) *overflow = 1; return 0; }
        oracle_vertex_triangles(h, Nn, nn, t);
        uint64_t half = 0;
        for (uint64_t a = 0; a < nn; ++a)
            if (__builtin_add_overflow(half, 2 * t[a], &half)) o = 1;
        if (__builtin_mul_overflow(half, half, &r)) o = 1;
        free(t);
    }
    if (overflow) *overflow = o;
    return r;
}

/* --------------------------------------------------- node orderings
 * The dictionary orderings of App. "Node Ordering", each straight from its
 * sequential definition.  Writes new_to_old[n] (position -> original id).
 *   0 Degree       degree descending, ties by id
 *   1 Rev-Degree   degree ascending, ties by id
 *   2 Random       by the top 64-b bits of h(v), ties by id (b = bits of n)
 *   3 BFS          FIFO breadth-first search from the first vertex of the
 *                  Degree order, neighbours in ascending id; the vertices it
 *                  does not reach follow in Degree order
 *   4 Strong-Runs  for p in Degree order: label p if unlabelled, then its
 *                  unlabelled neighbours in ascending id
 *   5 Shingle      by the top 64-b bits of min_{w in N(v)} h(w) (all ones
 *                  without neighbours), ties by id
 *   6 Hybrid       the BFS order, stably re-sorted by degree descending
 *   7 Identity
 * h(v) is SplitMix64's output for the counter seed * 2^32 + v. */
static uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t a, b; uint32_t id; } ord_key;
static int cmp_ord(const void *x, const void *y) {
    const ord_key *p = (const ord_key *)x, *q = (const ord_key *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return p->id < q->id ? -1 : p->id > q->id;
}

static void order_by(ord_key *k, uint32_t n, uint32_t *out) {
    qsort(k, n, sizeof(ord_key), cmp_ord);
    for (uint32_t i = 0; i < n; ++i) out[i] = k[i].id;
}

int oracle_vertex_order(void *h, int kind, uint32_t seed, uint32_t *out) {
    oracle_graph *g = (oracle_graph *)h;
    const uint32_t n = g->n;
    int b = 1;
    while (b < 63 && (1ULL << b) < n) ++b;
    ord_key *k = (ord_key *)malloc(sizeof(ord_key) * ((size_t)n + 1));
    uint32_t *deg_order = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint32_t *label = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    if (!k || !deg_order || !label) { free(k); free(deg_order); free(label); return -1; }
    for (uint32_t v = 0; v < n; ++v) {   /* the Degree order, used by several */
        k[v].a = ~0ULL - (g->off[v + 1] - g->off[v]); k[v].b = 0; k[v].id = v;
    }
    order_by(k, n, deg_order);
    uint32_t c = 0;
    switch (kind) {
    case 0:
        memcpy(out, deg_order, sizeof(uint32_t) * n);
        break;
    case 1:
        for (uint32_t v = 0; v < n; ++v) { k[v].a = g->off[v + 1] - g->off[v]; k[v].b = 0; k[v].id = v; }
        order_by(k, n, out);
        break;
    case 2:
        for (uint32_t v = 0; v < n; ++v) {
            k[v].a = splitmix64(((uint64_t)seed << 32) | v) >> b; k[v].b = 0; k[v].id = v;
        }
        order_by(k, n, out);
        break;
    case 3:
    case 6: {
        for (uint32_t v = 0; v < n; ++v) label[v] = 0xFFFFFFFFu;
        if (n) {   /* FIFO queue: out doubles as the queue */
            uint32_t head = 0;
            out[c] = deg_order[0]; label[deg_order[0]] = c++;
            while (head < c) {
                uint32_t p = out[head++];
                for (uint64_t i = g->off[p]; i < g->off[p + 1]; ++i) {
                    uint32_t w = g->adj[i];
                    if (label[w] == 0xFFFFFFFFu) { label[w] = c; out[c++] = w; }
                }
            }
            for (uint32_t i = 0; i < n; ++i)
                if (label[deg_order[i]] == 0xFFFFFFFFu) { label[deg_order[i]] = c; out[c++] = deg_order[i]; }
        }
        if (kind == 6) {   /* stable by degree descending: ties keep their BFS position */
            for (uint32_t v = 0; v < n; ++v) {
                k[v].a = ~0ULL - (g->off[v + 1] - g->off[v]); k[v].b = label[v]; k[v].id = v;
            }
            order_by(k, n, out);
        }
        break;
    }
    case 4:
        for (uint32_t v = 0; v < n; ++v) label[v] = 0;
        for (uint32_t s = 0; s < n; ++s) {
            uint32_t p = deg_order[s];
            if (!label[p]) { label[p] = 1; out[c++] = p; }
            for (uint64_t i = g->off[p]; i < g->off[p + 1]; ++i) {
                uint32_t w = g->adj[i];
                if (!label[w]) { label[w] = 1; out[c++] = w; }
            }
        }
        break;
    case 5:
        for (uint32_t v = 0; v < n; ++v) {
            uint64_t mn = ~0ULL;
            for (uint64_t i = g->off[v]; i < g->off[v + 1]; ++i) {
                uint64_t hw = splitmix64(((uint64_t)seed << 32) | g->adj[i]);
                if (hw < mn) mn = hw;
            }
            k[v].a = mn >> b; k[v].b = 0; k[v].id = v;
        }
        order_by(k, n, out);
        break;
    case 7:
        for (uint32_t v = 0; v < n; ++v) out[v] = v;
        break;
    default:
        free(k); free(deg_order); free(label);
        return -2;
    }
    free(k); free(deg_order); free(label);
    return 0;
}
