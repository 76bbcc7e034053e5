/*
 * synth.c -- seeded, counter-based synthetic graph generators.
 *
 * This module produces INPUTS only: raw edge lists (with whatever duplicates,
 * self-loops and direction the generator naturally emits) and vertex subsets
 * (ego networks).  It holds none of the pattern-counting method's arithmetic:
 * no canonicalisation of the edge relation, no ordering, no set layouts, no
 * intersections.  Both the CPU oracle and the CUDA path consume what it emits.
 *
 * Determinism across machines (x86-64 here, aarch64 on the accelerator host):
 *   - every random number is the i-th output of a SplitMix64 stream
 *     (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 *     OOPSLA 2014), so any index can be drawn independently by any thread;
 *   - thresholds and weights are computed with IEEE-754 basic operations only
 *     (+ - * / and exact frexp/ldexp); this file must be compiled with
 *     -ffp-contract=off so that no fused multiply-add changes a rounding.
 *     log/exp below are evaluated from their Taylor / atanh series, never
 *     through the C library, whose last-bit behaviour may differ by platform.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

/* ------------------------------------------------------------------ RNG */

static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
#define SM_GAMMA 0x9E3779B97F4A7C15ULL

/* i-th output of the SplitMix64 stream whose state starts at `key`. */
uint64_t synth_rng(uint64_t key, uint64_t i) { return sm_mix(key + (i + 1) * SM_GAMMA); }

/* A stream key derived from a base seed and two stream labels. */
uint64_t synth_key(uint64_t base, uint64_t a, uint64_t b) {
    return sm_mix(sm_mix(base * SM_GAMMA + a) ^ (b * 0xD1B54A32D192ED03ULL));
}

/* ------------------------------------------- deterministic log / exp */

static double det_log(double x) {            /* x > 0 */
    int e;
    double m = frexp(x, &e);                  /* x = m 2^e, m in [0.5,1) */
    if (m < 0.70710678118654752440) { m *= 2.0; e -= 1; }
    double s = (m - 1.0) / (m + 1.0), s2 = s * s, term = s, sum = 0.0;
    for (int k = 1; k <= 41; k += 2) { sum += term / (double)k; term *= s2; }
    return 2.0 * sum + (double)e * 0.69314718055994530942;
}

static double det_exp(double y) {
    double kf = floor(y / 0.69314718055994530942 + 0.5);
    double r = y - kf * 0.69314718055994530942;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k <= 24; ++k) { term = term * r / (double)k; sum += term; }
    return ldexp(sum, (int)kf);
}

double synth_det_log(double x) { return det_log(x); }
double synth_det_exp(double y) { return det_exp(y); }

/* uniform double in [0,1) from the top 53 bits */
static inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* --------------------------------------------------- tiny parallel-for */

typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi, int tid);
typedef struct { range_fn fn; void *ctx; int64_t n, chunk; int64_t next; int tid; } pf_t;
typedef struct { pf_t *pf; int tid; } pf_arg;

static void *pf_worker(void *p) {
    pf_arg *a = (pf_arg *)p;
    pf_t *pf = a->pf;
    for (;;) {
        int64_t lo = __atomic_fetch_add(&pf->next, pf->chunk, __ATOMIC_RELAXED);
        if (lo >= pf->n) break;
        int64_t hi = lo + pf->chunk < pf->n ? lo + pf->chunk : pf->n;
        pf->fn(pf->ctx, lo, hi, a->tid);
    }
    return NULL;
}

static void par_for(int nthreads, int64_t n, int64_t chunk, range_fn fn, void *ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pf_t pf = {fn, ctx, n, chunk < 1 ? 1 : chunk, 0, 0};
    pthread_t th[256];
    pf_arg args[256];
    for (int t = 0; t < nthreads; ++t) { args[t].pf = &pf; args[t].tid = t; }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, pf_worker, &args[t]);
    pf_worker(&args[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------ Erdos-Renyi G(n, m), exact
 * m distinct unordered pairs: the pair-index space [0, n(n-1)/2) is permuted
 * by a keyed 4-round Feistel bijection on [0, 2^k) with cycle walking, and the
 * first m images are unranked to (a<b).  Each output edge gets a random
 * direction so that consumers see both orientations. */

static uint64_t isqrt_u64(uint64_t x) {
    uint64_t r = (uint64_t)sqrt((double)x);
    while (r * r > x) --r;
    while ((r + 1) * (r + 1) <= x) ++r;
    return r;
}

static uint64_t feistel(uint64_t x, int half_bits, uint64_t key) {
    uint64_t mask = (1ULL << half_bits) - 1, L = x >> half_bits, R = x & mask;
    for (int round = 0; round < 4; ++round) {
        uint64_t F = sm_mix(R ^ synth_rng(key, (uint64_t)round)) & mask;
        uint64_t nL = R, nR = L ^ F;
        L = nL; R = nR;
    }
    return (L << half_bits) | R;
}

int synth_er(uint32_t n, uint64_t m, uint64_t key, uint32_t *src, uint32_t *dst) {
    if (n < 2) return m == 0 ? 0 : 1;
    uint64_t P = (uint64_t)n * (n - 1) / 2;
    if (m > P) return 1;
    int bits = 2;
    while (bits < 64 && (1ULL << bits) < P) bits += 2;
    int half = bits / 2;
    uint64_t fkey = synth_rng(key, 0xFE15);
    for (uint64_t i = 0; i < m; ++i) {
        uint64_t x = i;
        do { x = feistel(x, half, fkey); } while (x >= P);
        /* unrank x -> (a,b), a<b, x = b(b-1)/2 + a */
        uint64_t b = (1 + isqrt_u64(1 + 8 * x)) / 2;
        while (b * (b - 1) / 2 > x) --b;
        while ((b + 1) * b / 2 <= x) ++b;
        uint64_t a = x - b * (b - 1) / 2;
        if (synth_rng(key, i) & 1) { src[i] = (uint32_t)a; dst[i] = (uint32_t)b; }
        else { src[i] = (uint32_t)b; dst[i] = (uint32_t)a; }
    }
    return 0;
}

/* ------------------------------------------------------------ R-MAT
 * Chakrabarti, Zhan, Faloutsos, "R-MAT: A Recursive Model for Graph Mining",
 * SDM 2004.  Edge i descends `scale` levels; at each level a 32-bit uniform
 * draw selects one of the four quadrants with probabilities (a, b, c, d),
 * no noise.  Output keeps the generated direction, duplicates and loops. */

typedef struct { uint32_t scale; uint64_t key; uint32_t ta, tab, tabc; uint32_t *src, *dst; } rmat_ctx;

static void rmat_range(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    rmat_ctx *c = (rmat_ctx *)p;
    uint32_t draws = (c->scale + 1) / 2;
    for (int64_t i = lo; i < hi; ++i) {
        uint32_t s = 0, t = 0;
        for (uint32_t l = 0; l < c->scale; ++l) {
            uint64_t r64 = synth_rng(c->key, (uint64_t)i * draws + l / 2);
            uint32_t r = (l & 1) ? (uint32_t)(r64 >> 32) : (uint32_t)r64;
            uint32_t q = r < c->ta ? 0u : r < c->tab ? 1u : r < c->tabc ? 2u : 3u;
            s = (s << 1) | (q >> 1);
            t = (t << 1) | (q & 1);
        }
        c->src[i] = s;
        c->dst[i] = t;
    }
}

static uint32_t prob_threshold(double p) {
    double t = p * 4294967296.0;
    if (t >= 4294967295.0) return 4294967295u;
    if (t <= 0) return 0;
    return (uint32_t)t;
}

int synth_rmat(uint32_t scale, uint64_t n_edges, double a, double b, double c, uint64_t key,
               uint32_t *src, uint32_t *dst, int nthreads) {
    if (scale == 0 || scale > 31) return 1;
    rmat_ctx ctx = {scale, key, prob_threshold(a), prob_threshold(a + b), prob_threshold(a + b + c), src, dst};
    par_for(nthreads, (int64_t)n_edges, 1 << 16, rmat_range, &ctx);
    return 0;
}

/* ---------------------------------------------------------- Chung-Lu
 * Chung, Lu, "Connected components in random graphs with given expected
 * degree sequences", 2002.  Expected weights w_i = c (i + i0)^(-1/(gamma-1)),
 * i = 0..n-1; both endpoints of each of `n_pairs` raw pairs are drawn
 * independently with probability proportional to w (inverse-CDF search on
 * integer cumulative weights).  Loops and repeats are kept in the output. */

typedef struct { uint64_t *cum; uint32_t n; uint64_t total, key; uint32_t *src, *dst; } cl_ctx;

static inline uint32_t cl_pick(const cl_ctx *c, uint64_t r) {
    uint64_t x = (uint64_t)(((unsigned __int128)r * c->total) >> 64); /* in [0,total) */
    uint32_t lo = 0, hi = c->n - 1;                                  /* first i with cum[i] > x */
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (c->cum[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static void cl_range(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    cl_ctx *c = (cl_ctx *)p;
    for (int64_t i = lo; i < hi; ++i) {
        c->src[i] = cl_pick(c, synth_rng(c->key, 2 * (uint64_t)i));
        c->dst[i] = cl_pick(c, synth_rng(c->key, 2 * (uint64_t)i + 1));
    }
}

int synth_chunglu(uint32_t n, double gamma, double i0, double wmax, uint64_t n_pairs, uint64_t key,
                  uint32_t *src, uint32_t *dst, int nthreads) {
    if (n == 0 || gamma <= 1.0 || i0 <= 0) return 1;
    double beta = 1.0 / (gamma - 1.0);
    double cst = wmax * det_exp(beta * det_log(i0));
    uint64_t *cum = (uint64_t *)malloc(sizeof(uint64_t) * n);
    if (!cum) return 2;
    uint64_t acc = 0;
    for (uint32_t i = 0; i < n; ++i) {
        double w = cst * det_exp(-beta * det_log((double)i + i0));
        acc += (uint64_t)(w * 65536.0) + 1;
        cum[i] = acc;
    }
    cl_ctx ctx = {cum, n, acc, key, src, dst};
    par_for(nthreads, (int64_t)n_pairs, 1 << 15, cl_range, &ctx);
    free(cum);
    return 0;
}

/* weights as the generator uses them (for tests of the recipe) */
double synth_chunglu_weight(uint32_t i, double gamma, double i0, double wmax) {
    double beta = 1.0 / (gamma - 1.0);
    double cst = wmax * det_exp(beta * det_log(i0));
    return cst * det_exp(-beta * det_log((double)i + i0));
}

/* ------------------------------------------------------- ego networks
 * Vertex subsets of a raw edge list.  The adjacency built here is only a BFS
 * aid for the generator (simple, undirected, neighbours in ascending id).
 * Query q: a seed vertex uniform over vertices with at least one neighbour;
 * breadth-first search visiting neighbours in ascending id; the subset is the
 * first `target` vertices reached (mode 0: target vertex count), or the
 * shortest BFS prefix whose induced edge count reaches `target` (mode 1).
 * target = floor(lo * (hi/lo)^U), U uniform in [0,1).  A component smaller
 * than the target yields the whole component.  Output is in BFS order. */

typedef struct {
    uint32_t n;
    uint64_t *off;
    uint32_t *adj;
} synth_graph;

static int cmp_u32(const void *x, const void *y) {
    uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
    return a < b ? -1 : a > b;
}

typedef struct { uint32_t n; const uint32_t *src, *dst; uint64_t *slot; uint32_t *adj; } edge_ctx;

static void edge_count_range(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    edge_ctx *c = (edge_ctx *)p;
    for (int64_t i = lo; i < hi; ++i) {
        uint32_t s = c->src[i], t = c->dst[i];
        if (s == t || s >= c->n || t >= c->n) continue;
        __atomic_fetch_add(&c->slot[s], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&c->slot[t], 1, __ATOMIC_RELAXED);
    }
}

static void edge_fill_range(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    edge_ctx *c = (edge_ctx *)p;
    for (int64_t i = lo; i < hi; ++i) {
        uint32_t s = c->src[i], t = c->dst[i];
        if (s == t || s >= c->n || t >= c->n) continue;
        c->adj[__atomic_fetch_add(&c->slot[s], 1, __ATOMIC_RELAXED)] = t;
        c->adj[__atomic_fetch_add(&c->slot[t], 1, __ATOMIC_RELAXED)] = s;
    }
}

typedef struct { uint64_t *off; uint32_t *adj; uint64_t *len; } sortlist_ctx;

/* sorts the lists of vertices [lo, hi) in place and drops repeats; the new
 * length of each list goes to len[v] */
static void sortlist_range(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    sortlist_ctx *c = (sortlist_ctx *)p;
    for (int64_t v = lo; v < hi; ++v) {
        uint64_t b = c->off[v], e = c->off[v + 1], w = b;
        qsort(c->adj + b, e - b, sizeof(uint32_t), cmp_u32);
        for (uint64_t i = b; i < e; ++i)
            if (i == b || c->adj[i] != c->adj[i - 1]) c->adj[w++] = c->adj[i];
        c->len[v] = w - b;
    }
}

void *synth_graph_new(uint32_t n, const uint32_t *src, const uint32_t *dst, uint64_t n_edges, int nthreads) {
    synth_graph *g = (synth_graph *)calloc(1, sizeof(synth_graph));
    if (!g) return NULL;
    g->n = n;
    g->off = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint64_t *fill = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!g->off || !fill) { free(g->off); free(fill); free(g); return NULL; }
    /* list lengths, then each edge placed into both lists (atomic slots, so
     * the order inside a list depends on the threads; the sort below fixes it) */
    edge_ctx ec = {n, src, dst, g->off + 1, NULL};
    par_for(nthreads, (int64_t)n_edges, 1 << 16, edge_count_range, &ec);
    for (uint32_t v = 0; v < n; ++v) g->off[v + 1] += g->off[v];
    g->adj = (uint32_t *)malloc(sizeof(uint32_t) * (g->off[n] ? g->off[n] : 1));
    if (!g->adj) { free(g->off); free(fill); free(g); return NULL; }
    memcpy(fill, g->off, sizeof(uint64_t) * ((size_t)n + 1));
    ec.slot = fill;
    ec.adj = g->adj;
    par_for(nthreads, (int64_t)n_edges, 1 << 16, edge_fill_range, &ec);
    /* sort each list ascending and drop repeats (in parallel over vertices,
     * `fill` then holds each list's new length), then repack */
    sortlist_ctx sc = {g->off, g->adj, fill};
    par_for(nthreads, (int64_t)n, 4096, sortlist_range, &sc);
    uint64_t w = 0;
    for (uint32_t v = 0; v < n; ++v) {
        uint64_t b = g->off[v], len = fill[v];
        if (w != b) memmove(g->adj + w, g->adj + b, sizeof(uint32_t) * len);
        g->off[v] = w;
        w += len;
    }
    g->off[n] = w;
    free(fill);
    return g;
}

void synth_graph_free(void *h) {
    synth_graph *g = (synth_graph *)h;
    if (!g) return;
    free(g->off); free(g->adj); free(g);
}

uint64_t synth_graph_degree(void *h, uint32_t v) {
    synth_graph *g = (synth_graph *)h;
    return g->off[v + 1] - g->off[v];
}

typedef struct {
    synth_graph *g; uint64_t key; int mode; double lo, hi;
    uint32_t **res; uint32_t *len;
    uint32_t **mark; uint32_t **queue;   /* per thread */
} ego_ctx;

static void ego_one(ego_ctx *c, uint32_t q, int tid) {
    synth_graph *g = c->g;
    uint32_t *mark = c->mark[tid], *queue = c->queue[tid];
    uint32_t stamp = q + 1;
    uint64_t ctr = 0;
    uint32_t seed;
    for (;;) {
        seed = (uint32_t)(synth_rng(c->key, ((uint64_t)q << 20) + ctr++) % g->n);
        if (g->off[seed + 1] > g->off[seed]) break;
    }
    double U = u01(synth_rng(c->key, ((uint64_t)q << 20) | 0xFFFFF));
    double target = floor(c->lo * det_exp(U * det_log(c->hi / c->lo)));
    uint64_t induced = 0;
    uint32_t head = 0, tail = 0;
    queue[tail++] = seed;
    mark[seed] = stamp;
    /* mode 0: stop at `target` vertices; mode 1: stop once induced edges >= target */
    uint32_t taken = 0;
    while (head < tail) {
        uint32_t v = queue[head++];
        ++taken;
        if (c->mode == 1) {
            /* v joins the subset: its edges to earlier members become induced */
            for (uint64_t i = g->off[v]; i < g->off[v + 1]; ++i) {
                uint32_t w = g->adj[i];
                if (mark[w] == stamp + 0x80000000u) ++induced;
            }
            mark[v] = stamp + 0x80000000u;
            if ((double)induced >= target) break;
        } else if ((double)taken >= target) break;
        for (uint64_t i = g->off[v]; i < g->off[v + 1]; ++i) {
            uint32_t w = g->adj[i];
            if (mark[w] != stamp && mark[w] != stamp + 0x80000000u) { mark[w] = stamp; queue[tail++] = w; }
        }
    }
    c->len[q] = taken;
    c->res[q] = (uint32_t *)malloc(sizeof(uint32_t) * (taken ? taken : 1));
    memcpy(c->res[q], queue, sizeof(uint32_t) * taken);
}

static void ego_range(void *p, int64_t lo, int64_t hi, int tid) {
    ego_ctx *c = (ego_ctx *)p;
    for (int64_t q = lo; q < hi; ++q) ego_one(c, (uint32_t)q, tid);
}

typedef struct { uint32_t nq; uint32_t **res; uint32_t *len; } ego_result;

/* Generates `nq` subsets; returns a result handle and writes offsets
 * (nq+1 entries, prefix sums of the subset lengths). */
void *synth_ego_batch(void *h, uint64_t key, uint32_t nq, int mode, double lo, double hi, int nthreads,
                      uint64_t *out_off) {
    synth_graph *g = (synth_graph *)h;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    ego_ctx c = {g, key, mode, lo, hi, NULL, NULL, NULL, NULL};
    c.res = (uint32_t **)calloc(nq ? nq : 1, sizeof(uint32_t *));
    c.len = (uint32_t *)calloc(nq ? nq : 1, sizeof(uint32_t));
    c.mark = (uint32_t **)calloc((size_t)nthreads, sizeof(uint32_t *));
    c.queue = (uint32_t **)calloc((size_t)nthreads, sizeof(uint32_t *));
    for (int t = 0; t < nthreads; ++t) {
        c.mark[t] = (uint32_t *)calloc(g->n, sizeof(uint32_t));
        c.queue[t] = (uint32_t *)malloc(sizeof(uint32_t) * g->n);
    }
    par_for(nthreads, nq, 1, ego_range, &c);
    for (int t = 0; t < nthreads; ++t) { free(c.mark[t]); free(c.queue[t]); }
    free(c.mark); free(c.queue);
    out_off[0] = 0;
    for (uint32_t q = 0; q < nq; ++q) out_off[q + 1] = out_off[q] + c.len[q];
    ego_result *r = (ego_result *)malloc(sizeof(ego_result));
    r->nq = nq; r->res = c.res; r->len = c.len;
    return r;
}

void synth_ego_fetch(void *rh, uint32_t *pool) {
    ego_result *r = (ego_result *)rh;
    uint64_t w = 0;
    for (uint32_t q = 0; q < r->nq; ++q) {
        memcpy(pool + w, r->res[q], sizeof(uint32_t) * r->len[q]);
        w += r->len[q];
    }
}

void synth_ego_free(void *rh) {
    ego_result *r = (ego_result *)rh;
    if (!r) return;
    for (uint32_t q = 0; q < r->nq; ++q) free(r->res[q]);
    free(r->res); free(r->len); free(r);
}
