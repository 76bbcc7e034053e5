/* Drives every function of the CPU oracle on small graphs, for a build with
 * AddressSanitizer and UndefinedBehaviorSanitizer (tests/test_oracle_asan.py).
 * Checks closed forms along the way; exit status 0 = all good. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int64_t oracle_canon(const uint32_t *, const uint32_t *, uint64_t, uint32_t, uint32_t *, uint32_t *);
void *oracle_graph_new(uint32_t, const uint32_t *, const uint32_t *, uint64_t);
void oracle_graph_free(void *);
uint64_t oracle_neighbours(void *, uint32_t, uint32_t *);
uint64_t oracle_triangles(void *, int, int, int *);
uint64_t oracle_clique4(void *, int, int, int *);
uint64_t oracle_lollipop(void *, int, int *);
uint64_t oracle_lollipop_distinct(void *, int, int *);
void oracle_vertex_triangles(void *, const uint32_t *, uint64_t, uint64_t *);
void *oracle_induced(void *, const uint32_t *, uint64_t);
int oracle_layout_is_bitset(const uint32_t *, uint64_t, uint32_t);
void oracle_degree_order(void *, uint32_t *);
uint64_t oracle_triangles_outer(void *, const uint32_t *, uint64_t, int, uint64_t *, int *);
uint64_t oracle_barbell(void *, int *);

static int fails = 0;
#define CHECK(c)                                                     \
    do {                                                             \
        if (!(c)) { fprintf(stderr, "check failed: %s\n", #c); ++fails; } \
    } while (0)

static void *build(uint32_t n, const uint32_t *s, const uint32_t *d, uint64_t ne) {
    uint32_t *a = malloc(sizeof(uint32_t) * (ne + 1)), *b = malloc(sizeof(uint32_t) * (ne + 1));
    int64_t m = oracle_canon(s, d, ne, n, a, b);
    CHECK(m >= 0);
    void *g = oracle_graph_new(n, a, b, (uint64_t)m);
    free(a);
    free(b);
    return g;
}

int main(void) {
    /* complete graphs */
    for (uint32_t n = 1; n <= 12; ++n) {
        uint64_t ne = (uint64_t)n * (n - 1) / 2, k = 0;
        uint32_t *s = malloc(4 * (ne + 1)), *d = malloc(4 * (ne + 1));
        for (uint32_t i = 0; i < n; ++i)
            for (uint32_t j = i + 1; j < n; ++j) { s[k] = j; d[k] = i; ++k; }
        void *g = build(n, s, d, ne);
        int o = 0;
        uint64_t c3 = (uint64_t)n * (n - 1) * (n - 2) / 6, c4 = n >= 4 ? c3 * (n - 3) / 4 : 0;
        CHECK(oracle_triangles(g, 1, 1, &o) == c3 && !o);
        CHECK(oracle_triangles(g, 0, 3, &o) == 6 * c3);
        CHECK(oracle_clique4(g, 1, 2, &o) == c4);
        CHECK(oracle_clique4(g, 0, 1, &o) == 24 * c4);
        CHECK(n < 3 || oracle_lollipop(g, 2, &o) == (uint64_t)n * (n - 1) * (n - 2) * (n - 1));
        CHECK(oracle_barbell(g, &o) == (uint64_t)n * (n - 1) * (n >= 3 ? (uint64_t)(n - 1) * (n - 2) : 0) *
                                           (n >= 3 ? (uint64_t)(n - 1) * (n - 2) : 0) && !o);
        uint64_t ed = 0;
        uint32_t *all = malloc(4 * (n + 1));
        for (uint32_t i = 0; i < n; ++i) all[i] = i;
        CHECK(oracle_triangles_outer(g, all, n, 2, &ed, &o) == c3 && ed == ne);
        uint64_t *t = malloc(8 * (n + 1));
        oracle_vertex_triangles(g, all, n, t);
        for (uint32_t i = 0; i < n; ++i) CHECK(t[i] == (n >= 3 ? (uint64_t)(n - 1) * (n - 2) / 2 : 0));
        void *h = oracle_induced(g, all, n);
        CHECK(h && oracle_triangles(h, 1, 1, &o) == c3);
        oracle_graph_free(h);
        uint32_t *ord = malloc(4 * (n + 1));
        oracle_degree_order(g, ord);
        for (uint32_t i = 0; i < n; ++i) CHECK(ord[i] == i);
        free(ord); free(t); free(all); free(s); free(d);
        oracle_graph_free(g);
    }
    /* a random multigraph with loops and repeats */
    uint32_t n = 300;
    uint64_t ne = 20000;
    uint32_t *s = malloc(4 * ne), *d = malloc(4 * ne);
    uint64_t x = 88172645463325252ull;
    for (uint64_t i = 0; i < ne; ++i) {
        x ^= x << 13; x ^= x >> 7; x ^= x << 17;
        s[i] = (uint32_t)(x % n);
        d[i] = (uint32_t)((x >> 32) % n);
    }
    void *g = build(n, s, d, ne);
    int o = 0;
    uint64_t t1 = oracle_triangles(g, 1, 1, &o), t4 = oracle_triangles(g, 1, 4, &o);
    CHECK(t1 == t4 && oracle_triangles(g, 0, 2, &o) == 6 * t1);
    CHECK(oracle_clique4(g, 1, 1, &o) == oracle_clique4(g, 1, 5, &o));
    CHECK(oracle_lollipop_distinct(g, 3, &o) <= oracle_lollipop(g, 3, &o));
    uint32_t sub[50];
    for (uint32_t i = 0; i < 50; ++i) sub[i] = (i * 7) % n;
    void *h = oracle_induced(g, sub, 50);
    CHECK(h != NULL);
    CHECK(oracle_triangles(h, 1, 1, &o) <= t1);
    oracle_graph_free(h);
    uint32_t bad[2] = {1, n + 4};
    CHECK(oracle_induced(g, bad, 2) == NULL);
    uint32_t nb[400];
    CHECK(oracle_neighbours(g, 0, nb) <= 400);
    uint32_t set[4] = {0, 1, 2, 3};
    CHECK(oracle_layout_is_bitset(set, 4, 1) && !oracle_layout_is_bitset(set, 4, 0));
    CHECK(!oracle_layout_is_bitset(set, 0, 256));
    uint32_t bs[1] = {0}, bd[1] = {999};
    uint32_t oa[1], ob[1];
    CHECK(oracle_canon(bs, bd, 1, 10, oa, ob) == -1);
    oracle_graph_free(g);
    free(s); free(d);
    /* empty graph */
    void *e = oracle_graph_new(5, NULL, NULL, 0);
    CHECK(oracle_triangles(e, 1, 2, &o) == 0 && oracle_clique4(e, 1, 1, &o) == 0);
    oracle_graph_free(e);
    if (fails) fprintf(stderr, "%d checks failed\n", fails);
    return fails ? 1 : 0;
}
