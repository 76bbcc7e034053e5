"""The five benchmark workloads as concrete seeded inputs.

Each function returns a dict with ``n`` (vertex-id space), raw ``src``/``dst``
uint32 arrays and, for the query workloads, subset ``offsets``/``pool``.
Seeds derive from base seed 1503 and the workload number.
"""
from . import BASE_SEED, chunglu, ego_subsets, er, key, rmat

# Raw Chung-Lu pair count giving ~2.0e7 unique non-loop undirected edges
# (calibrated once with the oracle's canonicalisation; the generator itself
# never deduplicates).
CHUNGLU_RAW_PAIRS = 21_200_000


def er_10k_100k(seed=BASE_SEED + 1):
    """Erdos-Renyi G(n=10,000, m=100,000): triangle count, whole graph."""
    src, dst = er(10_000, 100_000, key(seed, 1))
    return {"name": "er_n10000_m100000", "n": 10_000, "src": src, "dst": dst}


def rmat_graph(scale, seed, edge_factor=16, nthreads=None):
    n_edges = edge_factor << scale
    src, dst = rmat(scale, n_edges, key(seed, 2, scale), nthreads=nthreads)
    return {"name": "rmat_s%d_ef%d" % (scale, edge_factor), "n": 1 << scale, "src": src, "dst": dst}


def rmat22(seed=BASE_SEED + 2, nthreads=None):
    """R-MAT scale 22, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05): triangle count."""
    return rmat_graph(22, seed, nthreads=nthreads)


def chunglu_1m(seed=BASE_SEED + 3, nthreads=None, n_pairs=CHUNGLU_RAW_PAIRS):
    """Chung-Lu n=1e6, gamma=2.1, max expected degree 5e4, ~2e7 edges: 4-clique count."""
    src, dst = chunglu(1_000_000, n_pairs, key(seed, 3), nthreads=nthreads)
    return {"name": "chunglu_n1000000_g2.1", "n": 1_000_000, "src": src, "dst": dst}


def rmat20_ego_batch(seed=BASE_SEED + 4, n_queries=4096, nthreads=None):
    """R-MAT scale 20 + 4,096 ego-net subsets, |S| log-uniform in [64, 65536];
    pattern = triangle for even query id, 4-clique for odd."""
    g = rmat_graph(20, seed, nthreads=nthreads)
    off, pool = ego_subsets(g["n"], g["src"], g["dst"], key(seed, 4, 1), n_queries, 0, 64, 65536,
                            nthreads=nthreads)
    g.update({"name": "rmat_s20_ego%d" % n_queries, "offsets": off, "pool": pool,
              "patterns": [q & 1 for q in range(n_queries)]})
    return g


def rmat24_serve(seed=BASE_SEED + 5, n_queries=10000, nthreads=None, lo=100, hi=1_000_000):
    """R-MAT scale 24 resident + ego-net subsets with induced edge counts
    log-uniform in [lo, hi]; patterns uniform over triangle / 4-clique / lollipop."""
    g = rmat_graph(24, seed, nthreads=nthreads)
    off, pool = ego_subsets(g["n"], g["src"], g["dst"], key(seed, 5, 1), n_queries, 1, lo, hi,
                            nthreads=nthreads)
    pats = [int(rng_pattern) for rng_pattern in _patterns(key(seed, 5, 2), n_queries, 3)]
    g.update({"name": "rmat_s24_serve", "offsets": off, "pool": pool, "patterns": pats})
    return g


def _patterns(k, n, m):
    from . import rng
    return [rng(k, i) % m for i in range(n)]
