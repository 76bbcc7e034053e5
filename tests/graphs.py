"""Small named graphs with textbook pattern counts, and brute-force counters.

Brute force works on a dense 0/1 adjacency matrix and shares nothing with the
oracle: triangles = trace(A^3)/6, 4-cliques by enumerating every 4-subset,
lollipops by enumerating every (x,y,z,w) assignment of the join.
"""
import itertools

import numpy as np


def complete(n):
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def complete_multipartite(*parts):
    ids, base = [], 0
    for p in parts:
        ids.append(list(range(base, base + p)))
        base += p
    e = []
    for i in range(len(ids)):
        for j in range(i + 1, len(ids)):
            e += [(a, b) for a in ids[i] for b in ids[j]]
    return base, e


def cycle(n):
    return [(i, (i + 1) % n) for i in range(n)]


def star(n):
    return [(0, i) for i in range(1, n)]


def wheel(n):
    """hub 0 joined to the cycle 1..n"""
    return [(0, i) for i in range(1, n + 1)] + [(i, i % n + 1) for i in range(1, n + 1)]


def petersen():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return outer + spokes + inner


def random_tree(n, rng):
    return [(i, int(rng.integers(0, i))) for i in range(1, n)]


def random_graph(n, p, rng, loops=True, dups=True):
    A = np.triu(rng.random((n, n)) < p, 1)
    e = [(int(i), int(j)) for i, j in zip(*np.nonzero(A))]
    if dups and e:
        e += [e[int(k)][::-1] for k in rng.integers(0, len(e), size=len(e) // 3)]
    if loops:
        e += [(int(v), int(v)) for v in rng.integers(0, n, size=3)]
    rng.shuffle(e)
    return e


def arrays(edges):
    if not edges:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    a = np.array(edges, dtype=np.uint32)
    return a[:, 0].copy(), a[:, 1].copy()


def adjacency(n, edges):
    A = np.zeros((n, n), np.int64)
    for a, b in edges:
        if a != b:
            A[a, b] = A[b, a] = 1
    return A


def bf_triangles(A):
    return int(np.trace(A @ A @ A)) // 6


def bf_vertex_triangles(A):
    return np.diag(A @ A @ A) // 2


def bf_clique4(A):
    n = len(A)
    c = 0
    for q in itertools.combinations(range(n), 4):
        if all(A[i, j] for i, j in itertools.combinations(q, 2)):
            c += 1
    return c


def bf_list(A, k):
    """Every k-clique of the 0/1 matrix A as a sorted tuple, by enumerating
    every k-subset in lexicographic order."""
    n = len(A)
    return [q for q in itertools.combinations(range(n), k)
            if all(A[i, j] for i, j in itertools.combinations(q, 2))]


def bf_lollipop(A):
    """COUNT(*) of R(x,y),S(y,z),T(x,z),U(x,w) over the symmetric relation,
    by enumerating x, y, z, w literally."""
    n = len(A)
    c = 0
    for x in range(n):
        for y in range(n):
            if not A[x, y]:
                continue
            for z in range(n):
                if not (A[y, z] and A[x, z]):
                    continue
                for w in range(n):
                    c += A[x, w]
    return int(c)


def bf_lollipop_distinct(A):
    """Subgraphs triangle {x,y,z} + pendant edge (x,w), w outside the triangle."""
    n = len(A)
    c = 0
    for tri in itertools.combinations(range(n), 3):
        x, y, z = tri
        if not (A[x, y] and A[y, z] and A[x, z]):
            continue
        for v in tri:
            for w in range(n):
                if w not in tri and A[v, w]:
                    c += 1
    return c


def bf_barbell(A):
    """COUNT(*) of the barbell join by enumerating (x, y, z, x', y', z')."""
    n = len(A)
    tri = [[(y, z) for y in range(n) for z in range(n) if A[x, y] and A[y, z] and A[x, z]] for x in range(n)]
    c = 0
    for x in range(n):
        for x2 in range(n):
            if A[x, x2]:
                for _ in tri[x]:
                    for _ in tri[x2]:
                        c += 1
    return c


def bf_sk4(A, node):
    """Ordered (x,y,z,w) with x in N(node) and all six pairs adjacent, by
    enumerating every tuple."""
    n = len(A)
    c = 0
    for x in range(n):
        if not A[node, x]:
            continue
        for y, z, w in itertools.product(range(n), repeat=3):
            if A[x, y] and A[x, z] and A[x, w] and A[y, z] and A[y, w] and A[z, w]:
                c += 1
    return c


def bf_sbarbell(A, node):
    """Ordered (x,y,z,x',y',z'): triangles at x and x', both x, x' in N(node)."""
    n = len(A)
    tri = [sum(1 for y in range(n) for z in range(n) if A[x, y] and A[y, z] and A[x, z]) for x in range(n)]
    c = 0
    for x in range(n):
        for x2 in range(n):
            if A[node, x] and A[node, x2]:
                c += tri[x] * tri[x2]
    return c
