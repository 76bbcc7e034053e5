// order.cu -- the node orderings of the dictionary encoding (Sec. 2.2's
// dictionary IDs; the orderings of App. "Node Ordering"), computed on the
// device as a permutation new2old of the vertex ids.
//
// Every ordering is defined so that it can be computed in parallel and still
// equals a plain sequential definition (the oracle's):
//   DEGREE       degree descending, ties by original id
//   REV_DEGREE   degree ascending, ties by original id
//   RANDOM       by h(v) = splitmix64(seed * 2^32 + v), ties by id
//   IDENTITY     the original ids
//   BFS          breadth-first order from the highest-degree vertex (ties by
//                id), neighbours visited in ascending id; the vertices it does
//                not reach follow in DEGREE order.  Level by level on the
//                device: a vertex of the next level takes its position from
//                (position of its first discoverer, id), which is exactly the
//                order a FIFO queue gives.
//   STRONG_RUNS  vertices taken in DEGREE order; each one, when reached, first
//                labels itself if unlabelled, then its unlabelled neighbours in
//                ascending id.  Vertex v is labelled at step
//                s(v) = min(r(v), min over neighbours w of r(w)) (r = DEGREE
//                rank), before or after the others of that step according to
//                whether v is the step's own vertex, then by id.
//   SHINGLE      by the min-hash shingle min over neighbours w of h(w) (the
//                neighbourhood-similarity ordering), ties by id; vertices
//                without neighbours last
//   HYBRID       BFS positions, then a stable sort by degree descending: equal
//                degrees keep their BFS order (the paper's proposal).
#include "eh_internal.cuh"

#include <algorithm>

namespace {

constexpr uint32_t UNSEEN = 0xFFFFFFFFu;

// SplitMix64 (Steele, Lea, Flood 2014), one output for a counter value
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t vhash(uint32_t seed, uint32_t v) { return mix64(((uint64_t)seed << 32) | v); }

__global__ void k_keys_degree(const uint32_t *__restrict__ deg, uint32_t n, uint32_t maxdeg, int nb, int rev,
                              uint64_t *keys) {
    uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const uint64_t d = rev ? deg[v] : maxdeg - deg[v];
    keys[v] = (d << nb) | v;
}

__global__ void k_keys_random(uint32_t n, uint32_t seed, int nb, uint64_t *keys) {
    uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    keys[v] = ((vhash(seed, (uint32_t)v) >> nb) << nb) | v;
}

__global__ void k_low_bits(const uint64_t *__restrict__ keys, uint32_t n, int nb, uint32_t *out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint32_t)(keys[i] & ((1ull << nb) - 1));
}

__global__ void k_iota(uint32_t n, uint32_t *out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint32_t)i;
}

__global__ void k_rank_of(const uint32_t *__restrict__ order, uint32_t n, uint32_t *rank) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rank[order[i]] = (uint32_t)i;
}

// both directions of every unique pair (lo << nb | hi), original ids
__global__ void k_sym_keys(const uint64_t *__restrict__ ukeys, uint64_t m, int nb, uint64_t *dk) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint64_t k = ukeys[i], mask = (1ull << nb) - 1;
    dk[2 * i] = k;
    dk[2 * i + 1] = ((k & mask) << nb) | (k >> nb);
}

__global__ void k_widen(const uint32_t *__restrict__ x, uint32_t n, uint64_t *out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = x[i];
}

// min-hash shingle of each vertex's neighbourhood; one warp per vertex
__global__ void k_keys_shingle(const uint64_t *__restrict__ off, const uint64_t *__restrict__ adj, uint32_t n,
                               uint32_t seed, int nb, uint64_t *keys) {
    const uint32_t v = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (v >= n) return;
    const uint64_t mask = (1ull << nb) - 1;
    uint64_t mn = ~0ull;
    for (uint64_t i = off[v] + lane; i < off[v + 1]; i += 32) mn = min(mn, vhash(seed, (uint32_t)(adj[i] & mask)));
    for (int d = 16; d > 0; d >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, d));
    if (lane == 0) keys[v] = ((mn >> nb) << nb) | v;
}

// strong runs: s(v) = min(r(v), min_{w in N(v)} r(w)); key (s, v != order[s], v)
__global__ void k_keys_strong(const uint64_t *__restrict__ off, const uint64_t *__restrict__ adj,
                              const uint32_t *__restrict__ rank, const uint32_t *__restrict__ deg_order, uint32_t n,
                              int nb, uint64_t *keys) {
    const uint32_t v = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (v >= n) return;
    const uint64_t mask = (1ull << nb) - 1;
    uint32_t s = rank[v];
    for (uint64_t i = off[v] + lane; i < off[v + 1]; i += 32) s = min(s, rank[(uint32_t)(adj[i] & mask)]);
    for (int d = 16; d > 0; d >>= 1) s = min(s, __shfl_xor_sync(0xffffffffu, s, d));
    if (lane == 0) keys[v] = ((uint64_t)s << (nb + 1)) | ((uint64_t)(deg_order[s] != v) << nb) | v;
}

// BFS: one warp per frontier vertex (global position base + f); a newly seen
// neighbour keeps the smallest discoverer position and is listed once
__global__ void k_bfs_expand(const uint32_t *__restrict__ frontier, uint32_t nf, uint32_t base,
                             const uint64_t *__restrict__ off, const uint64_t *__restrict__ adj, int nb,
                             const uint32_t *__restrict__ pos, uint32_t *cand, uint32_t *next, uint32_t *n_next) {
    const uint32_t f = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (f >= nf) return;
    const uint32_t p = frontier[f], P = base + f;
    const uint64_t mask = (1ull << nb) - 1;
    for (uint64_t i = off[p] + lane; i < off[p + 1]; i += 32) {
        const uint32_t w = (uint32_t)(adj[i] & mask);
        if (pos[w] != UNSEEN) continue;
        if (atomicMin(&cand[w], P) == UNSEEN) next[atomicAdd(n_next, 1u)] = w;
    }
}

__global__ void k_bfs_keys(const uint32_t *__restrict__ next, uint32_t c, const uint32_t *__restrict__ cand, int nb,
                           uint64_t *keys) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < c) keys[i] = ((uint64_t)cand[next[i]] << nb) | next[i];
}

__global__ void k_bfs_assign(const uint64_t *__restrict__ keys, uint32_t c, uint32_t base, int nb, uint32_t *pos,
                             uint32_t *order, uint32_t *frontier) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c) return;
    const uint32_t w = (uint32_t)(keys[i] & ((1ull << nb) - 1));
    pos[w] = base + (uint32_t)i;
    order[base + i] = w;
    frontier[i] = w;
}

__global__ void k_unseen_flags(const uint32_t *__restrict__ deg_order, uint32_t n, const uint32_t *__restrict__ pos,
                               uint32_t *flags) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = pos[deg_order[i]] == UNSEEN ? 1u : 0u;
}

__global__ void k_tail(const uint32_t *__restrict__ deg_order, const uint32_t *__restrict__ flags,
                       const uint32_t *__restrict__ fpos, uint32_t n, uint32_t base, uint32_t *pos, uint32_t *order) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flags[i]) return;
    const uint32_t v = deg_order[i];
    pos[v] = base + fpos[i];
    order[base + fpos[i]] = v;
}

__global__ void k_keys_hybrid(const uint32_t *__restrict__ deg, const uint32_t *__restrict__ pos, uint32_t n,
                              uint32_t maxdeg, int nb, uint64_t *keys) {
    uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) keys[v] = ((uint64_t)(maxdeg - deg[v]) << nb) | pos[v];
}

__global__ void k_gather(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ bfs_order, uint32_t n, int nb,
                         uint32_t *out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = bfs_order[(uint32_t)(keys[i] & ((1ull << nb) - 1))];
}

struct Scratch {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <typename T>
    eh_status alloc(T **p, uint64_t count) {
        eh_status st = dev_alloc(p, count, s);
        if (st == EH_OK) ptrs.push_back((void *)*p);
        return st;
    }
    ~Scratch() {
        for (void *q : ptrs) cudaFreeAsync(q, s);
    }
};

// keys (ending in the id in the low nb bits) sorted on key_bits -> order
eh_status sort_to_order(uint64_t **keys, uint64_t **tmp, uint32_t n, int key_bits, int nb, cudaStream_t s,
                        uint32_t *order) {
    if (!n) return EH_OK;
    EH_TRY(dev_radix_sort_u64(keys, tmp, n, std::min(64, key_bits), s));
    k_low_bits<<<blocks_for(n), 256, 0, s>>>(*keys, n, nb, order);
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}

// symmetric adjacency in original ids: off[n+1], adj[2m] (sorted keys v << nb | w)
eh_status old_csr(const uint64_t *ukeys, uint64_t m, uint32_t n, int nb, const uint32_t *deg, cudaStream_t s,
                  Scratch &sc, uint64_t **off, uint64_t **adj) {
    uint64_t *dk = nullptr, *dk2 = nullptr, *wide = nullptr;
    EH_TRY(sc.alloc(&dk, 2 * m));
    EH_TRY(sc.alloc(&dk2, 2 * m));
    EH_TRY(sc.alloc(&wide, (uint64_t)n + 1));
    EH_TRY(sc.alloc(off, (uint64_t)n + 1));
    if (m) k_sym_keys<<<blocks_for(m), 256, 0, s>>>(ukeys, m, nb, dk);
    if (m) EH_TRY(dev_radix_sort_u64(&dk, &dk2, 2 * m, 2 * nb, s));
    EH_CUDA_TRY(cudaMemsetAsync(wide, 0, ((uint64_t)n + 1) * 8, s));
    if (n) k_widen<<<blocks_for(n), 256, 0, s>>>(deg, n, wide);
    EH_TRY(dev_exclusive_scan_u64(wide, *off, (uint64_t)n + 1, s, nullptr));
    *adj = dk;   // entry i of the sorted keys is the i-th directed edge: its low bits are the neighbour
    return EH_OK;
}

eh_status bfs_order(const uint64_t *off, const uint64_t *adj, uint32_t n, int nb, const uint32_t *deg_order,
                    cudaStream_t s, Scratch &sc, uint32_t *order, uint32_t *pos) {
    uint32_t *cand = nullptr, *front = nullptr, *next = nullptr, *cnt = nullptr, *flags = nullptr, *fpos = nullptr;
    uint64_t *keys = nullptr, *keys2 = nullptr;
    EH_TRY(sc.alloc(&cand, n));
    EH_TRY(sc.alloc(&front, n));
    EH_TRY(sc.alloc(&next, n));
    EH_TRY(sc.alloc(&cnt, 1));
    EH_TRY(sc.alloc(&keys, n));
    EH_TRY(sc.alloc(&keys2, n));
    EH_CUDA_TRY(cudaMemsetAsync(pos, 0xFF, (uint64_t)n * 4, s));
    EH_CUDA_TRY(cudaMemsetAsync(cand, 0xFF, (uint64_t)n * 4, s));
    // root: the first vertex of the degree order
    uint32_t root = 0, zero = 0;
    EH_CUDA_TRY(cudaMemcpyAsync(&root, deg_order, 4, cudaMemcpyDeviceToHost, s));
    EH_CUDA_TRY(cudaStreamSynchronize(s));
    EH_CUDA_TRY(cudaMemcpyAsync(pos + root, &zero, 4, cudaMemcpyHostToDevice, s));
    EH_CUDA_TRY(cudaMemcpyAsync(order, &root, 4, cudaMemcpyHostToDevice, s));
    EH_CUDA_TRY(cudaMemcpyAsync(front, &root, 4, cudaMemcpyHostToDevice, s));
    uint32_t nf = 1, base = 0;
    while (nf) {
        EH_CUDA_TRY(cudaMemsetAsync(cnt, 0, 4, s));
        k_bfs_expand<<<blocks_for(nf, 8), 256, 0, s>>>(front, nf, base, off, adj, nb, pos, cand, next, cnt);
        uint32_t c = 0;
        EH_CUDA_TRY(cudaMemcpyAsync(&c, cnt, 4, cudaMemcpyDeviceToHost, s));
        EH_CUDA_TRY(cudaStreamSynchronize(s));
        base += nf;
        if (!c) break;
        k_bfs_keys<<<blocks_for(c), 256, 0, s>>>(next, c, cand, nb, keys);
        uint64_t *k = keys, *k2 = keys2;
        EH_TRY(dev_radix_sort_u64(&k, &k2, c, 2 * nb, s));
        k_bfs_assign<<<blocks_for(c), 256, 0, s>>>(k, c, base, nb, pos, order, front);
        EH_CUDA_TRY(cudaGetLastError());
        nf = c;
    }
    // the vertices the search did not reach, in degree order
    if (base < n) {
        EH_TRY(sc.alloc(&flags, n));
        EH_TRY(sc.alloc(&fpos, n));
        k_unseen_flags<<<blocks_for(n), 256, 0, s>>>(deg_order, n, pos, flags);
        EH_TRY(dev_exclusive_scan_u32(flags, fpos, n, s, nullptr));
        k_tail<<<blocks_for(n), 256, 0, s>>>(deg_order, flags, fpos, n, base, pos, order);
    }
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}

}  // namespace

eh_status eh_vertex_order(uint32_t ordering, uint32_t seed, const uint64_t *ukeys, uint64_t m, uint32_t n, int nb,
                          const uint32_t *deg, uint32_t maxdeg, cudaStream_t s, uint32_t *new2old) {
    if (!n) return EH_OK;
    Scratch sc(s);
    uint64_t *keys = nullptr, *keys2 = nullptr;
    EH_TRY(sc.alloc(&keys, n));
    EH_TRY(sc.alloc(&keys2, n));
    const int db = bits_for((uint64_t)maxdeg + 1);
    switch (ordering) {
        case EH_ORDER_DEGREE:
        case EH_ORDER_REV_DEGREE:
            k_keys_degree<<<blocks_for(n), 256, 0, s>>>(deg, n, maxdeg, nb, ordering == EH_ORDER_REV_DEGREE, keys);
            return sort_to_order(&keys, &keys2, n, nb + db, nb, s, new2old);
        case EH_ORDER_RANDOM:
            k_keys_random<<<blocks_for(n), 256, 0, s>>>(n, seed, nb, keys);
            return sort_to_order(&keys, &keys2, n, 64, nb, s, new2old);
        case EH_ORDER_IDENTITY:
            k_iota<<<blocks_for(n), 256, 0, s>>>(n, new2old);
            EH_CUDA_TRY(cudaGetLastError());
            return EH_OK;
        default:
            break;
    }
    if (ordering > EH_ORDER_IDENTITY) {
        eh_set_error("unknown vertex ordering %u", ordering);
        return EH_EINVAL;
    }
    uint64_t *off = nullptr, *adj = nullptr;
    EH_TRY(old_csr(ukeys, m, n, nb, deg, s, sc, &off, &adj));
    if (ordering == EH_ORDER_SHINGLE) {
        k_keys_shingle<<<blocks_for(n, 8), 256, 0, s>>>(off, adj, n, seed, nb, keys);
        return sort_to_order(&keys, &keys2, n, 64, nb, s, new2old);
    }
    // the remaining orderings start from the degree order
    uint32_t *deg_order = nullptr, *rank = nullptr;
    EH_TRY(sc.alloc(&deg_order, n));
    EH_TRY(sc.alloc(&rank, n));
    k_keys_degree<<<blocks_for(n), 256, 0, s>>>(deg, n, maxdeg, nb, 0, keys);
    EH_TRY(sort_to_order(&keys, &keys2, n, nb + db, nb, s, deg_order));
    if (ordering == EH_ORDER_STRONG_RUNS) {
        k_rank_of<<<blocks_for(n), 256, 0, s>>>(deg_order, n, rank);
        k_keys_strong<<<blocks_for(n, 8), 256, 0, s>>>(off, adj, rank, deg_order, n, nb, keys);
        return sort_to_order(&keys, &keys2, n, 2 * nb + 1, nb, s, new2old);
    }
    uint32_t *bfs = ordering == EH_ORDER_BFS ? new2old : nullptr, *pos = rank;
    if (!bfs) EH_TRY(sc.alloc(&bfs, n));
    EH_TRY(bfs_order(off, adj, n, nb, deg_order, s, sc, bfs, pos));
    if (ordering == EH_ORDER_BFS) return EH_OK;
    // HYBRID: BFS positions, then stable by degree descending
    k_keys_hybrid<<<blocks_for(n), 256, 0, s>>>(deg, pos, n, maxdeg, nb, keys);
    EH_TRY(dev_radix_sort_u64(&keys, &keys2, n, nb + db, s));
    k_gather<<<blocks_for(n), 256, 0, s>>>(keys, bfs, n, nb, new2old);
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}
