// trie_build.cu -- eh_build_trie: edge list -> device-resident two-level trie.
//
// Steps (EmptyHeaded Sec. 2.2 and 4.4, App. A.1):
//   1. canonical undirected pairs (lo, hi), self-loops dropped, ids checked;
//   2. radix sort + unique: the simple edge relation (m edges);
//   3. degrees, then new ids by the chosen node ordering (order.cu; default
//      (degree desc, original id asc), the "Degree" ordering);
//   4. every edge once as (hi, lo) in new ids, radix sorted: hi's run is the
//      pruned set N+(hi) (each undirected edge kept in the set of its larger
//      endpoint) and the lower part of the symmetric set N(hi); the same keys
//      re-sorted stably on lo alone give the upper part of N(lo);
//   5. per-set layout: a bitset copy of N+(v) when range <= tau*|N+(v)|.
#include "eh_internal.cuh"

#include <cmath>
#include <new>
#include <algorithm>

namespace {

__global__ void k_canon_keys(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst, uint64_t ne,
                             uint32_t n, int nb, uint64_t *keys, uint32_t *status) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    uint32_t a = src[i], b = dst[i];
    if (a >= n || b >= n) {
        atomicOr(status, DEV_ST_INVALID);
        keys[i] = ~0ull;
        return;
    }
    if (a == b) { keys[i] = ~0ull; return; }
    uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
    keys[i] = ((uint64_t)lo << nb) | hi;
}

__global__ void k_unique_flags(const uint64_t *__restrict__ keys, uint64_t ne, uint32_t *flags) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    uint64_t k = keys[i];
    flags[i] = (k != ~0ull && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
}

__global__ void k_unique_scatter(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ flags,
                                 const uint32_t *__restrict__ pos, uint64_t ne, uint64_t *out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    if (flags[i]) out[pos[i]] = keys[i];
}

// degrees of both endpoints; lanes hitting the same vertex (hubs) add once
// per warp, so high-degree counters do not serialise on atomics
__global__ void k_degrees(const uint64_t *__restrict__ ukeys, uint64_t m, int nb, uint32_t *deg) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < m;
    uint64_t k = valid ? ukeys[i] : 0ull;
    uint32_t ends[2] = {valid ? (uint32_t)(k >> nb) : 0xFFFFFFFFu,
                        valid ? (uint32_t)(k & ((1ull << nb) - 1)) : 0xFFFFFFFFu};
    const uint32_t lt = (1u << (threadIdx.x & 31)) - 1u;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        uint32_t peers = __match_any_sync(0xffffffffu, ends[e]);
        if (valid && (peers & lt) == 0) atomicAdd(&deg[ends[e]], (uint32_t)__popc(peers));
    }
}

__global__ void k_max_u32(const uint32_t *__restrict__ x, uint64_t n, uint32_t *out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t v = i < n ? x[i] : 0u;
    for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, d));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(out, v);
}

__global__ void k_maps_from_order(const uint32_t *__restrict__ new2old, uint32_t n,
                                  const uint32_t *__restrict__ deg_old, uint32_t *old2new, uint32_t *deg_new) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t old = new2old[i];
    old2new[old] = (uint32_t)i;
    deg_new[i] = deg_old[old];
}

// trie statistics: cnt = {vertices with edges, non-empty pruned sets, bitset
// sets, max |N+(v)|}; part[2 block] = sum of d(v), sum of d(v)^2 over the
// block's vertices; hist[d] = vertices of degree d
__global__ void k_stats(const uint32_t *__restrict__ deg, const uint32_t *__restrict__ odeg,
                        const uint64_t *__restrict__ nwords, uint32_t n, unsigned long long *cnt, double *part,
                        uint32_t *hist) {
    __shared__ double s1[8], s2[8];
    const uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = v < n;
    const uint32_t d = ok ? deg[v] : 0, od = ok ? odeg[v] : 0;
    const uint32_t FULLM = 0xffffffffu;
    const unsigned act = __popc(__ballot_sync(FULLM, ok && d)), nne = __popc(__ballot_sync(FULLM, ok && od)),
                   nbs = __popc(__ballot_sync(FULLM, ok && nwords[ok ? v : 0]));
    uint32_t mo = od;
    double a = d, b = (double)d * d;
    for (int k = 16; k > 0; k >>= 1) {
        mo = max(mo, __shfl_xor_sync(FULLM, mo, k));
        a += __shfl_xor_sync(FULLM, a, k);
        b += __shfl_xor_sync(FULLM, b, k);
    }
    {   // one atomic per distinct degree in the warp (many vertices share small degrees)
        const uint32_t peers = __match_any_sync(FULLM, ok ? d : 0xFFFFFFFFu);
        if (ok && (peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0) atomicAdd(&hist[d], (uint32_t)__popc(peers));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        if (act) atomicAdd(&cnt[0], (unsigned long long)act);
        if (nne) atomicAdd(&cnt[1], (unsigned long long)nne);
        if (nbs) atomicAdd(&cnt[2], (unsigned long long)nbs);
        if (mo) atomicMax(&cnt[3], (unsigned long long)mo);
        s1[w] = a;
        s2[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { x += s1[i]; y += s2[i]; }
        part[2 * blockIdx.x] = x;
        part[2 * blockIdx.x + 1] = y;
    }
}

// each unique edge once as (hi, lo) in new ids, hi > lo
__global__ void k_pruned_keys(const uint64_t *__restrict__ ukeys, uint64_t m, int nb,
                              const uint32_t *__restrict__ old2new, uint64_t *dk) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t k = ukeys[i];
    uint32_t a = old2new[(uint32_t)(k >> nb)], b = old2new[(uint32_t)(k & ((1ull << nb) - 1))];
    uint32_t hi = a > b ? a : b, lo = a > b ? b : a;
    dk[i] = ((uint64_t)hi << nb) | lo;
}

// |N+(v)|: the run length of each high endpoint in keys sorted by it (lanes of
// the same run add once per warp)
__global__ void k_count_hi(const uint64_t *__restrict__ keys, uint64_t m, int nb, uint32_t *cnt) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < m;
    const uint32_t v = valid ? (uint32_t)(keys[i] >> nb) : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xffffffffu, v);
    if (valid && (peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0) atomicAdd(&cnt[v], (uint32_t)__popc(peers));
}

__global__ void k_round4(const uint32_t *__restrict__ x, uint64_t n, uint64_t *out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ((uint64_t)x[i] + 3) & ~3ull;
}

__global__ void k_widen(const uint32_t *__restrict__ x, uint64_t n, uint64_t *out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = x[i];
}

__global__ void k_widen_diff(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b, uint64_t n,
                             uint64_t *out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint64_t)(a[i] - b[i]);
}

// keys sorted by (v, w), w < v: entry i is element i - astart[v] of N+(v),
// which is also the lower part of N(v)
// (an entry outside its vertex's range, which sorted input rules out, is not
// written and sets the status word)
__global__ void k_fill_lower(const uint64_t *__restrict__ A, uint64_t m, int nb, uint32_t n,
                             const uint64_t *__restrict__ astart, const uint64_t *__restrict__ soff,
                             const uint64_t *__restrict__ ooff, uint32_t *snbr, uint32_t *onbr, uint32_t *status) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint64_t k = A[i];
    const uint32_t v = (uint32_t)(k >> nb), w = (uint32_t)(k & ((1ull << nb) - 1));
    if (v >= n || i < astart[v] || i >= astart[v + 1]) { atomicOr(status, DEV_ST_RANGE); return; }
    const uint64_t j = i - astart[v];
    snbr[soff[v] + j] = w;
    onbr[ooff[v] + j] = w;
}

// the same keys re-sorted stably by w alone: for each w, its larger neighbours
// v in ascending order, the upper part of N(w) after its |N+(w)| lower entries
__global__ void k_fill_upper(const uint64_t *__restrict__ B, uint64_t m, int nb, uint32_t n,
                             const uint64_t *__restrict__ bstart, const uint64_t *__restrict__ soff,
                             const uint32_t *__restrict__ odeg, uint32_t *snbr, uint32_t *status) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint64_t k = B[i];
    const uint32_t v = (uint32_t)(k >> nb), w = (uint32_t)(k & ((1ull << nb) - 1));
    if (w >= n || i < bstart[w] || i >= bstart[w + 1]) { atomicOr(status, DEV_ST_RANGE); return; }
    snbr[soff[w] + odeg[w] + (i - bstart[w])] = v;
}

// set-level layout rule (Sec. 4.4): words needed by each set's bitset, 0 = uint
__global__ void k_layout(const uint32_t *__restrict__ onbr, const uint64_t *__restrict__ ooff,
                         const uint32_t *__restrict__ odeg, uint32_t n, uint32_t tau, uint32_t min_len,
                         uint64_t *nwords, uint32_t *lo_word) {
    uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    uint32_t len = odeg[v];
    uint64_t w = 0;
    uint32_t lw = 0;
    if (len > 0 && tau > 0 && len >= min_len) {
        uint32_t first = onbr[ooff[v]], last = onbr[ooff[v] + len - 1];
        uint64_t range = (uint64_t)last - first + 1;
        if (tau == 0xFFFFFFFFu || range <= (uint64_t)tau * len) {
            lw = (first >> 7) << 2;                       // 128-bit aligned
            uint64_t hw = (last >> 5) + 1;
            w = (hw - lw + 3) & ~3ull;
        }
    }
    nwords[v] = w;
    lo_word[v] = lw;
}

__global__ void k_fill_bits(const uint32_t *__restrict__ onbr, const uint64_t *__restrict__ ooff,
                            const uint32_t *__restrict__ odeg, const uint64_t *__restrict__ nwords,
                            const uint64_t *__restrict__ woff, const uint32_t *__restrict__ lo_word, uint32_t n,
                            uint32_t *words) {
    uint32_t v = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (v >= n || nwords[v] == 0) return;
    uint32_t len = odeg[v];
    uint64_t base = woff[v];
    uint32_t lw = lo_word[v];
    for (uint32_t j = threadIdx.x & 31; j < len; j += 32) {
        uint32_t x = onbr[ooff[v] + j];
        atomicOr(&words[base + ((x >> 5) - lw)], 1u << (x & 31));
    }
}

__global__ void k_desc(const uint64_t *__restrict__ ooff, const uint32_t *__restrict__ odeg,
                       const uint32_t *__restrict__ sdeg, const uint64_t *__restrict__ nwords,
                       const uint64_t *__restrict__ woff, const uint32_t *__restrict__ lo_word, uint32_t n,
                       SetDesc *desc) {
    uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    SetDesc d;
    d.off = ooff[v];
    d.len = odeg[v];
    d.deg = sdeg[v];
    d.woff = nwords[v] ? woff[v] : 0;
    d.lo_word = lo_word[v];
    d.nwords = (uint32_t)nwords[v];
    desc[v] = d;
}

void free_trie_arrays(eh_trie *t) {
    // the trie's arrays come from the default memory pool (stream-ordered); the
    // device is idle here (callers synchronise first), so the frees are
    // immediate and the pool keeps the memory for the next trie
    void *pooled[] = {t->d_new2old, t->d_old2new, t->d_soff, t->d_snbr, t->d_desc, t->d_onbr, t->d_words,
                      t->d_deg, t->d_scratch, t->d_status, t->d_boff, t->d_bdir, t->d_bwords};
    for (void *p : pooled)
        if (p) cudaFreeAsync(p, 0);
    cudaFree(t->d_arena);
    for (auto &kv : t->plans) {
        cudaFree(kv.second.d_heavy);
        cudaFree(kv.second.d_light);
        cudaFree(kv.second.d_heavy_blk);
        if (kv.second.d_cost) cudaFreeAsync(kv.second.d_cost, 0);
    }
    t->plans.clear();
}

// memory the trie keeps: from the device's default pool, on the build stream
template <typename T>
eh_status persist_alloc(T **p, uint64_t count, uint64_t *bytes, cudaStream_t s) {
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
    *bytes += sizeof(T) * count;
    return EH_OK;
}

// Scope guard for stream-ordered temporaries.
struct Temps {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Temps(cudaStream_t st) : s(st) {}
    template <typename T>
    eh_status alloc(T **p, uint64_t count) {
        eh_status st = dev_alloc(p, count, s);
        if (st == EH_OK) ptrs.push_back((void *)*p);
        return st;
    }
    template <typename T>
    void release(T *&p) {
        for (auto &q : ptrs)
            if (q == (void *)p) { cudaFreeAsync(q, s); q = nullptr; }
        p = nullptr;
    }
    ~Temps() {
        for (void *q : ptrs)
            if (q) cudaFreeAsync(q, s);
    }
};

eh_status build(const uint32_t *src, const uint32_t *dst, uint64_t ne, uint32_t n, const eh_build_opts &o,
                cudaStream_t s, eh_trie *t) {
    Temps tmp(s);
    uint64_t bytes = 0;
    const int nb = bits_for(n);
    t->nb = nb;
    if (2 * nb > 64) { eh_set_error("id space too large"); return EH_EINVAL; }

    // scratch shared by the count kernels
    EH_TRY(persist_alloc(&t->d_scratch, 16, &bytes, s));
    EH_TRY(persist_alloc(&t->d_status, 4, &bytes, s));
    EH_CUDA_TRY(cudaMemsetAsync(t->d_scratch, 0, 16 * sizeof(unsigned long long), s));
    EH_CUDA_TRY(cudaMemsetAsync(t->d_status, 0, 4 * sizeof(uint32_t), s));

    // 0. inputs on the device.  Pinned host arrays are read in place by the
    // first kernel (they are device-addressable; on a coherent CPU-GPU link
    // this streams them once instead of copying them first); other host
    // arrays are copied.
    const uint32_t *d_src = src, *d_dst = dst;
    bool host_mapped = false;
    if (!(o.flags & EH_BUILD_DEVICE_INPUT) && ne > 0) {
        cudaPointerAttributes as, ad;
        if (cudaPointerGetAttributes(&as, src) == cudaSuccess && cudaPointerGetAttributes(&ad, dst) == cudaSuccess &&
            as.type == cudaMemoryTypeHost && ad.type == cudaMemoryTypeHost && as.devicePointer && ad.devicePointer) {
            d_src = (const uint32_t *)as.devicePointer;
            d_dst = (const uint32_t *)ad.devicePointer;
            host_mapped = true;
        }
        cudaGetLastError();
    }
    if (!(o.flags & EH_BUILD_DEVICE_INPUT) && ne > 0 && !host_mapped) {
        uint32_t *a = nullptr, *b = nullptr;
        EH_TRY(tmp.alloc(&a, ne));
        EH_TRY(tmp.alloc(&b, ne));
        EH_CUDA_TRY(cudaMemcpyAsync(a, src, ne * 4, cudaMemcpyHostToDevice, s));
        EH_CUDA_TRY(cudaMemcpyAsync(b, dst, ne * 4, cudaMemcpyHostToDevice, s));
        d_src = a;
        d_dst = b;
    }

    // 1-2. canonical keys, sort, unique
    uint64_t *keys = nullptr, *keys2 = nullptr, *ukeys = nullptr;
    uint32_t *flags = nullptr, *pos = nullptr;
    uint64_t m = 0;
    if (ne > 0) {
        EH_TRY(tmp.alloc(&keys, ne));
        EH_TRY(tmp.alloc(&keys2, ne));
        k_canon_keys<<<blocks_for(ne), 256, 0, s>>>(d_src, d_dst, ne, n, nb, keys, t->d_status);
        uint32_t st_h = 0;
        EH_CUDA_TRY(cudaMemcpyAsync(&st_h, t->d_status, 4, cudaMemcpyDeviceToHost, s));
        EH_CUDA_TRY(cudaStreamSynchronize(s));
        if (st_h & DEV_ST_INVALID) {
            eh_set_error("an edge endpoint is >= n_vertices (%u)", n);
            return EH_EINVAL;
        }
        EH_TRY(dev_radix_sort_u64(&keys, &keys2, ne, 2 * nb, s));
        EH_TRY(tmp.alloc(&flags, ne));
        EH_TRY(tmp.alloc(&pos, ne));
        k_unique_flags<<<blocks_for(ne), 256, 0, s>>>(keys, ne, flags);
        EH_TRY(dev_exclusive_scan_u32(flags, pos, ne, s, &m));
        EH_TRY(tmp.alloc(&ukeys, m));
        k_unique_scatter<<<blocks_for(ne), 256, 0, s>>>(keys, flags, pos, ne, ukeys);
        tmp.release(flags);
        tmp.release(pos);
        tmp.release(keys);
        tmp.release(keys2);
    }
    t->m = m;

    // 3. degrees and the degree ordering
    uint32_t *deg_old = nullptr, *d_max = nullptr;
    EH_TRY(tmp.alloc(&deg_old, n));
    EH_TRY(tmp.alloc(&d_max, 1));
    EH_CUDA_TRY(cudaMemsetAsync(deg_old, 0, (uint64_t)n * 4, s));
    EH_CUDA_TRY(cudaMemsetAsync(d_max, 0, 4, s));
    if (m) k_degrees<<<blocks_for(m), 256, 0, s>>>(ukeys, m, nb, deg_old);
    if (n) k_max_u32<<<blocks_for(n), 256, 0, s>>>(deg_old, n, d_max);
    uint32_t maxdeg = 0;
    EH_CUDA_TRY(cudaMemcpyAsync(&maxdeg, d_max, 4, cudaMemcpyDeviceToHost, s));
    EH_CUDA_TRY(cudaStreamSynchronize(s));
    t->max_deg = maxdeg;

    EH_TRY(persist_alloc(&t->d_new2old, n, &bytes, s));
    EH_TRY(persist_alloc(&t->d_old2new, n, &bytes, s));
    EH_TRY(persist_alloc(&t->d_deg, n, &bytes, s));
    EH_TRY(eh_vertex_order(o.ordering, o.order_seed, ukeys, m, n, nb, deg_old, maxdeg, s, t->d_new2old));
    if (n) k_maps_from_order<<<blocks_for(n), 256, 0, s>>>(t->d_new2old, n, deg_old, t->d_old2new, t->d_deg);

    // 4. the pruned and symmetric tries.  Each edge once as (hi, lo) in new
    // ids, sorted: N+(v) is v's run.  The same keys re-sorted stably by lo
    // alone list each vertex's larger neighbours in ascending order, so N(v)
    // is N+(v) followed by v's run there (every lower neighbour precedes v,
    // every higher one follows it).
    uint64_t *dk = nullptr, *dk2 = nullptr;
    EH_TRY(tmp.alloc(&dk, m));
    EH_TRY(tmp.alloc(&dk2, m));
    if (m) k_pruned_keys<<<blocks_for(m), 256, 0, s>>>(ukeys, m, nb, t->d_old2new, dk);
    tmp.release(ukeys);
    EH_TRY(dev_radix_sort_u64(&dk, &dk2, m, 2 * nb, s));
    uint32_t *odeg = nullptr;
    EH_TRY(tmp.alloc(&odeg, n));
    EH_CUDA_TRY(cudaMemsetAsync(odeg, 0, (uint64_t)n * 4, s));
    if (m) k_count_hi<<<blocks_for(m), 256, 0, s>>>(dk, m, nb, odeg);

    uint64_t *astart = nullptr, *bstart = nullptr, *wide = nullptr, *ooff = nullptr;
    EH_TRY(tmp.alloc(&astart, (uint64_t)n + 1));
    EH_TRY(tmp.alloc(&bstart, (uint64_t)n + 1));
    EH_TRY(tmp.alloc(&wide, (uint64_t)n + 1));
    EH_TRY(tmp.alloc(&ooff, (uint64_t)n + 1));
    EH_CUDA_TRY(cudaMemsetAsync(wide, 0, ((uint64_t)n + 1) * 8, s));
    if (n) k_widen<<<blocks_for(n), 256, 0, s>>>(odeg, n, wide);
    EH_TRY(dev_exclusive_scan_u64(wide, astart, (uint64_t)n + 1, s, nullptr));
    if (n) k_widen_diff<<<blocks_for(n), 256, 0, s>>>(t->d_deg, odeg, n, wide);
    EH_TRY(dev_exclusive_scan_u64(wide, bstart, (uint64_t)n + 1, s, nullptr));
    EH_TRY(persist_alloc(&t->d_soff, (uint64_t)n + 1, &bytes, s));
    if (n) k_round4<<<blocks_for(n), 256, 0, s>>>(t->d_deg, n, wide);
    uint64_t slen = 0;
    EH_TRY(dev_exclusive_scan_u64(wide, t->d_soff, (uint64_t)n + 1, s, &slen));
    t->snbr_len = slen;
    if (n) k_round4<<<blocks_for(n), 256, 0, s>>>(odeg, n, wide);
    uint64_t olen = 0;
    EH_TRY(dev_exclusive_scan_u64(wide, ooff, (uint64_t)n + 1, s, &olen));
    t->onbr_len = olen;
    EH_TRY(persist_alloc(&t->d_snbr, slen, &bytes, s));
    EH_TRY(persist_alloc(&t->d_onbr, olen, &bytes, s));
    EH_CUDA_TRY(cudaMemsetAsync(t->d_snbr, 0xFF, (slen ? slen : 1) * 4, s));
    EH_CUDA_TRY(cudaMemsetAsync(t->d_onbr, 0xFF, (olen ? olen : 1) * 4, s));
    if (m)
        k_fill_lower<<<blocks_for(m), 256, 0, s>>>(dk, m, nb, n, astart, t->d_soff, ooff, t->d_snbr, t->d_onbr,
                                                   t->d_status);
    EH_TRY(dev_radix_sort_u64(&dk, &dk2, m, nb, s));
    if (m) k_fill_upper<<<blocks_for(m), 256, 0, s>>>(dk, m, nb, n, bstart, t->d_soff, odeg, t->d_snbr, t->d_status);
    {
        uint32_t st_h = 0;
        EH_CUDA_TRY(cudaMemcpyAsync(&st_h, t->d_status, 4, cudaMemcpyDeviceToHost, s));
        EH_CUDA_TRY(cudaStreamSynchronize(s));
        if (st_h & DEV_ST_RANGE) {
            eh_set_error("trie build: an adjacency entry fell outside its vertex's range");
            return EH_ECUDA;
        }
    }
    tmp.release(dk);
    tmp.release(dk2);
    tmp.release(astart);
    tmp.release(bstart);

    // 5. layouts
    uint64_t *nwords = nullptr, *woff = nullptr;
    uint32_t *lo_word = nullptr;
    EH_TRY(tmp.alloc(&nwords, (uint64_t)n + 1));
    EH_TRY(tmp.alloc(&woff, (uint64_t)n + 1));
    EH_TRY(tmp.alloc(&lo_word, (uint64_t)n + 1));
    EH_CUDA_TRY(cudaMemsetAsync(nwords, 0, ((uint64_t)n + 1) * 8, s));
    // set-level bitsets, or none when the composite layout replaces them
    const uint32_t set_tau = (o.flags & EH_BUILD_BLOCK_LAYOUT) ? 0u : o.bitset_tau;
    if (n) k_layout<<<blocks_for(n), 256, 0, s>>>(t->d_onbr, ooff, odeg, n, set_tau, o.min_bitset_len, nwords, lo_word);
    uint64_t tw = 0;
    EH_TRY(dev_exclusive_scan_u64(nwords, woff, (uint64_t)n + 1, s, &tw));
    t->n_words = tw;
    EH_TRY(persist_alloc(&t->d_words, tw, &bytes, s));
    EH_CUDA_TRY(cudaMemsetAsync(t->d_words, 0, (tw ? tw : 1) * 4, s));
    if (n) k_fill_bits<<<blocks_for(n, 8), 256, 0, s>>>(t->d_onbr, ooff, odeg, nwords, woff, lo_word, n, t->d_words);
    EH_TRY(persist_alloc(&t->d_desc, n, &bytes, s));
    if (n) k_desc<<<blocks_for(n), 256, 0, s>>>(ooff, odeg, t->d_deg, nwords, woff, lo_word, n, t->d_desc);

    // stats (diagnostics): counts and maxima by device atomics, the degree sums
    // as per-block partials summed on the host in block order (deterministic),
    // the degree mode from a device histogram
    {
        const uint32_t nblk = n ? blocks_for(n) : 1;
        unsigned long long *cnt = nullptr;   // active, nonempty, bitset, max out-degree
        double *part = nullptr;               // per block: sum d, sum d^2
        uint32_t *hist = nullptr;
        EH_TRY(tmp.alloc(&cnt, 4));
        EH_TRY(tmp.alloc(&part, 2 * (uint64_t)nblk));
        EH_TRY(tmp.alloc(&hist, (uint64_t)maxdeg + 1));
        EH_CUDA_TRY(cudaMemsetAsync(cnt, 0, 32, s));
        EH_CUDA_TRY(cudaMemsetAsync(part, 0, 16 * (uint64_t)nblk, s));
        EH_CUDA_TRY(cudaMemsetAsync(hist, 0, 4 * ((uint64_t)maxdeg + 1), s));
        if (n) k_stats<<<nblk, 256, 0, s>>>(t->d_deg, odeg, nwords, n, cnt, part, hist);
        unsigned long long hc[4] = {0, 0, 0, 0};
        std::vector<double> hp(2 * (size_t)nblk);
        std::vector<uint32_t> hh((size_t)maxdeg + 1);
        EH_CUDA_TRY(cudaMemcpyAsync(hc, cnt, 32, cudaMemcpyDeviceToHost, s));
        EH_CUDA_TRY(cudaMemcpyAsync(hp.data(), part, 16 * (uint64_t)nblk, cudaMemcpyDeviceToHost, s));
        EH_CUDA_TRY(cudaMemcpyAsync(hh.data(), hist, 4 * ((uint64_t)maxdeg + 1), cudaMemcpyDeviceToHost, s));
        EH_CUDA_TRY(cudaStreamSynchronize(s));
        EH_CUDA_TRY(cudaGetLastError());
        double sum = 0, sum2 = 0;
        for (uint32_t i = 0; i < nblk; ++i) { sum += hp[2 * i]; sum2 += hp[2 * i + 1]; }
        t->n_active = (uint32_t)hc[0];
        t->n_nonempty = hc[1];
        t->n_bitset = hc[2];
        t->max_out = (uint32_t)hc[3];
        double mean = n ? sum / n : 0, var = n ? sum2 / n - mean * mean : 0;
        uint32_t mode = 0, best = 0;
        for (uint32_t d = 0; d <= maxdeg; ++d)
            if (hh[d] > best) { best = hh[d]; mode = d; }
        t->density_skew = var > 0 ? 3.0 * (mean - mode) / std::sqrt(var) : 0.0;
    }
    t->device_bytes = bytes;
    if (o.flags & EH_BUILD_BLOCK_LAYOUT) EH_TRY(eh_build_blocks(t, o.bitset_tau, s));
    return EH_OK;
}

}  // namespace

// Set-level layouts (Sec. 4.4) for a pruned trie given as padded uint
// arrays: decides bitset/uint per set, fills the bitset pool and the
// descriptors.  Used for the induced sub-tries of query batches.
eh_status eh_build_layouts(const uint32_t *nbr, const uint64_t *off, const uint32_t *len, const uint32_t *deg,
                           uint32_t nv, uint32_t tau, uint32_t min_len, cudaStream_t s, SetDesc *desc_out,
                           uint32_t **words_out, uint64_t *n_words_out, uint64_t *n_bitset_out) {
    *words_out = nullptr;
    *n_words_out = 0;
    Temps tmp(s);
    uint64_t *nwords = nullptr, *woff = nullptr;
    uint32_t *lo_word = nullptr;
    EH_TRY(tmp.alloc(&nwords, (uint64_t)nv + 1));
    EH_TRY(tmp.alloc(&woff, (uint64_t)nv + 1));
    EH_TRY(tmp.alloc(&lo_word, (uint64_t)nv + 1));
    EH_CUDA_TRY(cudaMemsetAsync(nwords, 0, ((uint64_t)nv + 1) * 8, s));
    if (nv) k_layout<<<blocks_for(nv), 256, 0, s>>>(nbr, off, len, nv, tau, min_len, nwords, lo_word);
    uint64_t tw = 0;
    EH_TRY(dev_exclusive_scan_u64(nwords, woff, (uint64_t)nv + 1, s, &tw));
    uint32_t *words = nullptr;
    EH_TRY(dev_alloc(&words, tw, s));
    EH_CUDA_TRY(cudaMemsetAsync(words, 0, (tw ? tw : 1) * 4, s));
    if (nv) k_fill_bits<<<blocks_for(nv, 8), 256, 0, s>>>(nbr, off, len, nwords, woff, lo_word, nv, words);
    if (nv) k_desc<<<blocks_for(nv), 256, 0, s>>>(off, len, deg, nwords, woff, lo_word, nv, desc_out);
    if (n_bitset_out) *n_bitset_out = 0;   // not tracked for sub-tries
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        dev_free(words, s);
        eh_set_error("layouts: %s", cudaGetErrorString(e));
        return EH_ECUDA;
    }
    *words_out = words;
    *n_words_out = tw;
    return EH_OK;
}

// The stream-ordered temporaries of builds, plans and batches come from the
// device's default memory pool.  By default the pool returns freed memory to
// the driver at every synchronisation, so the next build maps it again; the
// process keeps it cached instead (a property of this process's pool only).
static void keep_pool_memory() {
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return; }
    std::lock_guard<std::mutex> g(mu);
    for (int d : done)
        if (d == dev) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done.push_back(dev);
}

extern "C" eh_status eh_trim_memory(void) {
    int dev = 0;
    cudaMemPool_t pool;
    EH_CUDA_TRY(cudaGetDevice(&dev));
    EH_CUDA_TRY(cudaDeviceSynchronize());
    EH_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    EH_CUDA_TRY(cudaMemPoolTrimTo(pool, 0));
    return EH_OK;
}

// |N+(v)| by original id on the host (the serving loop's footprint estimate),
// built on first use
eh_status eh_host_out_degrees(eh_trie *t) {
    std::lock_guard<std::mutex> g(t->mu);
    if (t->h_out_by_old.size() == t->n) return EH_OK;
    const uint32_t n = t->n;
    std::vector<uint32_t> n2o(n);
    std::vector<SetDesc> desc(n);
    if (n) {
        EH_CUDA_TRY(cudaMemcpy(n2o.data(), t->d_new2old, (uint64_t)n * 4, cudaMemcpyDeviceToHost));
        EH_CUDA_TRY(cudaMemcpy(desc.data(), t->d_desc, (uint64_t)n * sizeof(SetDesc), cudaMemcpyDeviceToHost));
    }
    std::vector<uint32_t> out(n, 0);
    for (uint32_t v = 0; v < n; ++v) out[n2o[v]] = desc[v].len;
    t->h_out_by_old.swap(out);
    return EH_OK;
}

extern "C" eh_status eh_build_trie(const uint32_t *src, const uint32_t *dst, uint64_t n_edges, uint32_t n_vertices,
                                   const eh_build_opts *opts, void *stream, eh_trie **out) {
    if (!out) { eh_set_error("eh_build_trie: out is NULL"); return EH_EINVAL; }
    *out = nullptr;
    if (n_edges > 0 && (!src || !dst)) { eh_set_error("eh_build_trie: src/dst NULL"); return EH_EINVAL; }
    if (n_vertices > 0xFFE00000u) { eh_set_error("eh_build_trie: n_vertices above 0xFFE00000"); return EH_EINVAL; }
    if (n_edges >= (1ull << 31)) { eh_set_error("eh_build_trie: more than 2^31 input edges"); return EH_EINVAL; }
    eh_build_opts o;
    o.bitset_tau = 32;
    o.min_bitset_len = 0;
    o.flags = 0;
    o.ordering = EH_ORDER_DEGREE;
    o.order_seed = 0;
    if (opts) o = *opts;
    if (o.ordering > EH_ORDER_IDENTITY) { eh_set_error("eh_build_trie: unknown ordering %u", o.ordering); return EH_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    NvtxRange nv("eh_build_trie");
    keep_pool_memory();
    eh_trie *t = new (std::nothrow) eh_trie();
    if (!t) { eh_set_error("host allocation failed"); return EH_ENOMEM; }
    t->n = n_vertices;
    t->opts = o;
    eh_status st = build(src, dst, n_edges, n_vertices, o, s, t);
    // eh_count_noalloc's static scratch and kernels made resident on this
    // device now, so that its calls load (and allocate) nothing
    if (st == EH_OK) st = eh_noalloc_setup(s);
    if (st != EH_OK) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        free_trie_arrays(t);
        delete t;
        return st;
    }
    *out = t;
    return EH_OK;
}

extern "C" void eh_free_trie(eh_trie *t) {
    if (!t) return;
    cudaDeviceSynchronize();
    free_trie_arrays(t);
    delete t;
}

extern "C" eh_status eh_trie_stats_get(const eh_trie *t, eh_trie_stats_t *o) {
    if (!t || !o) { eh_set_error("eh_trie_stats_get: NULL argument"); return EH_EINVAL; }
    memset(o, 0, sizeof(*o));
    o->n_vertices = t->n;
    o->n_active = t->n_active;
    o->n_edges = t->m;
    o->max_degree = t->max_deg;
    o->max_out_degree = t->max_out;
    o->n_bitset_sets = t->n_bitset;
    o->n_nonempty_sets = t->n_nonempty;
    o->bitset_words = t->n_words;
    o->density_skew = t->density_skew;
    o->device_bytes = t->device_bytes;
    o->bitset_tau = t->opts.bitset_tau;
    return EH_OK;
}

extern "C" eh_status eh_trie_stats(const eh_trie *t, eh_trie_stats_t *o) { return eh_trie_stats_get(t, o); }

extern "C" eh_status eh_trie_export(const eh_trie *t, uint32_t which, uint32_t *new_to_old, uint64_t *out_off,
                                    uint32_t *out_len, uint32_t *out_nbr, uint32_t *bits_lo, uint32_t *bits_nwords,
                                    uint64_t *bits_off, uint32_t *out_words) {
    if (!t || which > 1) { eh_set_error("eh_trie_export: bad argument"); return EH_EINVAL; }
    const uint32_t n = t->n;
    if (new_to_old && n) EH_CUDA_TRY(cudaMemcpy(new_to_old, t->d_new2old, (uint64_t)n * 4, cudaMemcpyDeviceToHost));
    std::vector<SetDesc> desc(n);
    if (n) EH_CUDA_TRY(cudaMemcpy(desc.data(), t->d_desc, (uint64_t)n * sizeof(SetDesc), cudaMemcpyDeviceToHost));
    if (which == 0) {
        for (uint32_t v = 0; v < n; ++v) {
            if (out_off) out_off[v] = desc[v].off;
            if (out_len) out_len[v] = desc[v].len;
            if (bits_lo) bits_lo[v] = desc[v].nwords ? desc[v].lo_word * 32u : 0xFFFFFFFFu;
            if (bits_nwords) bits_nwords[v] = desc[v].nwords;
            if (bits_off) bits_off[v] = desc[v].woff;
        }
        if (out_off) out_off[n] = t->onbr_len;
        if (out_nbr && t->onbr_len)
            EH_CUDA_TRY(cudaMemcpy(out_nbr, t->d_onbr, t->onbr_len * 4, cudaMemcpyDeviceToHost));
        if (out_words && t->n_words)
            EH_CUDA_TRY(cudaMemcpy(out_words, t->d_words, t->n_words * 4, cudaMemcpyDeviceToHost));
    } else {
        if (out_off) EH_CUDA_TRY(cudaMemcpy(out_off, t->d_soff, ((uint64_t)n + 1) * 8, cudaMemcpyDeviceToHost));
        if (out_len) for (uint32_t v = 0; v < n; ++v) out_len[v] = desc[v].deg;
        if (out_nbr && t->snbr_len)
            EH_CUDA_TRY(cudaMemcpy(out_nbr, t->d_snbr, t->snbr_len * 4, cudaMemcpyDeviceToHost));
        for (uint32_t v = 0; v < n; ++v) {
            if (bits_lo) bits_lo[v] = 0xFFFFFFFFu;
            if (bits_nwords) bits_nwords[v] = 0;
            if (bits_off) bits_off[v] = 0;
        }
    }
    return EH_OK;
}
