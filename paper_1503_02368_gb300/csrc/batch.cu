// batch.cu -- pattern counts over vertex-induced subgraphs, many queries per
// persistent launch (eh_count_batch), one query (eh_count with a subset), or
// one query at a time (the one-launch-per-query baseline).
//
// For each query q with vertex set S_q (original ids):
//   1. S_q is mapped to trie ids, sorted and deduplicated (one radix sort of
//      (q, id) keys for the whole batch);
//   2. a membership bitmap of S_q over the id space, with per-word prefix
//      popcounts, gives every member its rank in S_q;
//   3. the induced pruned trie: for every v in S_q, N+_q(v) = N+(v) ∩ S_q,
//      written as ranks (local ids, same order as the trie ids, so the
//      pruning of the whole graph carries over).  Each set is computed by the
//      same layout dispatch as the count kernels: the 128-bit AND of v's
//      bitset with the membership bitmap, or a probe of each element of
//      N+(v), with warp ballot/scan compaction of the survivors;
//   4. degrees in the induced graph (for the lollipop), set-level layouts;
//   5. a work list over the sub-vertices of all queries, heaviest first;
//   6. one launch of the fused batch kernel, captured in a CUDA graph with the
//      clears of its counters and launched as that graph.
#include "eh_internal.cuh"

#include <algorithm>
#include <chrono>
#include <vector>

namespace {

thread_local eh_batch_profile g_prof;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr uint32_t FULLM = 0xffffffffu;

__device__ __forceinline__ uint4 ldg4b(const uint32_t *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

__device__ __forceinline__ uint32_t wscan(uint32_t x, uint32_t &total) {
    const int lane = threadIdx.x & 31;
    uint32_t incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULLM, incl, d);
        if (lane >= d) incl += y;
    }
    total = __shfl_sync(FULLM, incl, 31);
    return incl - x;
}

__global__ void k_sub_keys(const uint32_t *__restrict__ pool, const uint64_t *__restrict__ qoff,
                           const uint32_t *__restrict__ qlen, const uint64_t *__restrict__ qpos,
                           const uint32_t *__restrict__ old2new, uint32_t n, int nb, uint64_t *keys, uint32_t *qstat) {
    const uint32_t q = blockIdx.x;
    const uint64_t off = qoff[q], pos = qpos[q];
    const uint32_t len = qlen[q];
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
        uint32_t id = pool[off + i];
        if (id >= n) {
            qstat[q] = 1;
            keys[pos + i] = ~0ull;
        } else {
            keys[pos + i] = ((uint64_t)q << nb) | old2new[id];
        }
    }
}

__global__ void k_sub_flags(const uint64_t *__restrict__ keys, uint64_t P, const uint32_t *__restrict__ qstat, int nb,
                            uint32_t *flags) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    uint64_t k = keys[i];
    bool f = k != ~0ull && (i == 0 || keys[i - 1] != k) && qstat[k >> nb] == 0;
    flags[i] = f ? 1u : 0u;
}

__global__ void k_sub_scatter(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ flags,
                              const uint32_t *__restrict__ pos, uint64_t P, int nb, uint32_t *sub_q, uint32_t *sub_v,
                              uint32_t *qcnt) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P || !flags[i]) return;
    uint64_t k = keys[i];
    uint32_t s = pos[i], q = (uint32_t)(k >> nb);
    sub_q[s] = q;
    sub_v[s] = (uint32_t)(k & ((1ull << nb) - 1));
    atomicAdd(&qcnt[q], 1u);
}

__global__ void k_sub_bits(const uint32_t *__restrict__ sub_q, const uint32_t *__restrict__ sub_v, uint32_t V,
                           uint64_t W, uint32_t *bm) {
    uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    uint32_t v = sub_v[s];
    atomicOr(&bm[(uint64_t)sub_q[s] * W + (v >> 5)], 1u << (v & 31));
}

__global__ void k_popc_words(const uint32_t *__restrict__ bm, uint64_t nw, uint32_t *pc) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nw) pc[i] = __popc(bm[i]);
}

// rank of member w of query q among all sub-vertices of the batch
__device__ __forceinline__ uint32_t member_rank(const uint32_t *qbm, const uint32_t *qrb, uint32_t w) {
    return qrb[w >> 5] + __popc(qbm[w >> 5] & ((1u << (w & 31)) - 1u));
}

// N+_q(v) = N+(v) ∩ S_q for every sub-vertex (one warp each).  FILL = false:
// lengths only; FILL = true: write local ids (ranks) in increasing order and
// count in-degrees.
template <bool FILL>
__global__ void k_sub_sets(TrieView tv, const uint32_t *__restrict__ sub_q, const uint32_t *__restrict__ sub_v,
                           uint32_t V, uint64_t W, const uint32_t *__restrict__ bm, const uint32_t *__restrict__ rb,
                           const uint32_t *__restrict__ qbase, const uint64_t *__restrict__ off, uint32_t *len,
                           uint32_t *nbr_out, uint32_t *indeg) {
    const uint32_t s = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= V) return;
    const uint32_t q = sub_q[s], v = sub_v[s];
    const SetDesc dv = tv.desc[v];
    const uint32_t *qbm = bm + (uint64_t)q * W;
    const uint32_t *qrb = rb + (uint64_t)q * W;
    const uint32_t base = FILL ? qbase[q] : 0u;
    uint32_t *outp = FILL ? nbr_out + off[s] : nullptr;
    uint32_t ns = 0;
    if (dv.nwords && dv.nwords <= dv.len) {
        // bitset ∩ bitset: v's words AND the membership bitmap (both 128-bit aligned)
        for (uint32_t b0 = 0; b0 < dv.nwords; b0 += 128) {
            const uint32_t i = b0 + lane * 4;
            uint32_t x[4] = {0, 0, 0, 0};
            const uint64_t gw = (uint64_t)dv.lo_word + i;
            if (i < dv.nwords && gw < W) {
                uint4 a = ldg4b(tv.words + dv.woff + i);
                uint4 b = ldg4b(qbm + gw);
                x[0] = a.x & b.x; x[1] = a.y & b.y; x[2] = a.z & b.z; x[3] = a.w & b.w;
            }
            uint32_t tot, pos = ns + wscan(__popc(x[0]) + __popc(x[1]) + __popc(x[2]) + __popc(x[3]), tot);
            if (FILL) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t w = x[k];
                    while (w) {
                        uint32_t bb = __ffs(w) - 1;
                        w &= w - 1;
                        uint32_t id = (uint32_t)(gw + k) * 32 + bb;
                        uint32_t r = member_rank(qbm, qrb, id);
                        outp[pos++] = r - base;
                        atomicAdd(&indeg[r], 1u);
                    }
                }
            }
            ns += tot;
        }
    } else {
        const uint32_t *B = tv.nbr + dv.off;
        for (uint32_t c = 0; c < dv.len; c += 128) {
            const uint32_t p = c + lane * 4;
            uint4 e = p < dv.len ? ldg4b(B + p) : make_uint4(EH_PAD, EH_PAD, EH_PAD, EH_PAD);
            uint32_t w[4] = {e.x, e.y, e.z, e.w};
            uint32_t f = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (w[k] != EH_PAD && ((__ldg(&qbm[w[k] >> 5]) >> (w[k] & 31)) & 1u)) f |= 1u << k;
            uint32_t tot, pos = ns + wscan(__popc(f), tot);
            if (FILL) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (f & (1u << k)) {
                        uint32_t r = member_rank(qbm, qrb, w[k]);
                        outp[pos++] = r - base;
                        atomicAdd(&indeg[r], 1u);
                    }
            }
            ns += tot;
        }
    }
    if (!FILL && lane == 0) len[s] = ns;
}

__global__ void k_add_u32(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b, uint32_t n, uint32_t *out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + b[i];
}

__global__ void k_round4_b(const uint32_t *__restrict__ x, uint32_t n, uint64_t *out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ((uint64_t)x[i] + 3) & ~3ull;
}

__global__ void k_max_b(const uint32_t *__restrict__ x, uint32_t n, uint32_t *out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t v = i < n ? x[i] : 0u;
    for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_xor_sync(FULLM, v, d));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(out, v);
}

// cost(s) = sum over v in N+_q(s) of |N+_q(v)| (warp per sub-vertex)
__global__ void k_bcost(BatchView bv, uint32_t V, uint64_t *cost) {
    const uint32_t s = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= V) return;
    const SetDesc ds = bv.desc[s];
    const uint32_t base = bv.qbase[bv.sub_q[s]];
    uint64_t c = 0;
    for (uint32_t j = lane; j < ds.len; j += 32) c += bv.desc[base + bv.nbr[ds.off + j]].len;
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(FULLM, c, d);
    if (lane == 0) cost[s] = c;
}

__global__ void k_bclass(const SetDesc *__restrict__ desc, uint32_t V, uint32_t light_max, int cls, uint32_t *flags) {
    uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    uint32_t len = desc[s].len;
    flags[s] = (cls == 0 ? len > light_max : (len >= 2 && len <= light_max)) ? 1u : 0u;
}

// a query's total cost (warps aggregate their sub-vertices of one query:
// a query's sub-vertices are contiguous)
__global__ void k_bqcost(const uint64_t *__restrict__ cost, const uint32_t *__restrict__ sub_q, uint32_t V,
                         unsigned long long *qcost) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = s < V;
    const uint32_t q = valid ? sub_q[s] : 0xFFFFFFFFu;
    unsigned long long c = valid ? cost[s] : 0ull;
    const uint32_t peers = __match_any_sync(FULLM, q);
    const uint32_t lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long y = __shfl_down_sync(FULLM, c, d);
        const uint32_t src = lane + d;
        if (src < 32 && ((peers >> src) & 1u)) c += y;   // peers are a contiguous run of lanes
    }
    if (valid && lane == leader && c) atomicAdd(&qcost[q], c);
}

// cost on a 14-bit logarithmic scale (exponent and the next 8 bits)
constexpr int BCOST_BITS = 14;
__device__ __forceinline__ uint32_t log_cost(uint64_t c) {
    if (!c) return 0;
    const int msb = 63 - __clzll((long long)c);
    return (uint32_t)msb * 256u + (uint32_t)(((c << (63 - msb)) >> 55) & 255u);
}

// Work-list order: query by query (qrank: the queries by total cost, heaviest
// first), and within a query its sub-vertices by cost, heaviest first.  The
// CTAs then work on one query's sub-trie at a time, which stays in L2, while
// the heaviest items still come first.
__global__ void k_bkeys(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos,
                        const uint64_t *__restrict__ cost, const uint32_t *__restrict__ sub_q,
                        const uint32_t *__restrict__ qrank, uint32_t V, int vb, uint64_t *keys) {
    uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V || !flags[s]) return;
    const uint64_t cmax = (1ull << BCOST_BITS) - 1;
    const uint64_t c = cmax - log_cost(cost[s]);
    keys[pos[s]] = (((uint64_t)qrank[sub_q[s]] << BCOST_BITS | c) << vb) | s;
}

__global__ void k_bids(const uint64_t *__restrict__ keys, uint32_t cnt, int vb, uint32_t *ids) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) ids[i] = (uint32_t)(keys[i] & ((1ull << vb) - 1));
}

inline unsigned nblk(uint64_t n, unsigned t = 256) { return (unsigned)((n + t - 1) / t); }

int bits_of(uint64_t n) {
    int b = 1;
    while (b < 63 && (1ull << b) < n) ++b;
    return b;
}

// Stream-ordered temporaries released on scope exit.
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

eh_status sorted_list(const SetDesc *desc, const uint64_t *cost, const uint32_t *sub_q, const uint32_t *qrank,
                      uint32_t nq, uint32_t V, uint32_t light_max, int cls, cudaStream_t s, Scratch &sc,
                      uint32_t **out, uint32_t *count) {
    uint32_t *flags = nullptr, *pos = nullptr;
    EH_TRY(sc.alloc(&flags, V));
    EH_TRY(sc.alloc(&pos, V));
    if (V) k_bclass<<<nblk(V), 256, 0, s>>>(desc, V, light_max, cls, flags);
    uint64_t cnt = 0;
    EH_TRY(dev_exclusive_scan_u32(flags, pos, V, s, &cnt));
    uint64_t *k1 = nullptr, *k2 = nullptr;
    uint32_t *ids = nullptr;
    EH_TRY(sc.alloc(&k1, cnt));
    EH_TRY(sc.alloc(&k2, cnt));
    EH_TRY(sc.alloc(&ids, cnt));
    const int vb = bits_of((uint64_t)V + 1), qb = bits_of((uint64_t)nq + 1);
    if (vb + qb + BCOST_BITS > 64) { eh_set_error("batch: too many sub-vertices for the work-list key"); return EH_EINVAL; }
    if (cnt) {
        k_bkeys<<<nblk(V), 256, 0, s>>>(flags, pos, cost, sub_q, qrank, V, vb, k1);
        EH_TRY(dev_radix_sort_u64(&k1, &k2, cnt, vb + qb + BCOST_BITS, s));
        k_bids<<<nblk(cnt), 256, 0, s>>>(k1, (uint32_t)cnt, vb, ids);
    }
    *out = ids;
    *count = (uint32_t)cnt;
    return EH_OK;
}

struct Host {
    std::vector<uint32_t> qidx;   // batch slot -> query index
};

// One device batch over the queries listed in `sel` (all with a subset).
// Writes counts/status for those queries.
eh_status run_batch(eh_trie *t, const eh_query *queries, const std::vector<uint32_t> &sel, const uint32_t *pool,
                    uint64_t pool_len, const eh_exec_opts &xo, cudaStream_t s, uint64_t *out_counts,
                    eh_status *out_status) {
    const uint32_t nq = (uint32_t)sel.size();
    if (nq == 0) return EH_OK;
    const double t_begin = now_s();
    NvtxRange nv("eh_count_batch: prepare + count");
    Scratch sc(s);
    const uint32_t n = t->n;
    // host tables
    std::vector<uint64_t> h_qoff(nq), h_qpos(nq);
    std::vector<uint32_t> h_qlen(nq), h_qpat(nq);
    uint64_t P = 0, lo = UINT64_MAX, hi = 0;
    for (uint32_t i = 0; i < nq; ++i) {
        const eh_query &qq = queries[sel[i]];
        h_qoff[i] = qq.subset_off;
        h_qlen[i] = qq.subset_len;
        h_qpos[i] = P;
        h_qpat[i] = qq.pattern;
        P += qq.subset_len;
        lo = std::min<uint64_t>(lo, qq.subset_off);
        hi = std::max<uint64_t>(hi, qq.subset_off + qq.subset_len);
    }
    for (uint32_t i = 0; i < nq; ++i) h_qoff[i] -= lo;
    // device copies of the pool slice and the tables
    uint32_t *d_pool = nullptr, *d_qlen = nullptr, *d_qpat = nullptr, *d_qstat = nullptr;
    uint64_t *d_qoff = nullptr, *d_qpos = nullptr;
    EH_TRY(sc.alloc(&d_pool, hi - lo));
    EH_TRY(sc.alloc(&d_qlen, nq));
    EH_TRY(sc.alloc(&d_qpat, nq));
    EH_TRY(sc.alloc(&d_qstat, nq));
    EH_TRY(sc.alloc(&d_qoff, nq));
    EH_TRY(sc.alloc(&d_qpos, nq));
    EH_CUDA_TRY(cudaMemcpyAsync(d_pool, pool + lo, (hi - lo) * 4, cudaMemcpyHostToDevice, s));
    EH_CUDA_TRY(cudaMemcpyAsync(d_qlen, h_qlen.data(), nq * 4, cudaMemcpyHostToDevice, s));
    EH_CUDA_TRY(cudaMemcpyAsync(d_qpat, h_qpat.data(), nq * 4, cudaMemcpyHostToDevice, s));
    EH_CUDA_TRY(cudaMemcpyAsync(d_qoff, h_qoff.data(), nq * 8, cudaMemcpyHostToDevice, s));
    EH_CUDA_TRY(cudaMemcpyAsync(d_qpos, h_qpos.data(), nq * 8, cudaMemcpyHostToDevice, s));
    EH_CUDA_TRY(cudaMemsetAsync(d_qstat, 0, nq * 4, s));

    // 1. keys, sort, unique
    const int nb = t->nb, qb = bits_of((uint64_t)nq + 1);
    if (nb + qb > 63) { eh_set_error("batch: too many queries for the id width"); return EH_EINVAL; }
    uint64_t *keys = nullptr, *keys2 = nullptr;
    EH_TRY(sc.alloc(&keys, P));
    EH_TRY(sc.alloc(&keys2, P));
    k_sub_keys<<<nq, 256, 0, s>>>(d_pool, d_qoff, d_qlen, d_qpos, t->d_old2new, n, nb, keys, d_qstat);
    EH_TRY(dev_radix_sort_u64(&keys, &keys2, P, nb + qb, s));
    uint32_t *flags = nullptr, *fpos = nullptr;
    EH_TRY(sc.alloc(&flags, P));
    EH_TRY(sc.alloc(&fpos, P));
    k_sub_flags<<<nblk(P), 256, 0, s>>>(keys, P, d_qstat, nb, flags);
    uint64_t V64 = 0;
    EH_TRY(dev_exclusive_scan_u32(flags, fpos, P, s, &V64));
    const uint32_t V = (uint32_t)V64;
    uint32_t *sub_q = nullptr, *sub_v = nullptr, *qcnt = nullptr, *qbase = nullptr;
    EH_TRY(sc.alloc(&sub_q, V));
    EH_TRY(sc.alloc(&sub_v, V));
    EH_TRY(sc.alloc(&qcnt, (uint64_t)nq + 1));
    EH_TRY(sc.alloc(&qbase, (uint64_t)nq + 1));
    EH_CUDA_TRY(cudaMemsetAsync(qcnt, 0, ((uint64_t)nq + 1) * 4, s));
    k_sub_scatter<<<nblk(P), 256, 0, s>>>(keys, flags, fpos, P, nb, sub_q, sub_v, qcnt);
    EH_TRY(dev_exclusive_scan_u32(qcnt, qbase, (uint64_t)nq + 1, s, nullptr));

    // 2. membership bitmaps and ranks
    const uint64_t W = (((uint64_t)n + 31) / 32 + 3) & ~3ull;
    uint32_t *bm = nullptr, *rb = nullptr;
    EH_TRY(sc.alloc(&bm, W * nq));
    EH_TRY(sc.alloc(&rb, W * nq));
    EH_CUDA_TRY(cudaMemsetAsync(bm, 0, W * nq * 4, s));
    if (V) k_sub_bits<<<nblk(V), 256, 0, s>>>(sub_q, sub_v, V, W, bm);
    k_popc_words<<<nblk(W * nq), 256, 0, s>>>(bm, W * nq, rb);
    EH_TRY(dev_exclusive_scan_u32(rb, rb, W * nq, s, nullptr));

    // 3. induced pruned sets
    uint32_t *len = nullptr, *indeg = nullptr, *deg = nullptr;
    uint64_t *off = nullptr, *wide = nullptr;
    EH_TRY(sc.alloc(&len, V));
    EH_TRY(sc.alloc(&indeg, V));
    EH_TRY(sc.alloc(&deg, V));
    EH_TRY(sc.alloc(&off, (uint64_t)V + 1));
    EH_TRY(sc.alloc(&wide, (uint64_t)V + 1));
    TrieView tv = t->view();
    if (V) k_sub_sets<false><<<nblk(V, 8), 256, 0, s>>>(tv, sub_q, sub_v, V, W, bm, rb, qbase, nullptr, len, nullptr, nullptr);
    EH_CUDA_TRY(cudaMemsetAsync(wide, 0, ((uint64_t)V + 1) * 8, s));
    if (V) k_round4_b<<<nblk(V), 256, 0, s>>>(len, V, wide);
    uint64_t total = 0;
    EH_TRY(dev_exclusive_scan_u64(wide, off, (uint64_t)V + 1, s, &total));
    uint32_t *nbr = nullptr;
    EH_TRY(sc.alloc(&nbr, total));
    EH_CUDA_TRY(cudaMemsetAsync(nbr, 0xFF, (total ? total : 1) * 4, s));
    EH_CUDA_TRY(cudaMemsetAsync(indeg, 0, (uint64_t)(V ? V : 1) * 4, s));
    if (V) k_sub_sets<true><<<nblk(V, 8), 256, 0, s>>>(tv, sub_q, sub_v, V, W, bm, rb, qbase, off, len, nbr, indeg);
    if (V) k_add_u32<<<nblk(V), 256, 0, s>>>(len, indeg, V, deg);

    // 4. layouts
    SetDesc *desc = nullptr;
    EH_TRY(sc.alloc(&desc, V));
    uint32_t *words = nullptr;
    uint64_t n_words = 0;
    EH_TRY(eh_build_layouts(nbr, off, len, deg, V, t->opts.bitset_tau, t->opts.min_bitset_len, s, desc, &words,
                            &n_words, nullptr));
    sc.ptrs.push_back(words);

    BatchView bv;
    bv.desc = desc; bv.nbr = nbr; bv.words = words; bv.deg = deg; bv.sub_q = sub_q; bv.qbase = qbase;
    bv.qpat = d_qpat;
    bv.n_sub = V;
    bv.n_nbr = total;
    bv.n_words = n_words;
    bv.n_queries = nq;

    // 5. work lists
    uint64_t *cost = nullptr;
    EH_TRY(sc.alloc(&cost, V));
    if (V) k_bcost<<<nblk(V, 8), 256, 0, s>>>(bv, V, cost);
    // the queries ranked by total cost, heaviest first (the lists' outer order)
    unsigned long long *d_qc = nullptr;
    uint32_t *d_qrank = nullptr;
    EH_TRY(sc.alloc(&d_qc, nq));
    EH_TRY(sc.alloc(&d_qrank, nq));
    EH_CUDA_TRY(cudaMemsetAsync(d_qc, 0, (uint64_t)nq * 8, s));
    if (V) k_bqcost<<<nblk(V), 256, 0, s>>>(cost, sub_q, V, d_qc);
    std::vector<unsigned long long> h_qc(nq);
    std::vector<uint32_t> order(nq), h_qrank(nq);
    EH_CUDA_TRY(cudaMemcpyAsync(h_qc.data(), d_qc, (uint64_t)nq * 8, cudaMemcpyDeviceToHost, s));
    EH_CUDA_TRY(cudaStreamSynchronize(s));
    for (uint32_t i = 0; i < nq; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return h_qc[a] > h_qc[b]; });
    for (uint32_t r = 0; r < nq; ++r) h_qrank[order[r]] = r;
    EH_CUDA_TRY(cudaMemcpyAsync(d_qrank, h_qrank.data(), (uint64_t)nq * 4, cudaMemcpyHostToDevice, s));
    uint32_t *heavy = nullptr, *light = nullptr, n_heavy = 0, n_light = 0;
    EH_TRY(sorted_list(desc, cost, sub_q, d_qrank, nq, V, xo.light_max, 0, s, sc, &heavy, &n_heavy));
    EH_TRY(sorted_list(desc, cost, sub_q, d_qrank, nq, V, xo.light_max, 1, s, sc, &light, &n_light));

    // 4-clique arena when a materialised S may exceed the shared buffer
    uint32_t *dmax = nullptr;
    EH_TRY(sc.alloc(&dmax, 1));
    EH_CUDA_TRY(cudaMemsetAsync(dmax, 0, 4, s));
    if (V) k_max_b<<<nblk(V), 256, 0, s>>>(len, V, dmax);
    uint32_t maxlen = 0;
    EH_CUDA_TRY(cudaMemcpyAsync(&maxlen, dmax, 4, cudaMemcpyDeviceToHost, s));
    EH_CUDA_TRY(cudaStreamSynchronize(s));
    bool any_k4 = false;
    for (uint32_t i = 0; i < nq; ++i) any_k4 |= h_qpat[i] == EH_CLIQUE4;
    uint32_t *arena = nullptr;
    const uint64_t per_warp = ((uint64_t)maxlen + 3) & ~3ull;
    if (any_k4 && maxlen > K4_S_CAP) {
        uint32_t gw = 0;
        EH_TRY(eh_launch_batch(bv, heavy, n_heavy, light, n_light, xo, s, nullptr, nullptr, nullptr, nullptr, 0, &gw));
        EH_TRY(sc.alloc(&arena, per_warp * gw));
    }

    // 6. one persistent launch for the whole batch
    const double t_prepared = now_s();   // the stream is idle here (synchronised above)
    unsigned long long *d_out = nullptr, *d_cnt = nullptr;
    uint32_t *d_bst = nullptr;   // this batch's device status word
    EH_TRY(sc.alloc(&d_out, 2ull * nq));
    EH_TRY(sc.alloc(&d_cnt, 2));
    EH_TRY(sc.alloc(&d_bst, 1));
    // The count phase (clears + the one persistent launch) is captured in a
    // CUDA graph on this thread's capture stream and launched as a graph.  The
    // thread keeps one executable graph: each batch's capture updates it in
    // place (cudaGraphExecUpdate: same nodes, new launch parameters), and it is
    // instantiated again only when the update is refused.  The batches of a
    // thread run one after another (each ends with a synchronisation), so the
    // executable graph is idle whenever it is updated.
    static thread_local cudaStream_t cs = nullptr;
    static thread_local cudaEvent_t ready = nullptr;
    static thread_local cudaGraphExec_t gexec = nullptr;
    if (!cs) EH_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (!ready) EH_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    // every buffer above is ready on `s`: the capture stream waits for it on the device
    EH_CUDA_TRY(cudaEventRecord(ready, s));
    EH_CUDA_TRY(cudaStreamWaitEvent(cs, ready, 0));
    cudaGraph_t graph = nullptr;
    EH_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    eh_status lst = EH_OK;
    if (cudaMemsetAsync(d_out, 0, 16ull * nq, cs) != cudaSuccess || cudaMemsetAsync(d_bst, 0, 4, cs) != cudaSuccess)
        lst = EH_ECUDA;
    if (lst == EH_OK)
        lst = eh_launch_batch(bv, heavy, n_heavy, light, n_light, xo, cs, d_out, d_cnt, d_bst, arena, per_warp,
                              nullptr);
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (lst != EH_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (lst == EH_OK) eh_set_error("batch graph capture: %s", cudaGetErrorString(ce));
        return lst != EH_OK ? lst : EH_ECUDA;
    }
    ce = cudaSuccess;
    if (gexec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(gexec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(gexec);
            gexec = nullptr;
        } else {
            g_prof.graph_reuses += 1;
        }
    }
    if (!gexec) ce = cudaGraphInstantiate(&gexec, graph, 0);
    if (ce == cudaSuccess) ce = cudaGraphLaunch(gexec, cs);
    std::vector<unsigned long long> h_out(2ull * nq);
    std::vector<uint32_t> h_stat(nq);
    uint32_t bst = 0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_out.data(), d_out, 16ull * nq, cudaMemcpyDeviceToHost, cs);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_stat.data(), d_qstat, 4ull * nq, cudaMemcpyDeviceToHost, cs);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&bst, d_bst, 4, cudaMemcpyDeviceToHost, cs);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(cs);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess && gexec) {
        cudaGraphExecDestroy(gexec);
        gexec = nullptr;
    }
    if (ce != cudaSuccess) {
        eh_set_error("batch count graph: %s", cudaGetErrorString(ce));
        return EH_ECUDA;
    }
    const double t_done = now_s();
    g_prof.queries += nq;
    g_prof.sub_vertices += V;
    g_prof.sub_set_elements += total;
    g_prof.heavy_items += n_heavy;
    g_prof.light_items += n_light;
    g_prof.prepare_s += t_prepared - t_begin;
    g_prof.count_s += t_done - t_prepared;
    g_prof.batches += 1;
    eh_status dst = EH_OK;
    if (bst & DEV_ST_TIMEOUT) { dst = EH_ETIMEOUT; eh_set_error("a bounded device wait timed out"); }
    else if (bst) { dst = EH_ECUDA; eh_set_error("batch kernel reported status 0x%x", bst); }
    for (uint32_t i = 0; i < nq; ++i) {
        const uint32_t qi = sel[i];
        if (dst != EH_OK) { out_status[qi] = dst; out_counts[qi] = 0; continue; }
        if (h_stat[i]) { out_status[qi] = EH_EINVAL; out_counts[qi] = 0; continue; }
        const unsigned long long T = h_out[2 * i], S = h_out[2 * i + 1];
        uint64_t r = 0;
        eh_status qs = EH_OK;
        switch (h_qpat[i]) {
            case EH_TRIANGLE: r = T; break;
            case EH_CLIQUE4: r = T; break;
            case EH_LOLLIPOP:
                if (S >> 63) qs = EH_EOVERFLOW;
                r = 2ull * S;
                break;
            default: r = S - 6ull * T; break;
        }
        out_counts[qi] = r;
        out_status[qi] = qs;
    }
    return dst;
}

}  // namespace

extern "C" eh_status eh_count_batch_ex(const eh_trie *trie, const eh_query *queries, uint32_t n_queries,
                                       const uint32_t *subset_pool, uint64_t pool_len, const eh_exec_opts *xopts,
                                       uint32_t mode, void *stream, uint64_t *out_counts, eh_status *out_status) {
    if (!trie || (n_queries && (!queries || !out_counts || !out_status))) {
        eh_set_error("eh_count_batch: NULL argument");
        return EH_EINVAL;
    }
    eh_trie *t = const_cast<eh_trie *>(trie);
    cudaStream_t s = (cudaStream_t)stream;
    const eh_exec_opts xo = eh_exec_defaults(xopts);
    memset(&g_prof, 0, sizeof(g_prof));
    std::vector<uint32_t> subset_q, whole_q;
    eh_status first = EH_OK;
    for (uint32_t i = 0; i < n_queries; ++i) {
        out_counts[i] = 0;
        const eh_query &q = queries[i];
        bool ok = (q.pattern <= EH_LOLLIPOP_DISTINCT || (q.pattern == EH_BARBELL && q.subset_len == 0)) &&
                  (q.subset_len == 0 || (subset_pool && q.subset_off + q.subset_len <= pool_len &&
                                         q.subset_off + q.subset_len >= q.subset_off));
        out_status[i] = ok ? EH_OK : EH_EINVAL;
        if (!ok) { if (first == EH_OK) { first = EH_EINVAL; eh_set_error("query %u: bad pattern or subset range", i); } continue; }
        (q.subset_len ? subset_q : whole_q).push_back(i);
    }
    if (!subset_q.empty()) {   // subset batches own all their device state: no lock
        eh_status st = EH_OK;
        if (mode == 1) {
            for (uint32_t qi : subset_q) {
                std::vector<uint32_t> one(1, qi);
                eh_status r = run_batch(t, queries, one, subset_pool, pool_len, xo, s, out_counts, out_status);
                if (r != EH_OK) { out_status[qi] = r; if (st == EH_OK) st = r; }
            }
        } else {
            st = run_batch(t, queries, subset_q, subset_pool, pool_len, xo, s, out_counts, out_status);
            if (st != EH_OK)
                for (uint32_t qi : subset_q)
                    if (out_status[qi] == EH_OK) out_status[qi] = st;
        }
        if (st != EH_OK && first == EH_OK) first = st;
    }
    std::unique_lock<std::mutex> g(t->call_mu, std::defer_lock);
    if (!whole_q.empty()) g.lock();   // whole-graph counts share the trie's scratch
    for (uint32_t qi : whole_q) {
        unsigned long long *d_out = t->d_scratch + 15;
        eh_status r = eh_enqueue_whole(t, (eh_pattern)queries[qi].pattern, xo, s, d_out);
        unsigned long long v = 0;
        if (r == EH_OK && cudaMemcpyAsync(&v, d_out, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) r = EH_ECUDA;
        if (r == EH_OK) r = eh_check_status(t, s);
        out_counts[qi] = r == EH_OK ? v : 0;
        out_status[qi] = r;
        if (r != EH_OK && first == EH_OK) first = r;
    }
    for (uint32_t i = 0; i < n_queries; ++i)
        if (out_status[i] != EH_OK && first == EH_OK) first = out_status[i];
    return first;
}

extern "C" eh_status eh_count_batch(const eh_trie *trie, const eh_query *queries, uint32_t n_queries,
                                    const uint32_t *subset_pool, uint64_t pool_len, void *stream, uint64_t *out_counts,
                                    eh_status *out_status) {
    return eh_count_batch_ex(trie, queries, n_queries, subset_pool, pool_len, nullptr, 0, stream, out_counts,
                             out_status);
}

eh_status eh_count_subset(const eh_trie *trie, eh_pattern pattern, const uint32_t *subset, uint32_t subset_len,
                          const eh_exec_opts *xopts, void *stream, uint64_t *out_count) {
    eh_query q;
    q.pattern = (uint32_t)pattern;
    q.subset_len = subset_len;
    q.subset_off = 0;
    eh_status st = EH_OK;
    eh_status r = eh_count_batch_ex(trie, &q, 1, subset, subset_len, xopts, 0, stream, out_count, &st);
    return r != EH_OK ? r : st;
}

extern "C" eh_status eh_batch_profile_get(eh_batch_profile *out) {
    if (!out) { eh_set_error("eh_batch_profile_get: NULL argument"); return EH_EINVAL; }
    *out = g_prof;
    return EH_OK;
}
