// plan.cu -- the per-vertex work list of the pruned trie (cost estimate,
// light/heavy split by |N+(u)|, heavy items by factor-2 cost class, heaviest
// first, then by locality), the split of its lists into
// cost-balanced ranges for counts divided among workers, and, on request,
// the algorithmic byte counts of one pass (triangle lower bound, triangle at
// the stored layouts' sizes, 4-clique lower bound).
#include "eh_internal.cuh"

namespace {

// |N+(v)| of every vertex as a compact array (4 bytes a vertex instead of a
// 32-byte descriptor: the cost pass gathers it once per pair)
__global__ void k_out_len(const SetDesc *__restrict__ desc, uint32_t n, uint32_t *len) {
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) len[v] = desc[v].len;
}

// one warp per vertex: cost(u) = sum_{v in N+(u)} |N+(v)|, the cost classes
// of the heavy list and the balance of range splits
__global__ void k_cost(const SetDesc *__restrict__ desc, const uint32_t *__restrict__ nbr,
                       const uint32_t *__restrict__ len, uint32_t n, uint64_t *cost) {
    const uint32_t u = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (u >= n) return;
    const SetDesc du = desc[u];
    uint64_t c = 0;
    for (uint32_t j = lane; j < du.len; j += 32) c += __ldg(&len[__ldg(&nbr[du.off + j])]);
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if (lane == 0) cost[u] = c;
}

// one warp per vertex: the bytes the method must move for u: A = N+(u) once
// (its cheaper stored form), then per pair (u, v = A[j]) the cheapest way to
// read what of B = N+(v) can meet A_<v: the uint array (4|B| bytes; at most 32
// bytes per probe of the j elements of A_<v when |B| > ratio*j, the galloping
// side), or the bitset words overlapping A's value range (at most 32 bytes per
// probe of A_<v).  A lower bound on what any of the kernel's dispatch choices
// reads; a reported figure that no count needs, so it runs on request only.
__global__ void k_alg_bytes(TrieView tv, uint32_t n, uint32_t ratio, unsigned long long *bytes_acc) {
    uint32_t u = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (u >= n) return;
    SetDesc du = tv.desc[u];
    uint64_t b = 0;
    if (du.len >= 2) {
        const uint32_t first = tv.nbr[du.off], last = tv.nbr[du.off + du.len - 1];
        const uint32_t a_lo = (first >> 7) << 2, a_hi = (last >> 5) + 1;   // A's word range
        for (uint32_t j = lane; j < du.len; j += 32) {
            uint32_t v = tv.nbr[du.off + j];
            SetDesc dv = tv.desc[v];
            if (j == 0 || dv.len == 0) continue;
            uint64_t bb = 4ull * dv.len;
            if ((uint64_t)dv.len > (uint64_t)ratio * j && 32ull * j < bb) bb = 32ull * j;
            if (dv.nwords) {
                uint32_t lo = a_lo > dv.lo_word ? a_lo : dv.lo_word;
                uint32_t hi = a_hi < dv.lo_word + dv.nwords ? a_hi : dv.lo_word + dv.nwords;
                uint64_t wb = hi > lo ? 4ull * (hi - lo) : 0ull;
                if (32ull * j < wb) wb = 32ull * j;
                if (wb < bb) bb = wb;
            }
            b += bb;
        }
        if (lane == 0) b += du.nwords && du.nwords < du.len ? 4ull * du.nwords : 4ull * du.len;
    }
    for (int d = 16; d > 0; d >>= 1) b += __shfl_xor_sync(0xffffffffu, b, d);
    if (lane == 0 && b) atomicAdd(bytes_acc, (unsigned long long)b);
}

// one warp per vertex: the same pass counted with every set at its stored
// layout's size -- bytes(X) = 4|X| for a uint set, 4 x its words for a bitset
// set -- and the pair (u, v) read as N+(u) ∩ N+(v) in full: u's set once,
// then per v in N+(u) the bytes of N+(v), or at most 32 bytes per element of
// N+(u) when |N+(v)| > ratio |N+(u)| (the galloping side).  Reported next to
// the lower bound above.
__global__ void k_alg_bytes_stored(TrieView tv, uint32_t n, uint32_t ratio, unsigned long long *bytes_acc) {
    const uint32_t u = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (u >= n) return;
    const SetDesc du = tv.desc[u];
    uint64_t b = 0;
    for (uint32_t j = lane; j < du.len; j += 32) {
        const SetDesc dv = tv.desc[tv.nbr[du.off + j]];
        uint64_t bb = dv.nwords ? 4ull * dv.nwords : 4ull * dv.len;
        if ((uint64_t)dv.len > (uint64_t)ratio * du.len && 32ull * du.len < bb) bb = 32ull * du.len;
        b += bb;
    }
    if (lane == 0) b += du.nwords ? 4ull * du.nwords : 4ull * du.len;
    for (int d = 16; d > 0; d >>= 1) b += __shfl_xor_sync(0xffffffffu, b, d);
    if (lane == 0 && b) atomicAdd(bytes_acc, (unsigned long long)b);
}

// the per-warp shared buffer of S in the 4-clique kernels (K4_S_CAP): a
// longer S is written to and read back from device memory
constexpr uint32_t K4_SPILL_FROM = K4_S_CAP;

// bytes of the pair (P, N+(z)) with P a set held on chip: r elements, words
// [p_lo, p_hi) of the value domain; the lower-bound reading of k_alg_bytes
__device__ __forceinline__ uint64_t pair_bytes(const SetDesc &dz, uint32_t r, uint32_t p_lo, uint32_t p_hi,
                                               uint32_t ratio) {
    uint64_t bb = 4ull * dz.len;
    if ((uint64_t)dz.len > (uint64_t)ratio * r && 32ull * r < bb) bb = 32ull * r;
    if (dz.nwords) {
        const uint32_t lo = p_lo > dz.lo_word ? p_lo : dz.lo_word;
        const uint32_t hi = p_hi < dz.lo_word + dz.nwords ? p_hi : dz.lo_word + dz.nwords;
        uint64_t wb = hi > lo ? 4ull * (hi - lo) : 0ull;
        if (32ull * r < wb) wb = 32ull * r;
        if (wb < bb) bb = wb;
    }
    return bb;
}

// one CTA per x: the bytes one 4-clique pass must move (Table 1's 4Clique,
// x > y > z > w).  A = N+(x) once, in its cheaper stored form; level 1 per
// (x, y = A[j]), j >= 2, |N+(y)| >= 2: the pair (A_<y, N+(y)) as in
// k_alg_bytes; level 2 per z = S[r], r >= 1, of S = A ∩ N+(y): the pair
// (S_<z, N+(z)), S_<z held on chip (r elements, words from S[0]'s down to
// S[r-1]'s); plus 8 bytes per element of S (written and read back) when S is
// longer than the on-chip buffer.  S is found by scanning N+(y) in rounds of
// 32 with a binary search of each element in A.
__global__ void k_alg_bytes_k4(TrieView tv, uint32_t n, uint32_t ratio, unsigned long long *bytes_acc) {
    const uint32_t x = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (x >= n) return;
    const SetDesc dx = tv.desc[x];
    if (dx.len < 3) return;
    const uint32_t *A = tv.nbr + dx.off;
    const uint32_t a_lo = (A[0] >> 7) << 2, a_hi = (A[dx.len - 1] >> 5) + 1;
    uint64_t b = 0;
    if (threadIdx.x == 0) b += dx.nwords && dx.nwords < dx.len ? 4ull * dx.nwords : 4ull * dx.len;
    for (uint32_t j = 2 + warp; j < dx.len; j += nwarps) {
        const SetDesc dy = tv.desc[A[j]];
        if (dy.len < 2) continue;
        if (lane == 0) b += pair_bytes(dy, j, a_lo, a_hi, ratio);
        const uint32_t *B = tv.nbr + dy.off;
        uint32_t ns = 0, s0 = 0, prev = 0;
        for (uint32_t c = 0; c < dy.len; c += 32) {
            const uint32_t i = c + lane;
            const uint32_t e = i < dy.len ? B[i] : 0u;
            bool hit = false;
            if (i < dy.len) {
                uint32_t lo = 0, hi = j;   // e < A[j]: only A_<y can hold it
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (A[mid] < e) lo = mid + 1; else hi = mid;
                }
                hit = lo < j && A[lo] == e;
            }
            const uint32_t m = __ballot_sync(0xffffffffu, hit);
            if (!m) continue;
            if (ns == 0) s0 = __shfl_sync(0xffffffffu, e, __ffs(m) - 1);
            const uint32_t below = m & ((1u << lane) - 1u);
            // the element before this lane's in S: a lower lane's, or the last of earlier rounds
            const uint32_t pl = below ? 31u - __clz(below) : 0u;
            const uint32_t pe = __shfl_sync(0xffffffffu, e, pl);
            if (hit) {
                const uint32_t r = ns + __popc(below);
                const uint32_t before = below ? pe : prev;
                if (r >= 1) {
                    const SetDesc dz = tv.desc[e];
                    if (dz.len) b += pair_bytes(dz, r, (s0 >> 7) << 2, (before >> 5) + 1, ratio);
                }
            }
            ns += __popc(m);
            prev = __shfl_sync(0xffffffffu, e, 31 - __clz(m));
        }
        if (lane == 0 && ns > K4_SPILL_FROM) b += 8ull * ns;
    }
    for (int d = 16; d > 0; d >>= 1) b += __shfl_xor_sync(0xffffffffu, b, d);
    if (lane == 0 && b) atomicAdd(bytes_acc, (unsigned long long)b);
}

// cost of the items of a list, in list order
__global__ void k_gather_cost(const uint32_t *__restrict__ ids, uint32_t cnt, const uint64_t *__restrict__ cost,
                              uint64_t *out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) out[i] = cost[ids[i]];
}

// class 0: heavy (len > light_max), 1: light (2 <= len <= light_max)
__global__ void k_class_flags(TrieView tv, uint32_t n, uint32_t light_max, int cls, uint32_t *flags) {
    uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    uint32_t len = tv.desc[u].len;
    bool f = cls == 0 ? len > light_max : (len >= 2 && len <= light_max);
    flags[u] = f ? 1u : 0u;
}

// cost on a 14-bit logarithmic scale: the exponent and the next 8 bits
// (monotone in the cost, 0.3% resolution: enough to put the heaviest first)
constexpr int COST_BITS = 14;

__global__ void k_class_keys(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos,
                             const uint64_t *__restrict__ cost, uint32_t n, int nb, uint64_t *keys) {
    uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n || !flags[u]) return;
    const uint64_t c = cost[u];
    uint32_t q = 0;
    if (c) {
        const int msb = 63 - __clzll((long long)c);
        q = (uint32_t)msb * 256u + (uint32_t)(((c << (63 - msb)) >> 55) & 255u);
    }
    const uint64_t qmax = (1ull << COST_BITS) - 1;
    keys[pos[u]] = ((qmax - q) << nb) | u;   // ascending key = descending cost
}

// Locality order of the work lists.  Heavy items in factor-2 cost classes,
// heaviest class first (the long items start early, the tail stays short),
// and inside a class by the last (largest) element of N+(u); light items by
// the last element of N+(u).  CTAs and warps that run at the same time then
// hold vertices whose sets reach the same neighbour ids, and the sets of
// those neighbours that their pairs read, N+(v) for v in N+(u), are shared
// in L2 (R-MAT-22 triangle count: 9.21 ms against 9.34 ms with both lists
// by cost alone).  Key: (class, last element, u), 2 nb + 6 bits.  Only lists
// long enough to hold many items per resident warp (light) or CTA (heavy)
// take this order: a short list runs in about one wave, where locality buys
// nothing and the heaviest-first order keeps the tail short (an ER graph of
// 10^4 vertices: 0.034 ms by cost, 0.037 ms in locality order).
constexpr uint64_t LOCALITY_MIN_PER_SM[2] = {256, 2048};   // heavy, light items per SM
__global__ void k_locality_keys(TrieView tv, const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos,
                                const uint64_t *__restrict__ cost, uint32_t n, int nb, int cls, uint64_t *keys) {
    uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n || !flags[u]) return;
    const SetDesc d = tv.desc[u];   // len >= 1 in both classes
    const uint64_t last = tv.nbr[d.off + d.len - 1];
    uint64_t c2 = 0;
    if (cls == 0) {
        const uint64_t c = cost[u];
        c2 = 63u - (c ? (uint32_t)(63 - __clzll((long long)c)) : 0u);
    }
    keys[pos[u]] = (((c2 << nb) | last) << nb) | u;
}

__global__ void k_key_ids(const uint64_t *__restrict__ keys, uint32_t cnt, int nb, uint32_t *ids) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) ids[i] = (uint32_t)(keys[i] & ((1ull << nb) - 1));
}

eh_status make_list(TrieView tv, uint32_t n, int nb, uint32_t light_max, int cls, const uint64_t *cost,
                    cudaStream_t s, uint32_t **out, uint32_t *count) {
    *out = nullptr;
    *count = 0;
    uint32_t *flags = nullptr, *pos = nullptr;
    EH_TRY(dev_alloc(&flags, n, s));
    eh_status st = dev_alloc(&pos, n, s);
    if (st != EH_OK) { dev_free(flags, s); return st; }
    unsigned blocks = (n + 255) / 256;
    uint64_t cnt = 0;
    if (n) k_class_flags<<<blocks, 256, 0, s>>>(tv, n, light_max, cls, flags);
    st = dev_exclusive_scan_u32(flags, pos, n, s, &cnt);
    uint64_t *k1 = nullptr, *k2 = nullptr;
    if (st == EH_OK) st = dev_alloc(&k1, cnt, s);
    if (st == EH_OK) st = dev_alloc(&k2, cnt, s);
    if (st == EH_OK && cnt) {
        if (2 * nb + 6 <= 64 && cnt >= LOCALITY_MIN_PER_SM[cls] * (uint64_t)eh_num_sms()) {
            k_locality_keys<<<blocks, 256, 0, s>>>(tv, flags, pos, cost, n, nb, cls, k1);
            st = dev_radix_sort_u64(&k1, &k2, cnt, 2 * nb + 6, s);
        } else {   // a short list, or ids too wide for the locality key: by cost alone
            k_class_keys<<<blocks, 256, 0, s>>>(flags, pos, cost, n, nb, k1);
            st = dev_radix_sort_u64(&k1, &k2, cnt, nb + COST_BITS, s);
        }
    }
    uint32_t *ids = nullptr;
    if (st == EH_OK) {
        cudaError_t e = eh_alloc_should_fail() ? cudaErrorMemoryAllocation
                                               : cudaMalloc((void **)&ids, (cnt ? cnt : 1) * 4);
        if (e != cudaSuccess) { cudaGetLastError(); eh_set_error("work list allocation failed"); st = EH_ENOMEM; }
    }
    if (st == EH_OK && cnt) k_key_ids<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(k1, (uint32_t)cnt, nb, ids);
    dev_free(k1, s);
    dev_free(k2, s);
    dev_free(flags, s);
    dev_free(pos, s);
    if (st != EH_OK) { cudaFree(ids); return st; }
    *out = ids;
    *count = (uint32_t)cnt;
    return EH_OK;
}

}  // namespace

eh_status eh_plan_get(eh_trie *t, uint32_t light_max, cudaStream_t s, WorkPlan **out) {
    std::lock_guard<std::mutex> g(t->mu);
    auto it = t->plans.find(light_max);
    if (it != t->plans.end()) { *out = &it->second; return EH_OK; }
    NvtxRange nv("eh work plan");
    WorkPlan p;
    p.light_max = light_max;
    TrieView tv = t->view();
    uint64_t *cost = nullptr;
    uint32_t *olen = nullptr;
    EH_TRY(dev_alloc(&cost, t->n, s));
    eh_status st = dev_alloc(&olen, t->n, s);
    if (st == EH_OK) {
        if (t->n) {
            k_out_len<<<(t->n + 255) / 256, 256, 0, s>>>(t->d_desc, t->n, olen);
            k_cost<<<(t->n + 7) / 8, 256, 0, s>>>(t->d_desc, t->d_onbr, olen, t->n, cost);
        }
        st = make_list(tv, t->n, t->nb, light_max, 0, cost, s, &p.d_heavy, &p.n_heavy);
    }
    if (st == EH_OK) st = make_list(tv, t->n, t->nb, light_max, 1, cost, s, &p.d_light, &p.n_light);
    if (st == EH_OK && t->d_boff) st = eh_plan_blocks(t, &p, s);
    if (st == EH_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        eh_set_error("plan: %s", cudaGetErrorString(cudaGetLastError()));
        st = EH_ECUDA;
    }
    dev_free(olen, s);
    if (st != EH_OK) {
        dev_free(cost, s);
        cudaFree(p.d_heavy);
        cudaFree(p.d_light);
        cudaFree(p.d_heavy_blk);
        return st;
    }
    p.d_cost = cost;      // kept: the range counts split the lists by it
    auto res = t->plans.emplace(light_max, p);
    *out = &res.first->second;
    return EH_OK;
}

eh_status eh_plan_alg_bytes(eh_trie *t, WorkPlan *p, cudaStream_t s, int which, double *out) {
    std::lock_guard<std::mutex> g(t->mu);
    double *slot = which == ALG_K4 ? &p->alg_bytes_k4 : which == ALG_TRI_STORED ? &p->alg_bytes_stored : &p->alg_bytes;
    if (*slot < 0) {
        unsigned long long *bytes_d = nullptr, bytes_h = 0;
        EH_TRY(dev_alloc(&bytes_d, 1, s));
        eh_status st = EH_OK;
        if (cudaMemsetAsync(bytes_d, 0, 8, s) != cudaSuccess) st = EH_ECUDA;
        if (st == EH_OK && t->n) {
            if (which == ALG_K4) k_alg_bytes_k4<<<t->n, 256, 0, s>>>(t->view(), t->n, 32, bytes_d);
            else if (which == ALG_TRI_STORED)
                k_alg_bytes_stored<<<(t->n + 7) / 8, 256, 0, s>>>(t->view(), t->n, 32, bytes_d);
            else k_alg_bytes<<<(t->n + 7) / 8, 256, 0, s>>>(t->view(), t->n, 32, bytes_d);
        }
        if (st == EH_OK && (cudaMemcpyAsync(&bytes_h, bytes_d, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                            cudaStreamSynchronize(s) != cudaSuccess)) {
            eh_set_error("algorithmic bytes: %s", cudaGetErrorString(cudaGetLastError()));
            st = EH_ECUDA;
        }
        dev_free(bytes_d, s);
        EH_TRY(st);
        *slot = (double)bytes_h + 8.0 * (double)t->m;
    }
    *out = *slot;
    return EH_OK;
}

void eh_split_range(const uint64_t *pre, uint64_t n, uint32_t part, uint32_t nparts, uint64_t *lo, uint64_t *hi) {
    // b(q) = the first i in [0, n] with pre[i] * nparts >= q * total; b(nparts) = n
    const unsigned __int128 total = pre[n];
    auto bound = [&](uint32_t q) -> uint64_t {
        if (q == 0) return 0;
        if (q >= nparts) return n;
        const unsigned __int128 target = total * q;
        uint64_t a = 0, b = n;
        while (a < b) {
            const uint64_t mid = a + (b - a) / 2;
            if ((unsigned __int128)pre[mid] * nparts >= target) b = mid; else a = mid + 1;
        }
        return a;
    };
    *lo = bound(part);
    *hi = bound(part + 1);
}

eh_status eh_plan_cost_prefix(eh_trie *t, WorkPlan *p, cudaStream_t s) {
    std::lock_guard<std::mutex> g(t->mu);
    if (p->h_heavy_pre.size() == (size_t)p->n_heavy + 1 && p->h_light_pre.size() == (size_t)p->n_light + 1)
        return EH_OK;
    const uint32_t cnt = p->n_heavy > p->n_light ? p->n_heavy : p->n_light;
    uint64_t *d = nullptr;
    EH_TRY(dev_alloc(&d, cnt, s));
    std::vector<uint64_t> hc[2];
    const uint32_t *ids[2] = {p->d_heavy, p->d_light};
    const uint32_t ns[2] = {p->n_heavy, p->n_light};
    eh_status st = EH_OK;
    for (int k = 0; k < 2 && st == EH_OK; ++k) {
        hc[k].assign((size_t)ns[k] + 1, 0);
        if (!ns[k]) continue;
        k_gather_cost<<<(ns[k] + 255) / 256, 256, 0, s>>>(ids[k], ns[k], p->d_cost, d);
        if (cudaMemcpyAsync(hc[k].data() + 1, d, (uint64_t)ns[k] * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            eh_set_error("range split: %s", cudaGetErrorString(cudaGetLastError()));
            st = EH_ECUDA;
        }
        for (uint32_t i = 1; i <= ns[k]; ++i) hc[k][i] += hc[k][i - 1];   // exclusive prefix at i
    }
    dev_free(d, s);
    EH_TRY(st);
    p->h_heavy_pre.swap(hc[0]);
    p->h_light_pre.swap(hc[1]);
    return EH_OK;
}
