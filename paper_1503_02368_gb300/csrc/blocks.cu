// blocks.cu -- the composite (block-level) set layout of Sec. 4.3 and the
// triangle count over it.
//
// The value domain is cut into blocks of 256 values.  A pruned set N+(v)
// keeps its sorted uint array; a directory lists the blocks it touches in
// ascending block id, each either a 256-bit bitset (8 words in a pool) when
// the block holds c values with 256 <= tau * c, or the run of the uint array
// holding its values.  Directory entry {id, info}:
//   info bit 31 set:   bitset block, bits 0..30 = its index in the word pool
//   info bit 31 clear: uint block, bits 0..22 = first position of the run in
//                      the set's uint array, bits 23..30 = run length - 1
// A trie built with EH_BUILD_BLOCK_LAYOUT holds these directories instead of
// set-level bitsets.  Its triangle count intersects two sets by their
// directories, the block ids treated as a uint set (Sec. 4.2): each id of one
// directory is found in the other by binary search (in shared memory, where
// u's directory is staged), and matching blocks are intersected by their
// layout pair: AND + popcount of 8 words, bit probes of a run's values, or a
// merge of two runs.
#include "eh_internal.cuh"

#include <algorithm>

namespace {

constexpr uint32_t BLK_BIT = 0x80000000u;

// persistent trie memory: from the default pool like the trie's other arrays
template <typename T>
eh_status trie_alloc(T **p, uint64_t count, cudaStream_t s) {
    *p = nullptr;
    if (eh_alloc_should_fail()) { eh_set_error("device allocation failed (injected)"); return EH_ENOMEM; }
    if (cudaMallocAsync((void **)p, sizeof(T) * (count ? count : 1), s) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        eh_set_error("device allocation of %llu bytes failed", (unsigned long long)(sizeof(T) * count));
        return EH_ENOMEM;
    }
    return EH_OK;
}

__device__ __forceinline__ bool is_bitset_block(uint32_t tau, uint32_t c) {
    return tau == 0xFFFFFFFFu || (tau != 0 && (uint64_t)tau * c >= 256);
}

// one thread per set: blocks touched and bitset blocks among them
__global__ void k_blk_count(const uint32_t *__restrict__ nbr, const SetDesc *__restrict__ desc, uint32_t n,
                            uint32_t tau, uint64_t *nblk, uint64_t *nbit) {
    const uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const SetDesc d = desc[v];
    const uint32_t *S = nbr + d.off;
    uint64_t nb = 0, nbits = 0;
    uint32_t i = 0;
    while (i < d.len) {
        const uint32_t b = S[i] >> 8;
        uint32_t c = 0;
        while (i < d.len && (S[i] >> 8) == b) { ++c; ++i; }
        ++nb;
        nbits += is_bitset_block(tau, c);
    }
    nblk[v] = nb;
    nbit[v] = nbits;
}

__global__ void k_blk_fill(const uint32_t *__restrict__ nbr, const SetDesc *__restrict__ desc, uint32_t n,
                           uint32_t tau, const uint64_t *__restrict__ boff, const uint64_t *__restrict__ bitoff,
                           uint2 *dir, uint32_t *words) {
    const uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const SetDesc d = desc[v];
    const uint32_t *S = nbr + d.off;
    uint64_t k = boff[v], kb = bitoff[v];
    uint32_t i = 0;
    while (i < d.len) {
        const uint32_t b = S[i] >> 8, start = i;
        while (i < d.len && (S[i] >> 8) == b) ++i;
        const uint32_t c = i - start;
        if (is_bitset_block(tau, c)) {
            uint32_t *w = words + kb * 8;
            for (uint32_t j = start; j < i; ++j) w[(S[j] & 255) >> 5] |= 1u << (S[j] & 31);
            dir[k] = make_uint2(b, BLK_BIT | (uint32_t)kb);
            ++kb;
        } else {
            dir[k] = make_uint2(b, start | ((c - 1) << 23));
        }
        ++k;
    }
}

// |block a ∩ block b| for two directory entries of the same block id
__device__ __forceinline__ uint32_t block_meet(uint32_t ia, const uint32_t *Sa, uint32_t ib, const uint32_t *Sb,
                                               const uint32_t *__restrict__ words) {
    const bool ba = ia & BLK_BIT, bb = ib & BLK_BIT;
    if (ba && bb) {
        const uint4 *wa = reinterpret_cast<const uint4 *>(words + (uint64_t)(ia & ~BLK_BIT) * 8);
        const uint4 *wb = reinterpret_cast<const uint4 *>(words + (uint64_t)(ib & ~BLK_BIT) * 8);
        uint32_t c = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 x = __ldg(wa + h), y = __ldg(wb + h);
            c += __popc(x.x & y.x) + __popc(x.y & y.y) + __popc(x.z & y.z) + __popc(x.w & y.w);
        }
        return c;
    }
    if (ba || bb) {   // a run's values probe the other block's bits
        const uint32_t ibit = ba ? ia : ib, irun = ba ? ib : ia;
        const uint32_t *Sr = ba ? Sb : Sa;
        const uint32_t *w = words + (uint64_t)(ibit & ~BLK_BIT) * 8;
        const uint32_t start = irun & 0x7FFFFFu, len = ((irun >> 23) & 0xFFu) + 1;
        uint32_t c = 0;
        for (uint32_t j = 0; j < len; ++j) {
            const uint32_t x = __ldg(&Sr[start + j]) & 255;
            c += (__ldg(&w[x >> 5]) >> (x & 31)) & 1u;
        }
        return c;
    }
    // two runs: merge
    const uint32_t *p = Sa + (ia & 0x7FFFFFu), *q = Sb + (ib & 0x7FFFFFu);
    const uint32_t la = ((ia >> 23) & 0xFFu) + 1, lb = ((ib >> 23) & 0xFFu) + 1;
    uint32_t i = 0, j = 0, c = 0;
    while (i < la && j < lb) {
        const uint32_t x = __ldg(&p[i]), y = __ldg(&q[j]);
        c += x == y;
        i += x <= y;
        j += y <= x;
    }
    return c;
}

constexpr uint32_t FULL = 0xffffffffu;
constexpr int BLK_WARPS = 8;                       // warps per CTA of the block-layout count
constexpr uint32_t U_CAP = 512;                    // directory entries of u a warp stages
constexpr uint32_t CTA_CAP = BLK_WARPS * U_CAP;    // ... a CTA stages for a big item (same buffer)
constexpr uint32_t BIG_LEN = 256;                  // an item with a longer N+(u) is big: one CTA
constexpr uint32_t SKEW = 8;                       // a v directory longer than SKEW x u's and than
constexpr uint32_t SKEW_MIN = 256;                 // SKEW_MIN entries is searched, not walked

// a warp's batch of 32 v's
struct BlkBatch {
    unsigned long long vb[32];       // first directory entry of each v
    uint32_t pre[32];                // exclusive prefix of the walked directory lengths
    uint32_t voff[32];               // offset of each v's uint array
};

// smallest index i in [0, n) with d[i].x >= id, or n
__device__ __forceinline__ uint32_t dir_lower_bound(const uint2 *d, uint32_t n, uint32_t id) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (d[mid].x < id) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Sum of |block ∩ block| over the block ids two directories share: the lanes
// walk the shorter one and find each id in the longer one by binary search.
__device__ __forceinline__ unsigned long long meet_searched(const uint2 *da, uint32_t na, const uint32_t *Sa,
                                                            const uint2 *db, uint32_t nb, const uint32_t *Sb,
                                                            const uint32_t *__restrict__ words, int lane) {
    const bool a_short = na <= nb;
    const uint2 *ds = a_short ? da : db, *dl = a_short ? db : da;
    const uint32_t ns = a_short ? na : nb, nl = a_short ? nb : na;
    const uint32_t *Ss = a_short ? Sa : Sb, *Sl = a_short ? Sb : Sa;
    unsigned long long c = 0;
    for (uint32_t i = lane; i < ns; i += 32) {
        const uint2 e = ds[i];
        const uint32_t k = dir_lower_bound(dl, nl, e.x);
        if (k < nl) {
            const uint2 f = dl[k];
            if (f.x == e.x) c += block_meet(e.y, Ss, f.y, Sl, words);
        }
    }
    return c;
}

// v = N+(u)[j] for j in [j0, j1) (at most 32), each intersected with u's
// directory: through ud (u's directory staged in shared memory) when staged,
// else by meet_searched on global memory.  With ud, the v's directories form
// one list of entries that the lanes walk in step, each entry's block id found
// among u's staged ids by binary search; a v whose directory is far longer
// than u's is searched instead (the lanes walk u's entries).
__device__ __forceinline__ void blk_pairs(const TrieView &tv, const uint64_t *__restrict__ boff,
                                          const uint2 *__restrict__ dir, const uint32_t *__restrict__ words,
                                          const uint32_t *Su, const uint2 *da, const uint2 *ud, uint32_t na,
                                          uint32_t j0, uint32_t j1, BlkBatch &b, int lane,
                                          unsigned long long &acc) {
    const uint32_t j = j0 + lane;
    uint32_t nb = 0, voff = 0;
    uint64_t bv = 0;
    if (j < j1) {
        const uint32_t v = __ldg(&Su[j]);
        bv = boff[v];
        nb = (uint32_t)(boff[v + 1] - bv);
        voff = tv.desc[v].off;
    }
    if (!ud) {
        for (int k = 0; k < 32; ++k) {
            const uint32_t nbk = __shfl_sync(FULL, nb, k);
            const uint64_t bk = __shfl_sync(FULL, bv, k);
            const uint32_t vk = __shfl_sync(FULL, voff, k);
            if (nbk) acc += meet_searched(da, na, Su, dir + bk, nbk, tv.nbr + vk, words, lane);
        }
        return;
    }
    const bool skew = nb > SKEW * na && nb > SKEW_MIN;
    const uint32_t walk = skew ? 0u : nb;
    uint32_t incl = walk;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    __syncwarp();                   // the previous batch's readers are done
    b.pre[lane] = incl - walk;
    b.voff[lane] = voff;
    b.vb[lane] = bv;
    __syncwarp();
    for (uint32_t e = lane; e < total; e += 32) {
        // the owner: the largest k with pre[k] <= e (a v with nothing to walk
        // shares its prefix with the next lane, which then wins)
        uint32_t lo = 0, hi = 31;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (b.pre[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const uint2 ev = dir[b.vb[lo] + (e - b.pre[lo])];
        const uint32_t k = dir_lower_bound(ud, na, ev.x);
        if (k < na) {
            const uint2 eu = ud[k];
            if (eu.x == ev.x) acc += block_meet(eu.y, Su, ev.y, tv.nbr + b.voff[lo], words);
        }
    }
    unsigned m = __ballot_sync(FULL, skew);
    while (m) {
        const int k = __ffs(m) - 1;
        m &= m - 1;
        const uint32_t nbk = __shfl_sync(FULL, nb, k);
        const uint2 *dv = dir + b.vb[k];
        const uint32_t *Sv = tv.nbr + b.voff[k];
        for (uint32_t i = lane; i < na; i += 32) {
            const uint2 eu = ud[i];
            const uint32_t p = dir_lower_bound(dv, nbk, eu.x);
            if (p < nbk) {
                const uint2 ev = dv[p];
                if (ev.x == eu.x) acc += block_meet(eu.y, Su, ev.y, Sv, words);
            }
        }
    }
}

__device__ __forceinline__ bool is_big(const TrieView &tv, const uint64_t *__restrict__ boff, uint32_t u) {
    return tv.desc[u].len > BIG_LEN || boff[u + 1] - boff[u] > U_CAP;
}

// For every work item u, v runs over N+(u) (v = min N+(u) excluded: nothing
// lies below it in N+(u)) and |N+(u) ∩ N+(v)| is added: the triangles
// (u, v, w) with w < v < u.
// The heavy list comes big items first (|N+(u)| > BIG_LEN, or a directory of
// more than U_CAP entries), heaviest first.  Big items: one CTA each; the CTA
// stages u's directory (up to CTA_CAP entries) and its warps take v's 32 at a
// time.  Every other item, of the heavy list and then of the light list: one
// warp each, u's directory staged in the warp's slice of the same buffer.
__global__ void __launch_bounds__(BLK_WARPS * 32, 6) k_tri_blocks(TrieView tv, const uint64_t *__restrict__ boff,
                                                                  const uint2 *__restrict__ dir,
                                                                  const uint32_t *__restrict__ words,
                                                                  const uint32_t *__restrict__ heavy,
                                                                  uint32_t n_big, uint32_t n_heavy,
                                                                  const uint32_t *__restrict__ light,
                                                                  uint32_t n_light, unsigned int *next,
                                                                  unsigned long long *out) {
    constexpr uint32_t NT = BLK_WARPS * 32;
    __shared__ uint2 s_dir[CTA_CAP];
    __shared__ BlkBatch s_bat[BLK_WARPS];
    __shared__ uint32_t s_item, s_next;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    BlkBatch &b = s_bat[warp];
    unsigned long long acc = 0;

    for (;;) {   // big items: one CTA each
        if (tid == 0) {
            s_item = atomicAdd(&next[0], 1u);
            s_next = 1;
        }
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_big) break;
        const uint32_t u = heavy[item];
        const SetDesc du = tv.desc[u];
        const uint32_t *Su = tv.nbr + du.off;
        const uint64_t bu = boff[u];
        const uint32_t na = (uint32_t)(boff[u + 1] - bu);
        const uint2 *da = dir + bu;
        const bool staged = na <= CTA_CAP;
        if (staged)
            for (uint32_t e = tid; e < na; e += NT) s_dir[e] = da[e];
        __syncthreads();
        for (;;) {
            uint32_t j0 = 0;
            if (lane == 0) j0 = atomicAdd(&s_next, 32u);
            j0 = __shfl_sync(FULL, j0, 0);
            if (j0 >= du.len) break;
            blk_pairs(tv, boff, dir, words, Su, da, staged ? s_dir : nullptr, na, j0, min(j0 + 32, du.len), b,
                      lane, acc);
        }
        __syncthreads();   // the staged directory, s_item and s_next are done with before the next u
    }

    uint2 *ud = s_dir + warp * U_CAP;
    const uint32_t n_rest = n_heavy - n_big;
    for (;;) {   // every other item: one warp each, the rest of the heavy list and then the light list
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(&next[1], 1u);
        it = __shfl_sync(FULL, it, 0);
        if (it >= n_rest + n_light) break;
        const uint32_t u = it < n_rest ? heavy[n_big + it] : light[it - n_rest];
        const SetDesc du = tv.desc[u];
        if (du.len < 2) continue;
        const uint32_t *Su = tv.nbr + du.off;
        const uint64_t bu = boff[u];
        const uint32_t na = (uint32_t)(boff[u + 1] - bu);
        const uint2 *da = dir + bu;
        const bool staged = na <= U_CAP;
        __syncwarp();                       // the previous u's readers are done
        if (staged)
            for (uint32_t e = lane; e < na; e += 32) ud[e] = da[e];
        __syncwarp();
        for (uint32_t j0 = 1; j0 < du.len; j0 += 32)
            blk_pairs(tv, boff, dir, words, Su, da, staged ? ud : nullptr, na, j0, min(j0 + 32, du.len), b, lane,
                      acc);
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(FULL, acc, d);
    if (lane == 0 && acc) atomicAdd(out, acc);
}

// 1 for a big heavy item (a CTA's work in k_tri_blocks), else 0
__global__ void k_big_flags(TrieView tv, const uint64_t *__restrict__ boff, const uint32_t *__restrict__ heavy,
                            uint32_t n, uint32_t *flags) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = is_big(tv, boff, heavy[i]) ? 1u : 0u;
}

// stable partition: big items first, each part in list order
__global__ void k_big_scatter(const uint32_t *__restrict__ heavy, const uint32_t *__restrict__ flags,
                              const uint32_t *__restrict__ pos, uint32_t n, uint32_t n_big, uint32_t *out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[flags[i] ? pos[i] : n_big + (i - pos[i])] = heavy[i];
}

}  // namespace

eh_status eh_build_blocks(eh_trie *t, uint32_t tau, cudaStream_t s) {
    const uint32_t n = t->n;
    if (t->max_out >= (1u << 23)) { eh_set_error("block layout: a set longer than 2^23 - 1"); return EH_EINVAL; }
    uint64_t *nblk = nullptr, *nbit = nullptr;
    EH_TRY(dev_alloc(&nblk, (uint64_t)n + 1, s));
    eh_status st = dev_alloc(&nbit, (uint64_t)n + 1, s);
    uint64_t total = 0, total_bit = 0;
    auto cuda_ok = [&](cudaError_t e, const char *what) {
        if (e == cudaSuccess) return true;
        eh_set_error("block layout: %s: %s", what, cudaGetErrorString(e));
        st = EH_ECUDA;
        return false;
    };
    if (st == EH_OK) cuda_ok(cudaMemsetAsync(nblk, 0, ((uint64_t)n + 1) * 8, s), "memset");
    if (st == EH_OK) cuda_ok(cudaMemsetAsync(nbit, 0, ((uint64_t)n + 1) * 8, s), "memset");
    if (st == EH_OK && n) {
        k_blk_count<<<blocks_for(n), 256, 0, s>>>(t->d_onbr, t->d_desc, n, tau, nblk, nbit);
        cuda_ok(cudaGetLastError(), "count launch");
    }
    if (st == EH_OK) st = trie_alloc(&t->d_boff, (uint64_t)n + 1, s);
    if (st == EH_OK) st = dev_exclusive_scan_u64(nblk, t->d_boff, (uint64_t)n + 1, s, &total);
    if (st == EH_OK) st = dev_exclusive_scan_u64(nbit, nbit, (uint64_t)n + 1, s, &total_bit);
    if (st == EH_OK && total_bit >= BLK_BIT) { eh_set_error("block layout: too many bitset blocks"); st = EH_EINVAL; }
    if (st == EH_OK) st = trie_alloc(&t->d_bdir, total, s);
    if (st == EH_OK) st = trie_alloc(&t->d_bwords, total_bit * 8, s);
    if (st == EH_OK && total_bit) cuda_ok(cudaMemsetAsync(t->d_bwords, 0, total_bit * 32, s), "memset");
    if (st == EH_OK && n) {
        k_blk_fill<<<blocks_for(n), 256, 0, s>>>(t->d_onbr, t->d_desc, n, tau, t->d_boff, nbit, t->d_bdir, t->d_bwords);
        cuda_ok(cudaGetLastError(), "fill launch");
    }
    if (st == EH_OK) cuda_ok(cudaStreamSynchronize(s), "synchronize");
    dev_free(nblk, s);
    dev_free(nbit, s);
    if (st != EH_OK) return st;
    t->n_blocks = total;
    t->n_bit_blocks = total_bit;
    t->device_bytes += total * 8 + total_bit * 32 + ((uint64_t)n + 1) * 8;
    return EH_OK;
}

eh_status eh_plan_blocks(eh_trie *t, WorkPlan *p, cudaStream_t s) {
    const uint32_t n = p->n_heavy;
    uint32_t *flags = nullptr, *pos = nullptr;
    EH_TRY(dev_alloc(&flags, n, s));
    eh_status st = dev_alloc(&pos, n, s);
    uint64_t n_big = 0;
    if (st == EH_OK) {   // held by the plan, freed with its other lists
        cudaError_t e = eh_alloc_should_fail() ? cudaErrorMemoryAllocation
                                               : cudaMalloc((void **)&p->d_heavy_blk, (n ? n : 1) * 4ull);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p->d_heavy_blk = nullptr;
            eh_set_error("block plan: allocation failed");
            st = EH_ENOMEM;
        }
    }
    if (st == EH_OK && n) {
        k_big_flags<<<blocks_for(n), 256, 0, s>>>(t->view(), t->d_boff, p->d_heavy, n, flags);
        st = dev_exclusive_scan_u32(flags, pos, n, s, &n_big);
    }
    if (st == EH_OK && n) {
        k_big_scatter<<<blocks_for(n), 256, 0, s>>>(p->d_heavy, flags, pos, n, (uint32_t)n_big, p->d_heavy_blk);
        if (cudaGetLastError() != cudaSuccess) { eh_set_error("block plan: launch failed"); st = EH_ECUDA; }
    }
    dev_free(flags, s);
    dev_free(pos, s);
    if (st != EH_OK) {
        cudaFree(p->d_heavy_blk);
        p->d_heavy_blk = nullptr;
        return st;
    }
    p->n_big = (uint32_t)n_big;
    return EH_OK;
}

eh_status eh_launch_tri_blocks(eh_trie *t, const WorkPlan &plan, cudaStream_t s, unsigned long long *d_acc,
                               unsigned int *d_next) {
    if (!plan.n_heavy && !plan.n_light) return EH_OK;
    if (plan.n_heavy && !plan.d_heavy_blk) { eh_set_error("block layout: the work plan has no block order"); return EH_EINVAL; }
    int per_sm = 0;
    EH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tri_blocks, BLK_WARPS * 32, 0));
    const uint64_t want = plan.n_big + ((uint64_t)(plan.n_heavy - plan.n_big) + plan.n_light + BLK_WARPS - 1) / BLK_WARPS;
    const uint32_t grid = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>((uint64_t)eh_num_sms() * (uint32_t)std::max(1, per_sm), want));
    EH_CUDA_TRY(cudaMemsetAsync(d_next, 0, 8, s));
    k_tri_blocks<<<grid, BLK_WARPS * 32, 0, s>>>(t->view(), t->d_boff, t->d_bdir, t->d_bwords, plan.d_heavy_blk,
                                                 plan.n_big, plan.n_heavy, plan.d_light, plan.n_light, d_next, d_acc);
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}

extern "C" eh_status eh_trie_export_blocks(const eh_trie *trie, uint64_t *off, uint32_t *dir, uint32_t *words,
                                           uint64_t *n_blocks, uint64_t *n_bit_blocks) {
    if (!trie || !n_blocks || !n_bit_blocks) { eh_set_error("eh_trie_export_blocks: NULL argument"); return EH_EINVAL; }
    if (!trie->d_boff) { eh_set_error("eh_trie_export_blocks: the trie has no block layout"); return EH_EINVAL; }
    *n_blocks = trie->n_blocks;
    *n_bit_blocks = trie->n_bit_blocks;
    if (off) EH_CUDA_TRY(cudaMemcpy(off, trie->d_boff, ((uint64_t)trie->n + 1) * 8, cudaMemcpyDeviceToHost));
    if (dir && trie->n_blocks)
        EH_CUDA_TRY(cudaMemcpy(dir, trie->d_bdir, trie->n_blocks * 8, cudaMemcpyDeviceToHost));
    if (words && trie->n_bit_blocks)
        EH_CUDA_TRY(cudaMemcpy(words, trie->d_bwords, trie->n_bit_blocks * 32, cudaMemcpyDeviceToHost));
    return EH_OK;
}
