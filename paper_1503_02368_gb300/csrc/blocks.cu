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
// directories: the lanes of a warp walk the shorter directory, find each
// block id in the longer one by binary search (the offsets-as-uint
// intersection of Sec. 4.2), and intersect matching blocks by the layout pair:
// AND + popcount of 8 words, bit probes of a run's values, or a merge of two
// runs.
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

// one warp per vertex u (any order); v runs over N+(u); counts |N+(u) ∩ N+(v)|
__global__ void k_tri_blocks(TrieView tv, const uint64_t *__restrict__ boff, const uint2 *__restrict__ dir,
                             const uint32_t *__restrict__ words, const uint32_t *__restrict__ items,
                             uint32_t n_items, unsigned int *next, unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    unsigned long long acc = 0;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(next, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const uint32_t u = items[it];
        const SetDesc du = tv.desc[u];
        const uint32_t *Sa = tv.nbr + du.off;
        const uint2 *da = dir + boff[u];
        const uint32_t na = (uint32_t)(boff[u + 1] - boff[u]);
        for (uint32_t j = 1; j < du.len; ++j) {
            const uint32_t v = __ldg(&Sa[j]);
            const SetDesc dv = tv.desc[v];
            if (dv.len == 0) continue;
            const uint32_t *Sb = tv.nbr + dv.off;
            const uint2 *db = dir + boff[v];
            const uint32_t nbk = (uint32_t)(boff[v + 1] - boff[v]);
            // walk the shorter directory, search the longer one
            const bool a_short = na <= nbk;
            const uint2 *ds = a_short ? da : db, *dl = a_short ? db : da;
            const uint32_t ns = a_short ? na : nbk, nl = a_short ? nbk : na;
            const uint32_t *Ss = a_short ? Sa : Sb, *Sl = a_short ? Sb : Sa;
            for (uint32_t i = lane; i < ns; i += 32) {
                const uint2 e = ds[i];
                uint32_t lo = 0, hi = nl;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (dl[mid].x < e.x) lo = mid + 1; else hi = mid;
                }
                if (lo < nl && dl[lo].x == e.x) acc += block_meet(e.y, Ss, dl[lo].y, Sl, words);
            }
        }
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if (lane == 0 && acc) atomicAdd(out, acc);
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

eh_status eh_launch_tri_blocks(eh_trie *t, const WorkPlan &plan, cudaStream_t s, unsigned long long *d_acc,
                               unsigned int *d_next) {
    const uint32_t n_items = plan.n_heavy + plan.n_light;
    if (!n_items) return EH_OK;
    // heavy items, then light ones (the plan's two lists), a counter each
    const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)eh_num_sms() * 8, (n_items + 7) / 8);
    EH_CUDA_TRY(cudaMemsetAsync(d_next, 0, 8, s));
    if (plan.n_heavy)
        k_tri_blocks<<<std::max(1u, std::min(grid, (plan.n_heavy + 7) / 8)), 256, 0, s>>>(
            t->view(), t->d_boff, t->d_bdir, t->d_bwords, plan.d_heavy, plan.n_heavy, d_next, d_acc);
    if (plan.n_light)
        k_tri_blocks<<<std::max(1u, std::min(grid, (plan.n_light + 7) / 8)), 256, 0, s>>>(
            t->view(), t->d_boff, t->d_bdir, t->d_bwords, plan.d_light, plan.n_light, d_next + 1, d_acc);
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
