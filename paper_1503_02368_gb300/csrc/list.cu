// list.cu -- triangle and 4-clique listing into a caller's device buffer (eh_list).
//
// The joins of the count path with their head variables kept (Table 1's
// Triangle(x,y,z) and 4Clique(x,y,z,w) without the COUNT aggregation): every
// match of the innermost level of the generic join (Algorithm 1) becomes one
// output row, the caller's ids of the clique in ascending order.
//
// Work items are those of the count plan: a vertex u with |N+(u)| above the
// light bound is taken by a CTA, which stages A = N+(u) in shared memory (a
// bitmap when its value range fits, else the sorted array) and whose warps take the
// v in A dynamically; a lighter u is taken by one warp holding A one element
// per lane.  Two passes.  The first stores each item's number of rows (for
// triangles, the count kernel's per-item mode gives them; for 4-cliques, this
// file's traversal in counting mode), an exclusive scan turns those into
// output ranges, and the second pass runs the traversal again and writes the
// rows.  Inside an item the lanes of a warp take positions from ballot /
// prefix-sum ranks, stage the round's rows in shared memory and store them
// as one contiguous run; the warps of a CTA reserve runs from a shared-memory
// cursor (a device-memory one when an item's rows could pass 2^32).  A heavy
// item's triangle rows are first collected per pair (the third vertices, in a
// per-warp buffer) and then built and stored 128 at a time, every lane
// building one row, so a reservation and a store run serve up to 128 rows
// instead of one round's matches.  The
// output is dense and the rows of an item fill exactly the range the first
// pass gave it.  The same 4-clique passes, fed with A = N(x) for the
// neighbours x of a selected vertex, count the selection query SK4.
//
// Per pair the intersection works on what the lanes can enumerate (Sec. 4.2's
// operations): with A as an on-chip bitmap every element of N+(v) probes one
// bit of it; with A as a sorted array its elements probe N+(v)'s stored bitset
// or binary-search its uint array, or N+(v)'s elements binary-search A,
// whichever side is smaller.  Every loop over a set runs in warp-uniform rounds
// of 32 lanes so that the matches of a round can be ranked by one ballot or
// one warp prefix sum.  Staging uses plain loads (no bulk copy) and bitset
// pairs go through the uint array of N+(v): the rows, not the reads, bound
// this path.
#include "eh_internal.cuh"
#include "dev_util.cuh"

#include <algorithm>

namespace {

using namespace ehd;

constexpr uint32_t LIST_WARPS = 8;
constexpr uint32_t LA_CAP_WORDS = 8192;   // on-chip A: bitmap words or sorted elements (32 KB)
constexpr uint32_t S_CAP = 512;           // per-warp level-1 set of the 4-clique in shared memory
constexpr uint32_t TC_CAP = 256;          // per-warp matches of a triangle pair collected before their rows are written

enum { P_TRI = 3, P_K4 = 4 };   // row width

struct ListArgs {
    TrieView tv;
    const uint32_t *new2old;
    const uint32_t *heavy;
    uint32_t n_heavy;
    const uint32_t *light;
    uint32_t n_light;
    uint32_t ratio;
    uint32_t arena_stride;                 // words per warp slot of the arena (4-clique, large S)
    uint32_t flags;                        // EH_EXEC_SORTED_A / EH_EXEC_GLOBAL_A
    const uint64_t *a_off;                 // non-null: A(u) is the symmetric set N(u) (selection queries):
    const uint32_t *a_nbr;                 //   a_nbr[a_off[u] ..] of a_len[u] ids; null: A(u) = N+(u)
    const uint32_t *a_len;
    unsigned int *next_item;               // heavy items taken so far
    unsigned long long *cursor;            // write pass: next row of each heavy CTA's current item
    uint32_t rel32;                        // 1: an item's rows fit 32 bits (shared-memory cursor instead)
    unsigned long long *cnt;               // count pass: rows per item (heavy items, then light)
    const unsigned long long *offs;        // write pass: first row of each item (n_items + 1 entries)
    uint32_t *out;                         // rows of width 3 or 4
    unsigned long long cap;                // rows the buffer holds
    uint32_t *arena;
    uint32_t *status;
};

// Output state of one warp for the current item.
struct Sink {
    unsigned long long n;        // count pass: rows found by this warp
    unsigned long long cur;      // write pass, light item: next row of the warp
    unsigned long long *s_cur;   // write pass, heavy item: the CTA's cursor (device memory); null if light
    uint32_t *s_rel;             // write pass, heavy item: rows taken so far (shared memory), when 32 bits suffice
    unsigned long long rel_base; //   ... counted from this first row of the item
    unsigned long long end;      // write pass: end of the item's range
    uint32_t key[3];             // caller ids of the bound prefix: u, v (and z)
    uint32_t *stage;             // write pass: this warp's rows of the current round (shared memory)
};

constexpr uint32_t STAGE_ROWS = 128;   // rows one round can produce (four candidates per lane)

__device__ __forceinline__ void sort2(uint32_t &a, uint32_t &b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// row r of the round in the warp's staging buffer: the clique's caller ids, ascending
template <int W>
__device__ __forceinline__ void stage_row(const ListArgs &a, const Sink &sk, uint32_t r, uint32_t w_new) {
    uint32_t x0 = sk.key[0], x1 = sk.key[1], x2 = __ldg(&a.new2old[w_new]);
    uint32_t *o = sk.stage + r * W;
    if (W == P_TRI) {
        sort2(x0, x1); sort2(x1, x2); sort2(x0, x1);
        o[0] = x0; o[1] = x1; o[2] = x2;
    } else {
        uint32_t x3 = sk.key[2];
        sort2(x0, x1); sort2(x2, x3); sort2(x0, x2); sort2(x1, x3); sort2(x1, x2);
        *reinterpret_cast<uint4 *>(o) = make_uint4(x0, x1, x2, x3);
    }
}

// the round's `total` staged rows to rows base .. base+total-1 of the output,
// consecutive lanes on consecutive words (never outside the item's range)
template <int W>
__device__ __forceinline__ void flush(const ListArgs &a, const Sink &sk, unsigned long long base, uint32_t total) {
    const uint32_t lane = threadIdx.x & 31;
    __syncwarp();
    if (base + total > sk.end || base + total > a.cap) {   // the two passes disagree
        if (lane == 0) atomicOr(a.status, DEV_ST_RANGE);
    } else if (W == P_K4) {
        uint4 *o = reinterpret_cast<uint4 *>(a.out + base * 4);
        const uint4 *st = reinterpret_cast<const uint4 *>(sk.stage);
        for (uint32_t i = lane; i < total; i += 32) o[i] = st[i];
    } else {
        uint32_t *o = a.out + base * 3;
        for (uint32_t i = lane; i < total * 3; i += 32) o[i] = sk.stage[i];
    }
    __syncwarp();
}

// first output row of a round whose matches total `total` (warp-uniform);
// a heavy item's warps share its CTA's cursor, a light item's warp keeps its own
template <bool EMIT>
__device__ __forceinline__ unsigned long long reserve(Sink &sk, uint32_t total) {
    if (!EMIT) {
        sk.n += total;
        return 0;
    }
    unsigned long long base = 0;
    if (total) {
        if (sk.s_rel) {
            uint32_t r = 0;
            if ((threadIdx.x & 31) == 0) r = atomicAdd(sk.s_rel, total);
            base = sk.rel_base + __shfl_sync(FULL, r, 0);
        } else if (sk.s_cur) {
            if ((threadIdx.x & 31) == 0) base = atomicAdd(sk.s_cur, (unsigned long long)total);
            base = __shfl_sync(FULL, base, 0);
        } else {
            base = sk.cur;
            sk.cur += total;
        }
    }
    return base;
}

// One round where each lane has at most one candidate w (hit = w matches).
template <int W, bool EMIT>
__device__ __forceinline__ void emit_one(const ListArgs &a, Sink &sk, bool hit, uint32_t w) {
    const uint32_t b = __ballot_sync(FULL, hit);
    const uint32_t total = __popc(b);
    if (!EMIT) {
        sk.n += total;
        return;
    }
    if (!total) return;
    const unsigned long long base = reserve<EMIT>(sk, total);
    if (hit) stage_row<W>(a, sk, __popc(b & ((1u << (threadIdx.x & 31)) - 1u)), w);
    flush<W>(a, sk, base, total);
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(FULL, x, d);
    return x;
}

// exclusive warp prefix sum of x; total in *total
__device__ __forceinline__ uint32_t warp_excl(uint32_t x, uint32_t &total) {
    const int lane = threadIdx.x & 31;
    uint32_t incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += y;
    }
    total = __shfl_sync(FULL, incl, 31);
    return incl - x;
}

// One round where each lane has four candidate values v[c], matching where bit c of m is set.
template <int W, bool EMIT>
__device__ __forceinline__ void emit_four(const ListArgs &a, Sink &sk, uint32_t m, const uint4 &v) {
    const uint32_t k = __popc(m);
    if (!EMIT) {
        sk.n += warp_sum(k);
        return;
    }
    uint32_t total;
    const uint32_t r = warp_excl(k, total);
    if (!total) return;
    const unsigned long long base = reserve<EMIT>(sk, total);
    const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
    uint32_t i = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if ((m >> c) & 1u) stage_row<W>(a, sk, r + i++, vv[c]);
    flush<W>(a, sk, base, total);
}

// x in the set with descriptor d (bit probe of its bitset, else binary search of its uint array)
__device__ __forceinline__ bool in_set(const TrieView &tv, const SetDesc &d, uint32_t x) {
    if (d.nwords) {
        const uint32_t r = x - d.lo_word * 32;
        return r < d.nwords * 32 && ((__ldg(&tv.words[d.woff + (r >> 5)]) >> (r & 31)) & 1u);
    }
    const uint32_t *B = tv.nbr + d.off;
    const uint32_t p = lower_bound(B, 0, d.len, x);
    return p < d.len && __ldg(&B[p]) == x;
}

// ------------------------------------------------------------ staged A

struct StagedA {
    uint32_t mode;        // 0 bitmap in shared memory, 1 sorted array in shared memory, 2 sorted array in global
    uint32_t len;
    uint32_t a_lo, a_nw;  // bitmap: first word (value / 32) and number of words
    const uint32_t *Ag;   // the stored uint array of A
    const uint32_t *A;    // sorted elements (modes 1, 2)
};

// Stages A = N+(u) for the CTA with plain loads: an on-chip bitmap of its
// value range when that fits, else the sorted array when it fits, else A is
// read from device memory.
__device__ __forceinline__ void stage_a(const uint32_t *Ag, uint32_t len, uint32_t flags, uint32_t *sA,
                                        StagedA &st) {
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    st.len = len;
    st.Ag = Ag;
    const uint32_t first = __ldg(&st.Ag[0]), last = __ldg(&st.Ag[st.len - 1]);
    st.a_lo = (first >> 7) << 2;
    st.a_nw = (((last >> 5) + 1 - st.a_lo) + 3) & ~3u;
    if (!(flags & (EH_EXEC_SORTED_A | EH_EXEC_GLOBAL_A)) && st.a_nw <= LA_CAP_WORDS) {
        st.mode = 0;
        for (uint32_t i = tid * 4; i < st.a_nw; i += nthr * 4)
            *reinterpret_cast<uint4 *>(sA + i) = make_uint4(0, 0, 0, 0);
        __syncthreads();
        for (uint32_t i = tid; i < st.len; i += nthr) {
            const uint32_t x = __ldg(&st.Ag[i]);
            atomicOr(&sA[(x >> 5) - st.a_lo], 1u << (x & 31));
        }
    } else if (!(flags & EH_EXEC_GLOBAL_A) && st.len <= LA_CAP_WORDS) {
        st.mode = 1;
        for (uint32_t i = tid; i < st.len; i += nthr) sA[i] = __ldg(&st.Ag[i]);
    } else {
        st.mode = 2;
    }
    __syncthreads();
    st.A = st.mode == 2 ? st.Ag : sA;
}

// ------------------------------------------------- level-1 intersections
//
// A ∩ N+(v) for A staged by the CTA, v = A[j].  Each match w goes to
// `out_fn(hit-round ...)`: the emit_* rounds above when listing triangles,
// the collection of S when listing 4-cliques.  Matches come out in ascending
// order of w in every branch (rounds walk the sets upwards, lanes in order).

// BATCH (triangle rows, write pass): the matches are collected like COLLECT
// and turned into rows by drain(), 128 rows per cursor reservation, every lane
// building one row, whenever more than TC_CAP - 128 are waiting (a round adds
// at most 128) and at the end of the pair.
template <int W, bool EMIT, bool COLLECT, bool BATCH = false>
struct Level1 {
    const ListArgs &a;
    Sink &sk;
    uint32_t *S;      // COLLECT: destination of the matches
    uint32_t ns;      // COLLECT: matches so far

    __device__ __forceinline__ void one(bool hit, uint32_t w) {
        if (COLLECT) {
            const uint32_t b = __ballot_sync(FULL, hit);
            if (hit) S[ns + __popc(b & ((1u << (threadIdx.x & 31)) - 1u))] = w;
            ns += __popc(b);
            if (BATCH && ns > TC_CAP - STAGE_ROWS) drain();
        } else {
            emit_one<W, EMIT>(a, sk, hit, w);
        }
    }
    __device__ __forceinline__ void four(uint32_t m, const uint4 &v) {
        if (COLLECT) {
            uint32_t total;
            const uint32_t r = warp_excl(__popc(m), total);
            const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
            uint32_t i = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if ((m >> c) & 1u) S[ns + r + i++] = vv[c];
            ns += total;
            if (BATCH && ns > TC_CAP - STAGE_ROWS) drain();
        } else {
            emit_four<W, EMIT>(a, sk, m, v);
        }
    }
    // BATCH: rows (key[0], key[1], S[i]) for the collected matches, then empty S
    __device__ __forceinline__ void drain() {
        const uint32_t lane = threadIdx.x & 31;
        __syncwarp();
        for (uint32_t c0 = 0; c0 < ns; c0 += STAGE_ROWS) {
            const uint32_t cn = min(STAGE_ROWS, ns - c0);
            const unsigned long long base = reserve<EMIT>(sk, cn);
            for (uint32_t i = lane; i < cn; i += 32) stage_row<W>(a, sk, i, S[c0 + i]);
            flush<W>(a, sk, base, cn);
        }
        ns = 0;
    }
    // A as the on-chip bitmap of words [a_lo, a_lo + a_nw): every element of
    // N+(v) probes it (B's uint array; the padding EH_PAD is out of range)
    __device__ __forceinline__ void bitmap(const uint32_t *sA, uint32_t a_lo, uint32_t a_nw, const SetDesc &dv) {
        const TrieView &tv = a.tv;
        const uint32_t lane = threadIdx.x & 31;
        const uint32_t *bp = tv.nbr + dv.off;
        const uint32_t base = a_lo * 32, nbits = a_nw * 32;
        for (uint32_t p0 = 0; p0 < dv.len; p0 += 128) {
            const uint32_t p = p0 + lane * 4;
            const uint4 e = p < dv.len ? ldg4(bp + p) : make_uint4(EH_PAD, EH_PAD, EH_PAD, EH_PAD);
            const uint32_t ev[4] = {e.x, e.y, e.z, e.w};
            uint32_t m = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t x = ev[c] - base;
                if (x < nbits && ((sA[x >> 5] >> (x & 31)) & 1u)) m |= 1u << c;
            }
            four(m, e);
        }
    }

    // A as a sorted array, of which only the prefix A[0..j) can meet N+(v)
    __device__ __forceinline__ void sorted(const uint32_t *A, uint32_t j, const SetDesc &dv) {
        const TrieView &tv = a.tv;
        const uint32_t lane = threadIdx.x & 31;
        // the smaller side enumerates (the min property of Sec. 4.2): A's prefix probes
        // N+(v) when it is no longer than N+(v) (bit probes) or far shorter (binary search)
        if ((uint64_t)dv.len > (uint64_t)a.ratio * j || (dv.nwords && j <= dv.len)) {
            // A's elements probe N+(v): its bitset, or a binary search of its uint array
            for (uint32_t i0 = 0; i0 < j; i0 += 32) {
                const uint32_t i = i0 + lane;
                const uint32_t x = i < j ? A[i] : EH_PAD;
                one(i < j && in_set(tv, dv, x), x);
            }
            return;
        }
        // N+(v)'s elements search A[0..j)
        const uint32_t *B = tv.nbr + dv.off;
        for (uint32_t p0 = 0; p0 < dv.len; p0 += 32) {
            const uint32_t p = p0 + lane;
            const uint32_t x = p < dv.len ? __ldg(&B[p]) : EH_PAD;
            bool hit = false;
            if (p < dv.len) {
                const uint32_t q = lower_bound(A, 0, j, x);
                hit = q < j && A[q] == x;
            }
            one(hit, x);
        }
    }
};

// Level 2 of the 4-clique for z = S[r]: S[0..r) ∩ N+(z), rows (u, v, z, w).
template <bool EMIT>
__device__ __forceinline__ void k4_level2(const ListArgs &a, Sink &sk, const uint32_t *S, uint32_t r,
                                          const SetDesc &dz) {
    const uint32_t lane = threadIdx.x & 31;
    if (dz.len == 0 || r == 0) return;
    if ((uint64_t)dz.len > (uint64_t)a.ratio * r || (dz.nwords && r <= dz.len)) {   // the smaller side enumerates
        for (uint32_t i0 = 0; i0 < r; i0 += 32) {
            const uint32_t i = i0 + lane;
            const uint32_t x = i < r ? S[i] : EH_PAD;
            emit_one<P_K4, EMIT>(a, sk, i < r && in_set(a.tv, dz, x), x);
        }
        return;
    }
    const uint32_t *B = a.tv.nbr + dz.off;
    for (uint32_t p0 = 0; p0 < dz.len; p0 += 32) {
        const uint32_t p = p0 + lane;
        const uint32_t x = p < dz.len ? __ldg(&B[p]) : EH_PAD;
        bool hit = false;
        if (p < dz.len) {
            const uint32_t q = lower_bound(S, 0, r, x);
            hit = q < r && S[q] == x;
        }
        emit_one<P_K4, EMIT>(a, sk, hit, x);
    }
}

// ------------------------------------------------------------- kernels

// Heavy items: a persistent grid, one item per CTA at a time.
template <int W, bool EMIT>
__global__ void __launch_bounds__(LIST_WARPS * 32, W == P_TRI ? (EMIT ? 4 : 8) : (EMIT ? 6 : 8)) k_list_heavy(ListArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sA = smem;
    __shared__ uint32_t s_item, s_next, s_rel;
    __shared__ unsigned long long s_wcnt[LIST_WARPS];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr bool TBATCH = W == P_TRI && EMIT;   // triangle rows through Level1's BATCH mode
    uint32_t *S = nullptr;
    if (W == P_K4) S = smem + LA_CAP_WORDS + warp * S_CAP;
    if (TBATCH) S = smem + LA_CAP_WORDS + warp * TC_CAP;
    uint32_t *S_big = a.arena ? a.arena + (uint64_t)(blockIdx.x * LIST_WARPS + warp) * a.arena_stride : nullptr;
    uint32_t *stage = EMIT ? smem + LA_CAP_WORDS + (W == P_K4 ? LIST_WARPS * S_CAP : LIST_WARPS * TC_CAP) +
                                 warp * STAGE_ROWS * W
                           : nullptr;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(a.next_item, 1u);
            s_next = 1;
            s_rel = 0;
            if (EMIT && !a.rel32 && s_item < a.n_heavy) atomicExch(a.cursor + blockIdx.x, a.offs[s_item]);
        }
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= a.n_heavy) break;
        const uint32_t u = a.heavy[item];
        StagedA st;
        if (a.a_off) stage_a(a.a_nbr + a.a_off[u], a.a_len[u], a.flags, sA, st);
        else {
            const SetDesc du = a.tv.desc[u];
            stage_a(a.tv.nbr + du.off, du.len, a.flags, sA, st);
        }
        Sink sk;
        sk.n = 0;
        sk.cur = 0;
        sk.s_cur = EMIT && !a.rel32 ? a.cursor + blockIdx.x : nullptr;
        sk.s_rel = EMIT && a.rel32 ? &s_rel : nullptr;
        sk.rel_base = EMIT ? a.offs[item] : 0;
        sk.stage = stage;
        sk.end = EMIT ? a.offs[item + 1] : 0;
        sk.key[0] = __ldg(&a.new2old[u]);
        for (;;) {
            uint32_t j = 0;
            if (lane == 0) j = atomicAdd(&s_next, 1u);
            j = __shfl_sync(FULL, j, 0);
            if (j >= st.len) break;
            const uint32_t v = st.mode == 0 ? __ldg(&st.Ag[j]) : st.A[j];
            const SetDesc dv = a.tv.desc[v];
            if (dv.len == 0) continue;
            sk.key[1] = __ldg(&a.new2old[v]);
            if (TBATCH) {
                Level1<P_TRI, EMIT, true, true> l1{a, sk, S, 0};
                if (st.mode == 0) l1.bitmap(sA, st.a_lo, st.a_nw, dv);
                else l1.sorted(st.A, j, dv);
                if (l1.ns) l1.drain();
                __syncwarp();
            } else if (W == P_TRI) {
                Level1<P_TRI, EMIT, false> l1{a, sk, nullptr, 0};
                if (st.mode == 0) l1.bitmap(sA, st.a_lo, st.a_nw, dv);
                else l1.sorted(st.A, j, dv);
            } else {
                // level 1: S = A ∩ N+(v), sorted, in the warp's buffer
                uint32_t *Sw = min(j, dv.len) <= S_CAP ? S : S_big;
                if (!Sw) { atomicOr(a.status, DEV_ST_RANGE); continue; }
                Level1<P_K4, EMIT, true> l1{a, sk, Sw, 0};
                if (st.mode == 0) l1.bitmap(sA, st.a_lo, st.a_nw, dv);
                else l1.sorted(st.A, j, dv);
                __syncwarp();
                // level 2: for z in S, S_<z ∩ N+(z)
                for (uint32_t r = 1; r < l1.ns; ++r) {
                    const uint32_t z = Sw[r];
                    sk.key[2] = __ldg(&a.new2old[z]);
                    k4_level2<EMIT>(a, sk, Sw, r, a.tv.desc[z]);
                }
                __syncwarp();
            }
        }
        if (!EMIT && lane == 0) s_wcnt[warp] = sk.n;   // warp-uniform
        __syncthreads();
        if (!EMIT && threadIdx.x == 0) {
            unsigned long long c = 0;
            for (uint32_t w = 0; w < LIST_WARPS; ++w) c += s_wcnt[w];
            a.cnt[item] = c;
        }
    }
}

// Light items: one warp each, A = N+(u) one element per lane (|A| <= 32).
template <int W, bool EMIT>
__global__ void __launch_bounds__(LIST_WARPS * 32) k_list_light(ListArgs a) {
    __shared__ __align__(16) uint32_t s_stage[EMIT ? LIST_WARPS * 32 * W : 4];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t item = blockIdx.x * LIST_WARPS + (threadIdx.x >> 5);
    if (item >= a.n_light) return;
    const uint32_t u = a.light[item];
    const uint32_t *Ag = a.a_off ? a.a_nbr + a.a_off[u] : a.tv.nbr + a.tv.desc[u].off;
    const uint32_t L = min(a.a_off ? a.a_len[u] : a.tv.desc[u].len, 32u);
    const uint32_t x = lane < L ? __ldg(&Ag[lane]) : EH_PAD;
    SetDesc mine = empty_desc();
    if (lane < L) mine = a.tv.desc[x];
    Sink sk;
    sk.n = 0;
    sk.s_cur = nullptr;
    sk.s_rel = nullptr;
    sk.rel_base = 0;
    sk.stage = s_stage + (threadIdx.x >> 5) * 32 * W;
    sk.cur = EMIT ? a.offs[a.n_heavy + item] : 0;
    sk.end = EMIT ? a.offs[a.n_heavy + item + 1] : 0;
    sk.key[0] = __ldg(&a.new2old[u]);
    for (uint32_t j = 1; j < L; ++j) {
        const SetDesc dv = bcast_desc(mine, j);
        if (dv.len == 0) continue;
        const uint32_t v = __shfl_sync(FULL, x, j);
        sk.key[1] = __ldg(&a.new2old[v]);
        const bool h1 = lane < j && in_set(a.tv, dv, x);
        if (W == P_TRI) {
            emit_one<P_TRI, EMIT>(a, sk, h1, x);
        } else {
            const uint32_t bS = __ballot_sync(FULL, h1);   // S = A ∩ N+(v), one lane per element
            for (uint32_t rest = bS; rest;) {
                const uint32_t r = __ffs(rest) - 1;
                rest &= rest - 1;
                const SetDesc dz = bcast_desc(mine, r);
                sk.key[2] = __ldg(&a.new2old[__shfl_sync(FULL, x, r)]);
                const bool h2 = ((bS >> lane) & 1u) && lane < r && dz.len && in_set(a.tv, dz, x);
                emit_one<P_K4, EMIT>(a, sk, h2, x);
            }
        }
    }
    if (!EMIT) {
        if (lane == 0) a.cnt[a.n_heavy + item] = sk.n;
    }
}

template <int W, bool EMIT>
eh_status launch_pass(const ListArgs &a, uint32_t heavy_grid, cudaStream_t s) {
    const uint32_t smem = LA_CAP_WORDS * 4 + (W == P_K4 ? LIST_WARPS * S_CAP * 4 : 0) +
                          (EMIT ? LIST_WARPS * (STAGE_ROWS * W + (W == P_TRI ? TC_CAP : 0)) * 4 : 0);
    EH_CUDA_TRY(cudaFuncSetAttribute(k_list_heavy<W, EMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    if (a.n_heavy) k_list_heavy<W, EMIT><<<heavy_grid, LIST_WARPS * 32, smem, s>>>(a);
    EH_CUDA_TRY(cudaGetLastError());
    if (a.n_light) k_list_light<W, EMIT><<<ceil_div_u32(a.n_light, LIST_WARPS), LIST_WARPS * 32, 0, s>>>(a);
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}

template <int W>
eh_status heavy_grid_size(uint32_t n_heavy, uint32_t *grid) {
    const uint32_t smem = LA_CAP_WORDS * 4 + (W == P_K4 ? LIST_WARPS * S_CAP * 4 : 0);
    EH_CUDA_TRY(cudaFuncSetAttribute(k_list_heavy<W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    EH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_list_heavy<W, false>, LIST_WARPS * 32, smem));
    const uint64_t g = (uint64_t)std::max(per_sm, 1) * eh_num_sms();
    *grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(g, n_heavy));
    return EH_OK;
}

struct ListBuffers {
    unsigned long long *cnt = nullptr, *offs = nullptr;
    unsigned int *next = nullptr;
    unsigned long long *cursor = nullptr, *scr = nullptr;
    uint32_t *arena = nullptr;
    cudaStream_t s = nullptr;
    ~ListBuffers() {
        dev_free(cnt, s);
        dev_free(offs, s);
        dev_free(next, s);
        dev_free(cursor, s);
        dev_free(scr, s);
        dev_free(arena, s);
        cudaStreamSynchronize(s);
    }
};

// The work items of one run and where their A sets come from.
struct Items {
    const uint32_t *heavy = nullptr, *light = nullptr;   // device lists
    uint32_t n_heavy = 0, n_light = 0;
    const uint64_t *a_off = nullptr;                      // symmetric sets (selection queries); null: N+(u)
    const uint32_t *a_nbr = nullptr, *a_len = nullptr;
};

__global__ void k_gather_u32(const uint32_t *__restrict__ idx, uint32_t n, const uint32_t *__restrict__ val,
                             uint32_t *out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = val[idx[i]];
}

// Count pass (and, when d_out is set, the write pass) over the items.
// plan: the whole-graph work plan the items come from, or null.  With a plan,
// the triangle rows per item come from the count kernel's per-item mode (the
// same items, the same numbers: the triangles whose largest id is the item).
template <int W>
eh_status run_items(eh_trie *t, const Items &it, const WorkPlan *plan, const eh_exec_opts &xo, cudaStream_t s,
                    uint32_t *d_out, uint64_t capacity, uint64_t *out_n) {
    const uint64_t n_items = (uint64_t)it.n_heavy + it.n_light;
    ListBuffers b;
    b.s = s;
    EH_TRY(dev_alloc(&b.cnt, n_items + 1, s));
    EH_TRY(dev_alloc(&b.offs, n_items + 1, s));
    EH_TRY(dev_alloc(&b.next, 2, s));
    EH_CUDA_TRY(cudaMemsetAsync(b.cnt, 0, (n_items + 1) * 8, s));
    EH_CUDA_TRY(cudaMemsetAsync(b.next, 0, 8, s));
    uint32_t grid = 1;
    EH_TRY(heavy_grid_size<W>(it.n_heavy, &grid));
    EH_TRY(dev_alloc(&b.cursor, grid, s));
    ListArgs a;
    a.tv = t->view();
    a.new2old = t->d_new2old;
    a.heavy = it.heavy;
    a.n_heavy = it.n_heavy;
    a.light = it.light;
    a.n_light = it.n_light;
    a.a_off = it.a_off;
    a.a_nbr = it.a_nbr;
    a.a_len = it.a_len;
    a.ratio = xo.gallop_ratio;
    a.flags = xo.flags;
    a.arena_stride = 0;
    a.arena = nullptr;
    // |S| <= |N+(v)| <= max out-degree, whatever A is
    if (W == P_K4 && t->max_out > S_CAP && it.n_heavy) {
        a.arena_stride = (t->max_out + 3) & ~3u;
        EH_TRY(dev_alloc(&b.arena, (uint64_t)grid * LIST_WARPS * a.arena_stride, s));
        a.arena = b.arena;
    }
    a.status = t->d_status;
    a.cursor = b.cursor;
    {   // rows of one item: at most C(|A|, 2) triangles or C(|A|, 3) 4-cliques
        const double L = it.a_off ? (double)t->max_deg : (double)t->max_out;
        const double bound = W == P_TRI ? L * (L - 1) / 2 : L * (L - 1) * (L - 2) / 6;
        a.rel32 = bound < 4294967295.0 ? 1u : 0u;
    }
    a.out = d_out;
    a.cap = capacity;
    // pass 1: rows per item
    a.next_item = b.next;
    a.cnt = b.cnt;
    a.offs = nullptr;
    if (W == P_TRI && plan && !it.a_off) {
        EH_TRY(dev_alloc(&b.scr, 4, s));
        EH_CUDA_TRY(cudaMemsetAsync(b.scr, 0, 32, s));
        EH_TRY(eh_launch_triangle(t, *plan, t->view(), TRI_MODE_APEX, xo, s, b.scr, b.scr + 1, t->d_status, b.cnt,
                                  nullptr));
    } else {
        EH_TRY((launch_pass<W, false>(a, grid, s)));
    }
    uint64_t total = 0;
    EH_TRY(dev_exclusive_scan_u64(reinterpret_cast<const uint64_t *>(b.cnt), reinterpret_cast<uint64_t *>(b.offs),
                                  n_items + 1, s, &total));
    EH_TRY(eh_check_status(t, s));
    *out_n = total;
    if (!d_out) return EH_OK;
    if (total > capacity) {
        eh_set_error("eh_list: the result has %llu rows, the buffer holds %llu", (unsigned long long)total,
                     (unsigned long long)capacity);
        return EH_ECAPACITY;
    }
    // pass 2: rows written into each item's range
    a.next_item = b.next + 1;
    a.offs = b.offs;
    EH_TRY((launch_pass<W, true>(a, grid, s)));
    return eh_check_status(t, s);
}

template <int W>
eh_status run_list(eh_trie *t, const eh_exec_opts &xo, cudaStream_t s, uint32_t *d_out, uint64_t capacity,
                   uint64_t *out_n) {
    NvtxRange nv("eh_list");
    WorkPlan *plan = nullptr;
    EH_TRY(eh_plan_get(t, xo.light_max, s, &plan));
    Items it;
    it.heavy = plan->d_heavy;
    it.n_heavy = plan->n_heavy;
    it.light = plan->d_light;
    it.n_light = plan->n_light;
    return run_items<W>(t, it, plan, xo, s, d_out, capacity, out_n);
}

// 4-cliques through each x in N(node): the triangles of G[N(x)], counted by
// the 4-clique passes with A = N(x) (symmetric) and y over all of A.  Items
// are the x with d(x) >= 3 (fewer neighbours hold no triangle), split by d(x).
eh_status sk4_total(eh_trie *t, uint32_t node_new, const eh_exec_opts &xo, cudaStream_t s, uint64_t *total) {
    *total = 0;
    uint64_t base = 0;
    uint32_t dn = 0;
    EH_CUDA_TRY(cudaMemcpyAsync(&base, t->d_soff + node_new, 8, cudaMemcpyDeviceToHost, s));
    EH_CUDA_TRY(cudaMemcpyAsync(&dn, t->d_deg + node_new, 4, cudaMemcpyDeviceToHost, s));
    EH_CUDA_TRY(cudaStreamSynchronize(s));
    if (!dn) return EH_OK;
    std::vector<uint32_t> xs(dn), dx(dn), heavy, light;
    {
        uint32_t *d_dx = nullptr;
        EH_TRY(dev_alloc(&d_dx, dn, s));
        k_gather_u32<<<(dn + 255) / 256, 256, 0, s>>>(t->d_snbr + base, dn, t->d_deg, d_dx);
        cudaError_t e1 = cudaMemcpyAsync(xs.data(), t->d_snbr + base, (uint64_t)dn * 4, cudaMemcpyDeviceToHost, s);
        cudaError_t e2 = cudaMemcpyAsync(dx.data(), d_dx, (uint64_t)dn * 4, cudaMemcpyDeviceToHost, s);
        cudaError_t e3 = cudaStreamSynchronize(s);
        dev_free(d_dx, s);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            eh_set_error("sk4: reading the selected vertex's neighbours failed");
            return EH_ECUDA;
        }
    }
    for (uint32_t i = 0; i < dn; ++i) {
        if (dx[i] > xo.light_max) heavy.push_back(xs[i]);
        else if (dx[i] >= 3) light.push_back(xs[i]);
    }
    uint32_t *d_items = nullptr;
    EH_TRY(dev_alloc(&d_items, heavy.size() + light.size(), s));
    eh_status st = EH_OK;
    if (!heavy.empty() &&
        cudaMemcpyAsync(d_items, heavy.data(), heavy.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = EH_ECUDA;
    if (st == EH_OK && !light.empty() &&
        cudaMemcpyAsync(d_items + heavy.size(), light.data(), light.size() * 4, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        st = EH_ECUDA;
    if (st == EH_OK) {
        Items it;
        it.heavy = d_items;
        it.n_heavy = (uint32_t)heavy.size();
        it.light = d_items + heavy.size();
        it.n_light = (uint32_t)light.size();
        it.a_off = t->d_soff;
        it.a_nbr = t->d_snbr;
        it.a_len = t->d_deg;
        st = run_items<P_K4>(t, it, nullptr, xo, s, nullptr, 0, total);
    } else {
        eh_set_error("sk4: copying the selected items failed");
    }
    cudaStreamSynchronize(s);
    dev_free(d_items, s);
    return st;
}

}  // namespace

extern "C" eh_status eh_list(const eh_trie *trie, eh_pattern pattern, const eh_exec_opts *xopts, void *stream,
                             uint32_t *d_out, uint64_t capacity, uint64_t *out_n) {
    if (!trie || !out_n) { eh_set_error("eh_list: NULL argument"); return EH_EINVAL; }
    if (pattern != EH_TRIANGLE && pattern != EH_CLIQUE4) {
        eh_set_error("eh_list: only EH_TRIANGLE and EH_CLIQUE4 have rows to list");
        return EH_EINVAL;
    }
    if (!d_out && capacity) { eh_set_error("eh_list: NULL buffer with a non-zero capacity"); return EH_EINVAL; }
    const uintptr_t align = pattern == EH_CLIQUE4 ? 16 : 4;
    if ((uintptr_t)d_out % align) {
        eh_set_error("eh_list: the buffer must be %u-byte aligned", (unsigned)align);
        return EH_EINVAL;
    }
    *out_n = 0;
    eh_trie *t = const_cast<eh_trie *>(trie);
    cudaStream_t s = (cudaStream_t)stream;
    const eh_exec_opts xo = eh_exec_defaults(xopts);
    std::lock_guard<std::mutex> g(t->call_mu);
    return pattern == EH_TRIANGLE ? run_list<P_TRI>(t, xo, s, d_out, capacity, out_n)
                                  : run_list<P_K4>(t, xo, s, d_out, capacity, out_n);
}

// SK4 (Sec. 5.3): 6 x the 4-cliques through each neighbour x of the selected
// vertex, summed over x (original-id lookup and overflow checks in api.cu)
eh_status eh_sk4_total(eh_trie *t, uint32_t node_new, const eh_exec_opts &xo, cudaStream_t s, uint64_t *total) {
    return sk4_total(t, node_new, xo, s, total);
}
