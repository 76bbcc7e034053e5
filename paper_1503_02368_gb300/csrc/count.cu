// count.cu -- the intersection kernels of the pattern counts.
//
// Triangle (EmptyHeaded Sec. 3.3.2 loop nest, on the degree-pruned trie of
// App. A.1.2):  T = sum_u sum_{v in N+(u)} |N+(u) ∩ N+(v)|.
// For u, the set A = N+(u) is staged once on chip and reused by every v.
// Because N+(v) ⊂ [0, v) and A is sorted, only the prefix A_<v = A[0..j) of
// A (v = A[j]) can meet N+(v); every intersection below works on that prefix.
//
// Each intersection A ∩ B, B = N+(v), picks its algorithm from the layout
// pair and the sizes, as the paper's execution engine does (Sec. 4.2):
//   A bitmap  ∩ B bitset : 128-bit AND of the overlapping words + popc      (bitset ∩ bitset)
//   A bitmap  ∩ B uint   : each element of B probes one bit of A            (uint ∩ bitset)
//   A sorted  ∩ B bitset : each element of A_<v probes one bit of B         (uint ∩ bitset)
//   A sorted  ∩ B uint   : |B| > ratio*|A_<v| -> binary search of A_<v in B (galloping side)
//                          otherwise          -> B streamed in 128-element chunks against
//                                                the window of A_<v the chunk spans (merge)
// A is a bitmap when its stored layout is a bitset, or when its value range
// fits the CTA's shared-memory budget (an on-chip re-encoding of the stored
// uint array).  Work is split by degree: vertices with |N+(u)| > light_max get
// a whole CTA whose warps share the staged A and take the v's dynamically;
// lighter ones get one warp each, A held one element per lane.
#include "eh_internal.cuh"
#include "dev_util.cuh"

namespace {

using namespace ehd;

// the checked build's per-CTA table of the arrays a count kernel reads
// (thread 0, before the kernel's first barrier)
#ifdef EH_CHECK_LOADS
__device__ __forceinline__ void chk_trie(const TrieView &tv, const uint32_t *heavy, uint32_t nh, const uint32_t *light,
                                         uint32_t nl, uint32_t *status) {
    chk_reset(status);
    chk_add(tv.nbr, tv.n_nbr * 4);
    chk_add(tv.words, tv.n_words * 4);
    chk_add(tv.deg, (uint64_t)tv.n * 4);
    chk_add(tv.desc, (uint64_t)tv.n * sizeof(SetDesc));
    chk_add(heavy, (uint64_t)nh * 4);
    chk_add(light, (uint64_t)nl * 4);
}
__device__ __forceinline__ void chk_batch(const BatchView &b, const uint32_t *heavy, uint32_t nh,
                                          const uint32_t *light, uint32_t nl, uint32_t *status) {
    chk_reset(status);
    chk_add(b.desc, b.n_sub * sizeof(SetDesc));
    chk_add(b.nbr, b.n_nbr * 4);
    chk_add(b.words, b.n_words * 4);
    chk_add(b.deg, b.n_sub * 4);
    chk_add(b.sub_q, b.n_sub * 4);
    chk_add(b.qbase, (b.n_queries + 1) * 4);
    chk_add(b.qpat, b.n_queries * 4);
    chk_add(heavy, (uint64_t)nh * 4);
    chk_add(light, (uint64_t)nl * 4);
}
#define CHK_TRIE(tv, h, nh, l, nl, st) chk_trie(tv, h, nh, l, nl, st)
#define CHK_BATCH(b, h, nh, l, nl, st) chk_batch(b, h, nh, l, nl, st)
#define CHK_ADD(p, bytes) chk_add(p, bytes)
#else
#define CHK_TRIE(tv, h, nh, l, nl, st) ((void)0)
#define CHK_BATCH(b, h, nh, l, nl, st) ((void)0)
#define CHK_ADD(p, bytes) ((void)0)
#endif

constexpr uint32_t BM_CAP_WORDS = 8192;        // 32 KB on-chip bitmap: value ranges up to 262,144

enum { M_COUNT = 0, M_LOLLI = 1, M_VERTEX = 2, M_APEX = TRI_MODE_APEX };

struct Acc {
    unsigned long long t;   // triangles
    unsigned long long s;   // sum over triangles of d(a)+d(b)+d(c)  (lollipop)
};

// --------------------------------------------------------------- matches

// (per-vertex mode: cnt, when given, is the staged vertex's shared counter
// array and r the position of w in its set; else w's global counter)
template <int MODE>
__device__ __forceinline__ void on_match(Acc &acc, uint32_t w, uint32_t duv, const TrieView &tv,
                                         unsigned long long *vt, uint32_t *cnt = nullptr, uint32_t r = 0) {
    acc.t += 1;
    if (MODE == M_LOLLI) acc.s += duv + ldg1(&tv.deg[w]);
    if (MODE == M_VERTEX) {
        if (cnt) atomicAdd(&cnt[r], 1u);
        else atomicAdd(&vt[w], 1ull);
    }
}

// Per-vertex triangle counts of a heavy vertex u (the barbell's and the
// selection's triangle nodes, eh_vertex_triangles): the triangles of each
// element of A = N+(u) are counted in shared memory, cnt[i] for A[i], and
// added to the global counters once per element when u is done -- one
// global atomic per (u, element) instead of one per triangle (hub vertices
// sit in millions of triangles).  A match w in the on-chip bitmap is found at
// position sP[g] + (bits before it in its 128-bit group g) of A.
constexpr uint32_t VT_CAP = 2048;   // elements of A counted on chip
struct RankStage {
    uint32_t *cnt;       // nullptr: counts go straight to the global counters
    const uint16_t *sP;  // set bits of the bitmap's groups [0, g)
};
// shared words of the staging: counters, group prefixes, one word per warp
constexpr uint32_t VT_WORDS = VT_CAP + BM_CAP_WORDS / 8 + 32;

__device__ __forceinline__ uint32_t popc4(const uint32_t *p) {
    const uint4 g = *reinterpret_cast<const uint4 *>(p);
    return __popc(g.x) + __popc(g.y) + __popc(g.z) + __popc(g.w);
}

// sP[g] = set bits of the 128-bit groups [0, g) of the bitmap sA (ng groups):
// each warp scans its contiguous segment of groups in rounds of 32 after the
// warps' totals are combined (contains a CTA barrier)
template <int WARPS>
__device__ __forceinline__ void bitmap_prefix(const uint32_t *sA, uint32_t ng, uint16_t *sP, uint32_t *s_tmp) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t seg = (ng + WARPS - 1) / WARPS, b = min(ng, warp * seg), e = min(ng, b + seg);
    uint32_t c = 0;
    for (uint32_t g = b + lane; g < e; g += 32) c += popc4(sA + 4 * g);
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if (lane == 0) s_tmp[warp] = c;
    __syncthreads();
    uint32_t run = 0;
    for (uint32_t k = 0; k < warp; ++k) run += s_tmp[k];
    for (uint32_t g0 = b; g0 < e; g0 += 32) {
        const uint32_t g = g0 + lane;
        const uint32_t x = g < e ? popc4(sA + 4 * g) : 0u;
        uint32_t incl = x;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= (uint32_t)d) incl += y;
        }
        if (g < e) sP[g] = (uint16_t)(run + incl - x);
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// all set bits of x (value base + bit) are matches
template <int MODE>
__device__ __forceinline__ void on_word(Acc &acc, uint32_t x, uint32_t base, uint32_t duv, const TrieView &tv,
                                        unsigned long long *vt) {
    if (MODE == M_COUNT || MODE == M_APEX) {
        acc.t += __popc(x);
    } else {
        while (x) {
            uint32_t b = __ffs(x) - 1;
            x &= x - 1;
            on_match<MODE>(acc, base + b, duv, tv, vt);
        }
    }
}

// ------------------------------------------------------ per-pair routines

// A bitmap (shared memory, words [a_lo, a_lo+a_nw)) ∩ B
template <int MODE>
__device__ __forceinline__ void pair_bitmap(const TrieView &tv, const uint32_t *sA, uint32_t a_lo, uint32_t a_nw,
                                            const SetDesc &dv, uint32_t duv, Acc &acc, unsigned long long *vt) {
    const int lane = threadIdx.x & 31;
    if (dv.nwords) {
        uint32_t lo = max(a_lo, dv.lo_word), hi = min(a_lo + a_nw, dv.lo_word + dv.nwords);
        uint32_t ov = hi > lo ? hi - lo : 0;
        if (ov <= dv.len) {   // fewer words than elements: bitset ∩ bitset
            const uint32_t *bw = tv.words + dv.woff - dv.lo_word;
            for (uint32_t i = lo + lane * 4; i < hi; i += 128) {
                uint4 b = ldg4(bw + i);
                uint4 a = *reinterpret_cast<const uint4 *>(sA + (i - a_lo));
                on_word<MODE>(acc, a.x & b.x, i * 32, duv, tv, vt);
                on_word<MODE>(acc, a.y & b.y, i * 32 + 32, duv, tv, vt);
                on_word<MODE>(acc, a.z & b.z, i * 32 + 64, duv, tv, vt);
                on_word<MODE>(acc, a.w & b.w, i * 32 + 96, duv, tv, vt);
            }
            return;
        }
    }
    // uint B: each element probes A's bitmap (padding EH_PAD is out of range);
    // two 128-bit loads in flight per lane
    const uint32_t *bp = tv.nbr + dv.off;
    const uint32_t base = a_lo * 32, nbits = a_nw * 32;
    for (uint32_t p = lane * 4; p < dv.len; p += 256) {
        uint4 e0 = ldg4(bp + p);
        uint4 e1 = p + 128 < dv.len ? ldg4(bp + p + 128) : make_uint4(EH_PAD, EH_PAD, EH_PAD, EH_PAD);
        uint32_t w[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint32_t x = w[c] - base;
            if (x < nbits && ((sA[x >> 5] >> (x & 31)) & 1u)) on_match<MODE>(acc, w[c], duv, tv, vt);
        }
    }
}

// A sorted array (shared or global), effective prefix A[0..j) ∩ B
// (cnt: the per-vertex mode's shared counters of A, indexed like A, or nullptr)
template <int MODE>
__device__ __forceinline__ void pair_sorted(const TrieView &tv, const uint32_t *A, uint32_t j, const SetDesc &dv,
                                            uint32_t duv, uint32_t ratio, Acc &acc, unsigned long long *vt,
                                            uint32_t *cnt = nullptr) {
    const int lane = threadIdx.x & 31;
    if (dv.nwords && j <= dv.len) {   // uint ∩ bitset: probe A's elements
        const uint32_t *bw = tv.words + dv.woff;
        const uint32_t base = dv.lo_word * 32, nbits = dv.nwords * 32;
        for (uint32_t i = lane; i < j; i += 32) {
            uint32_t a = ld_any(&A[i]), x = a - base;
            if (x < nbits && ((ldg1(&bw[x >> 5]) >> (x & 31)) & 1u)) on_match<MODE>(acc, a, duv, tv, vt, cnt, i);
        }
        return;
    }
    const uint32_t *B = tv.nbr + dv.off;
    if ((uint64_t)dv.len > (uint64_t)ratio * j) {   // galloping side: search A's elements in B
        for (uint32_t i = lane; i < j; i += 32) {
            uint32_t a = ld_any(&A[i]);
            uint32_t pos = lower_bound(B, 0, dv.len, a);
            if (pos < dv.len && ldg1(&B[pos]) == a) on_match<MODE>(acc, a, duv, tv, vt, cnt, i);
        }
        return;
    }
    // merge side: B in 128-element chunks; each chunk meets the window of A it spans
    uint32_t wlo = 0;
    for (uint32_t c = 0; c < dv.len; c += 128) {
        uint32_t p = c + lane * 4;
        uint4 e = p < dv.len ? ldg4(B + p) : make_uint4(EH_PAD, EH_PAD, EH_PAD, EH_PAD);
        uint32_t bmin = __shfl_sync(FULL, e.x, 0);
        uint32_t mx = e.w != EH_PAD ? e.w : e.z != EH_PAD ? e.z : e.y != EH_PAD ? e.y : e.x != EH_PAD ? e.x : 0u;
        uint32_t bmax = __reduce_max_sync(FULL, mx);
        uint32_t lo = 0, hi = 0;
        if (lane == 0) lo = lower_bound(A, wlo, j, bmin);
        if (lane == 1) hi = lower_bound(A, wlo, j, bmax + 1);
        lo = __shfl_sync(FULL, lo, 0);
        hi = __shfl_sync(FULL, hi, 1);
        wlo = lo;
        if (hi <= lo) continue;
        uint32_t w[4] = {e.x, e.y, e.z, e.w};
        if (hi - lo <= 8) {
            for (uint32_t i = lo; i < hi; ++i) {
                uint32_t a = ld_any(&A[i]);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (w[k] == a) on_match<MODE>(acc, a, duv, tv, vt, cnt, i);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (w[k] == EH_PAD) continue;
                uint32_t pos = lower_bound(A, lo, hi, w[k]);
                if (pos < hi && ld_any(&A[pos]) == w[k]) on_match<MODE>(acc, w[k], duv, tv, vt, cnt, pos);
            }
        }
    }
}

// A held one element per lane (lanes < eff active, sorted): is the lane's
// element in B?  The algorithm follows the layout pair and the sizes.
__device__ __forceinline__ bool light_match(const TrieView &tv, uint32_t a, uint32_t eff, const SetDesc &dB,
                                            uint32_t ratio) {
    const int lane = threadIdx.x & 31;
    const bool act = (uint32_t)lane < eff;
    if (dB.nwords && eff <= dB.len) {   // uint ∩ bitset: probe one bit
        uint32_t x = a - dB.lo_word * 32;
        return act && x < dB.nwords * 32 && ((ldg1(&tv.words[dB.woff + (x >> 5)]) >> (x & 31)) & 1u);
    }
    const uint32_t *B = tv.nbr + dB.off;
    if ((uint64_t)dB.len > (uint64_t)ratio * eff) {   // galloping side: binary search in B
        if (!act) return false;
        uint32_t pos = lower_bound(B, 0, dB.len, a);
        return pos < dB.len && ldg1(&B[pos]) == a;
    }
    // merge side: B in 128-element chunks against the lanes whose value falls in the chunk's span
    bool hit = false;
    for (uint32_t c = 0; c < dB.len; c += 128) {
        uint32_t p = c + lane * 4;
        uint4 e = p < dB.len ? ldg4(B + p) : make_uint4(EH_PAD, EH_PAD, EH_PAD, EH_PAD);
        uint32_t bmin = __shfl_sync(FULL, e.x, 0);
        uint32_t mx = e.w != EH_PAD ? e.w : e.z != EH_PAD ? e.z : e.y != EH_PAD ? e.y : e.x != EH_PAD ? e.x : 0u;
        uint32_t bmax = __reduce_max_sync(FULL, mx);
        uint32_t win = __ballot_sync(FULL, act && a >= bmin && a <= bmax);
        while (win) {
            uint32_t i = __ffs(win) - 1;
            win &= win - 1;
            uint32_t ai = __shfl_sync(FULL, a, i);
            bool any = __any_sync(FULL, e.x == ai || e.y == ai || e.z == ai || e.w == ai);
            if (any && (uint32_t)lane == i) hit = true;
        }
    }
    return hit;
}

// light vertex: A = N+(u) (2 <= |A| <= 32) one element per lane
template <int MODE>
__device__ void light_vertex(const TrieView &tv, uint32_t u, uint32_t ratio, Acc &acc, unsigned long long *vt) {
    const int lane = threadIdx.x & 31;
    const SetDesc du = ld_desc(&tv.desc[u]);
    const uint32_t k = du.len;
    const uint32_t a = lane < k ? ldg1(&tv.nbr[du.off + lane]) : EH_PAD;
    const SetDesc mine = (lane >= 1 && lane < k) ? ld_desc(&tv.desc[a]) : empty_desc();
    // per-vertex triangle counts: each lane counts the triangles of its own
    // element a (as the lowest vertex w, or as v when its pair is processed),
    // lane 0 those of u; one atomic per element and vertex at the end
    unsigned long long mine_t = 0, u_t = 0;
    for (uint32_t j = 1; j < k; ++j) {
        const SetDesc dv = bcast_desc(mine, j);
        if (dv.len == 0) continue;
        const bool hit = light_match(tv, a, j, dv, ratio);
        if (MODE == M_VERTEX) {
            const uint32_t pc = __popc(__ballot_sync(FULL, hit));
            acc.t += hit ? 1u : 0u;
            mine_t += (hit ? 1u : 0u) + ((uint32_t)lane == j ? pc : 0u);
            u_t += pc;
        } else if (hit) {
            on_match<MODE>(acc, a, du.deg + dv.deg, tv, vt);
        }
    }
    if (MODE == M_VERTEX) {
        if ((uint32_t)lane < k && mine_t) atomicAdd(&vt[a], mine_t);
        if (lane == 0 && u_t) atomicAdd(&vt[u], u_t);
    }
}

// ------------------------------------------------------------ heavy items
//
// A heavy vertex gets the whole CTA: A = N+(u) is staged once (bitset words
// copied by cp.async.bulk when A is stored as a bitset of at most 4 words per
// element, or a bitmap built from the uint array when its range fits, or the
// sorted array copied by cp.async.bulk), then the warps take the v = A[j]
// dynamically through a shared counter.

struct StagedA {
    const uint32_t *Ag;   // A in global memory
    const uint32_t *A;    // A as a sorted array (shared or global) when amode != 0
    uint32_t len, a_lo, a_nw;
    int amode;            // 0 bitmap in shared memory, 1 sorted in shared memory, 2 sorted in global memory
};

// A pair's plan against an on-chip bitmap A, computed by the lane that holds
// the pair's descriptor: kind 1 = 128-bit AND over words [begin, end) of
// `base`, kind 2 = B's elements [0, end) of `base` probe A, 0 = nothing.
__device__ __forceinline__ void bitmap_plan(const TrieView &tv, uint32_t a_lo, uint32_t a_nw, const SetDesc &dv,
                                            uint32_t &kind, int64_t &base, uint32_t &begin, uint32_t &end) {
    kind = 0;
    base = 0;
    begin = end = 0;
    if (dv.len == 0) return;
    if (dv.nwords) {
        const uint32_t lo = max(a_lo, dv.lo_word), hi = min(a_lo + a_nw, dv.lo_word + dv.nwords);
        const uint32_t ov = hi > lo ? hi - lo : 0;
        // a word of the AND covers 32 values; it pays up to 1.5 words per element (measured)
        if (2 * ov <= 3 * dv.len) {
            kind = ov ? 1u : 0u;
            base = (int64_t)dv.woff - (int64_t)dv.lo_word;   // word w of B is words[base + w]
            begin = lo;
            end = hi;
            return;
        }
    }
    kind = 2;
    base = (int64_t)dv.off;
    end = dv.len;
}

// PW warps share one pair: this warp takes part `part` of B's range (every
// PW-th step of 128 words or 256 elements)
template <int MODE, int PW = 1>
__device__ __forceinline__ void run_plan(const TrieView &tv, const uint32_t *sA, uint32_t a_lo, uint32_t a_nw,
                                         uint32_t kind, int64_t base, uint32_t begin, uint32_t end, uint32_t duv,
                                         Acc &acc, unsigned long long *vt, uint32_t part = 0,
                                         const RankStage *rs = nullptr) {
    const uint32_t lane4 = (threadIdx.x & 31) * 4;
    if (MODE == M_VERTEX) {   // staged per-element counters (tri_heavy takes this path only with rs)
        if (kind == 1) {
            const uint32_t *bw = tv.words + base;
            for (uint32_t i = begin + lane4; i < end; i += 128) {
                const uint4 b = ldg4(bw + i);
                const uint4 a = *reinterpret_cast<const uint4 *>(sA + (i - a_lo));
                const uint32_t aw[4] = {a.x, a.y, a.z, a.w}, bw4[4] = {b.x, b.y, b.z, b.w};
                uint32_t p = rs->sP[(i - a_lo) >> 2];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t x = aw[q] & bw4[q];
                    acc.t += __popc(x);
                    while (x) {
                        const uint32_t bit = __ffs(x) - 1;
                        x &= x - 1;
                        atomicAdd(&rs->cnt[p + __popc(aw[q] & ((1u << bit) - 1u))], 1u);
                    }
                    p += __popc(aw[q]);
                }
            }
        } else if (kind == 2) {
            const uint32_t *bp = tv.nbr + base;
            const uint32_t abase = a_lo * 32, nbits = a_nw * 32;
            for (uint32_t p = lane4; p < end; p += 256) {
                const uint4 e0 = ldg4(bp + p);
                const uint4 e1 = p + 128 < end ? ldg4(bp + p + 128) : make_uint4(EH_PAD, EH_PAD, EH_PAD, EH_PAD);
                const uint32_t w[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint32_t x = w[c] - abase;
                    if (x < nbits && ((sA[x >> 5] >> (x & 31)) & 1u)) {
                        // the 128-bit group holding x: A's position of its first element, bits before x
                        const uint4 g = *reinterpret_cast<const uint4 *>(sA + ((x >> 7) << 2));
                        const uint32_t q = (x >> 5) & 3u;
                        const uint32_t aw = q == 0 ? g.x : q == 1 ? g.y : q == 2 ? g.z : g.w;
                        const uint32_t before = (q > 0 ? __popc(g.x) : 0u) + (q > 1 ? __popc(g.y) : 0u) +
                                                (q > 2 ? __popc(g.z) : 0u);
                        acc.t += 1;
                        atomicAdd(&rs->cnt[rs->sP[x >> 7] + before + __popc(aw & ((1u << (x & 31)) - 1u))], 1u);
                    }
                }
            }
        }
        return;
    }
    if (kind == 1) {
        const uint32_t *bw = tv.words + base;
        for (uint32_t i = begin + part * 128 + lane4; i < end; i += 128 * PW) {
            const uint4 b = ldg4(bw + i);
            const uint4 a = *reinterpret_cast<const uint4 *>(sA + (i - a_lo));
            on_word<MODE>(acc, a.x & b.x, i * 32, duv, tv, vt);
            on_word<MODE>(acc, a.y & b.y, i * 32 + 32, duv, tv, vt);
            on_word<MODE>(acc, a.z & b.z, i * 32 + 64, duv, tv, vt);
            on_word<MODE>(acc, a.w & b.w, i * 32 + 96, duv, tv, vt);
        }
    } else if (kind == 2) {
        const uint32_t *bp = tv.nbr + base;
        const uint32_t abase = a_lo * 32, nbits = a_nw * 32;
        for (uint32_t p = part * 256 + lane4; p < end; p += 256 * PW) {
            const uint4 e0 = ldg4(bp + p);
            const uint4 e1 = p + 128 < end ? ldg4(bp + p + 128) : make_uint4(EH_PAD, EH_PAD, EH_PAD, EH_PAD);
            const uint32_t w[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint32_t x = w[c] - abase;
                if (x < nbits && ((sA[x >> 5] >> (x & 31)) & 1u)) on_match<MODE>(acc, w[c], duv, tv, vt);
            }
        }
    }
}

// Returns false when the bounded wait for the bulk copy ran out (every thread
// of the CTA then returns false; the caller must leave the kernel).
template <int WARPS>
__device__ __forceinline__ bool stage_set(const TrieView &tv, const SetDesc &du, uint32_t *sA, uint64_t *mbar,
                                          uint32_t &phase, StagedA &st, uint32_t *status) {
    const int tid = threadIdx.x;
    st.len = du.len;
    st.Ag = tv.nbr + du.off;
    const uint32_t first = ldg1(&st.Ag[0]), last = ldg1(&st.Ag[st.len - 1]);
    st.a_lo = (first >> 7) << 2;
    st.a_nw = (((last >> 5) + 1 - st.a_lo) + 3) & ~3u;
    bool copy = false;
    // a stored bitset is copied whole when it is not much larger than the uint
    // array (at most 4 words per element); a sparser one is rebuilt on chip from
    // the elements below, which reads 4|A| bytes instead of 4 x its words
    if (du.nwords && du.nwords <= BM_CAP_WORDS && du.nwords <= 4ull * du.len &&
        bulk_src_ok(tv.words + du.woff, du.nwords * 4)) {
        st.amode = 0;
        st.a_lo = du.lo_word;
        st.a_nw = du.nwords;
        copy = true;
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(mbar, st.a_nw * 4);
            bulk_g2s(sA, tv.words + du.woff, st.a_nw * 4, mbar);
        }
    } else if (st.a_nw <= BM_CAP_WORDS) {
        st.amode = 0;
        for (uint32_t i = tid * 4; i < st.a_nw; i += WARPS * 128)
            *reinterpret_cast<uint4 *>(sA + i) = make_uint4(0, 0, 0, 0);
        __syncthreads();
        for (uint32_t i = tid; i < st.len; i += WARPS * 32) {
            uint32_t x = ldg1(&st.Ag[i]);
            atomicOr(&sA[(x >> 5) - st.a_lo], 1u << (x & 31));
        }
    } else if (st.len <= BM_CAP_WORDS && bulk_src_ok(st.Ag, ((st.len + 3) & ~3u) * 4)) {
        st.amode = 1;
        copy = true;
        if (tid == 0) {
            uint32_t bytes = ((st.len + 3) & ~3u) * 4;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(mbar, bytes);
            bulk_g2s(sA, st.Ag, bytes, mbar);
        }
    } else {
        st.amode = 2;
    }
    if (copy) {
        bool ok = mbar_wait(mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(status, DEV_ST_TIMEOUT);
            mbar_wait(mbar, phase ^ 1);   // drain the copy still in flight, bounded
            return false;
        }
    } else {
        __syncthreads();
    }
    st.A = st.amode == 2 ? st.Ag : sA;
    return true;
}

constexpr uint32_t PAIR_BATCH = 4;   // pairs a warp takes at a time from its CTA's vertex

// One grab of the count and lollipop modes against the on-chip bitmap: a
// quarter warp per pair.  The quarter's 8 lanes load its pair's descriptor
// (one address a quarter) and plan it; the AND pairs then run side by side,
// 8 lanes x 4 words a step with the four pairs' loads in flight together, and
// the probe pairs one after another on the whole warp.  Against one pair per
// warp in turn this drops the per-pair broadcasts and most steps of short AND
// pairs (half of them are 80 words or fewer on R-MAT).  The lollipop walks
// the set bits of its AND words, each match adding d(u) + d(v) + d(w).
static_assert(PAIR_BATCH == 4, "one quarter warp per pair of a grab");
template <int MODE>
__device__ __forceinline__ void quarter_grab(const TrieView &tv, const uint32_t *sA, const StagedA &st, uint32_t j0,
                                             uint32_t du_deg, Acc &acc, unsigned long long *vt) {
    const uint32_t lane = threadIdx.x & 31, jq = j0 + (lane >> 3);
    uint32_t kind = 0, b = 0, e = 0, duv = 0;
    int64_t base = 0;
    if (jq < st.len) {
        const SetDesc dq = ld_desc(&tv.desc[ldg1(&st.Ag[jq])]);
        bitmap_plan(tv, st.a_lo, st.a_nw, dq, kind, base, b, e);
        if constexpr (MODE == M_LOLLI) duv = du_deg + dq.deg;
    }
    if (kind == 1) {
        const uint32_t *bw = tv.words + base;
        uint32_t c = 0;
        for (uint32_t i = b + (lane & 7) * 4; i < e; i += 32) {
            const uint4 bv = ldg4(bw + i);
            const uint4 av = *reinterpret_cast<const uint4 *>(sA + (i - st.a_lo));
            if constexpr (MODE == M_LOLLI) {
                on_word<MODE>(acc, av.x & bv.x, i * 32, duv, tv, vt);
                on_word<MODE>(acc, av.y & bv.y, i * 32 + 32, duv, tv, vt);
                on_word<MODE>(acc, av.z & bv.z, i * 32 + 64, duv, tv, vt);
                on_word<MODE>(acc, av.w & bv.w, i * 32 + 96, duv, tv, vt);
            } else {
                c += __popc(av.x & bv.x) + __popc(av.y & bv.y) + __popc(av.z & bv.z) + __popc(av.w & bv.w);
            }
        }
        acc.t += c;
    }
    __syncwarp();
    for (uint32_t q = 0; q < 4; ++q) {
        if (__shfl_sync(FULL, kind, 8 * q) != 2) continue;
        run_plan<MODE, 1>(tv, sA, st.a_lo, st.a_nw, 2u, __shfl_sync(FULL, base, 8 * q), 0u,
                          __shfl_sync(FULL, e, 8 * q), MODE == M_LOLLI ? __shfl_sync(FULL, duv, 8 * q) : 0u, acc, vt);
    }
}

// light items a warp takes per grab: 32 when the list gives every resident
// warp at least 4 such grabs (the atomic amortised), fewer on short lists so
// that the items spread over more warps (small graphs, small batches)
__device__ __forceinline__ uint32_t light_chunk(uint32_t n_light, uint32_t warps_per_cta) {
    const uint64_t warps = (uint64_t)gridDim.x * warps_per_cta;
    const uint64_t c = n_light / (4 * warps);
    return c >= 32 ? 32u : c < 1 ? 1u : (uint32_t)c;
}

__device__ __forceinline__ uint32_t next_j(uint32_t *s_next, uint32_t batch = PAIR_BATCH) {
    uint32_t j = 0;
    if ((threadIdx.x & 31) == 0) j = atomicAdd(s_next, batch);
    return __shfl_sync(FULL, j, 0);
}

// Warps per intersection: with PW > 1 the warps of the CTA take work units
// (pair j, part p), p < PW, so that PW warps share each pair's B against the
// on-chip bitmap (every PW-th step of its range each, run_plan); the other
// dispatches run the whole pair in part 0.  PW = 1 is one pair per warp.
// s_rank: VT_WORDS shared words for the per-vertex mode's staged counters, or
// nullptr (then every match adds to its global counter)
template <int MODE, int WARPS, int PW = 1>
__device__ __forceinline__ bool tri_heavy(const TrieView &tv, uint32_t u, uint32_t ratio, uint32_t *sA,
                                          uint64_t *mbar, uint32_t &phase, uint32_t *s_next, Acc &acc,
                                          uint32_t *status, unsigned long long *vt, uint32_t *s_rank = nullptr) {
    const int lane = threadIdx.x & 31;
    const SetDesc du = ld_desc(&tv.desc[u]);
    if (threadIdx.x == 0) *s_next = PW;   // the first unit of pair 1
    StagedA st;
    if (!stage_set<WARPS>(tv, du, sA, mbar, phase, st, status)) return false;
    const uint32_t n_units = st.len * PW;
    const unsigned long long t_start = acc.t;   // u's triangles, added once per vertex (per-vertex mode)
    RankStage rs{nullptr, nullptr};
    if (MODE == M_VERTEX && s_rank && st.len <= VT_CAP) {
        uint16_t *sP = reinterpret_cast<uint16_t *>(s_rank + VT_CAP);
        for (uint32_t i = threadIdx.x; i < st.len; i += WARPS * 32) s_rank[i] = 0;
        if (st.amode == 0) bitmap_prefix<WARPS>(sA, st.a_nw / 4, sP, s_rank + VT_CAP + BM_CAP_WORDS / 8);
        __syncthreads();
        rs.cnt = s_rank;
        rs.sP = sP;
    }
    for (;;) {
        const uint32_t j0 = next_j(s_next);   // first unit of this grab
        if (j0 >= n_units) break;
        if constexpr ((MODE == M_COUNT || MODE == M_APEX || MODE == M_LOLLI) && PW == 1) {
            if (st.amode == 0) {
                quarter_grab<MODE>(tv, sA, st, j0, du.deg, acc, vt);
                continue;
            }
        }
        // the next PAIR_BATCH units: their pair's v and descriptor loaded one per lane
        const uint32_t jl = (j0 + lane) / PW;
        uint32_t vl = 0;
        SetDesc mine = empty_desc();
        if (lane < PAIR_BATCH && jl < st.len) {
            vl = st.amode == 0 ? ldg1(&st.Ag[jl]) : ld_any(&st.A[jl]);
            mine = ld_desc(&tv.desc[vl]);
        }
        const uint32_t nb = min(PAIR_BATCH, n_units - j0);
        if (st.amode == 0 && (MODE != M_VERTEX || rs.cnt)) {
            // each descriptor lane plans its unit's pair; the warp runs the plans in turn
            uint32_t pk, pb, pe;
            int64_t pbase;
            bitmap_plan(tv, st.a_lo, st.a_nw, mine, pk, pbase, pb, pe);
            const uint32_t pduv = du.deg + mine.deg;
            for (uint32_t i = 0; i < nb; ++i) {
                const uint32_t kind = __shfl_sync(FULL, pk, i);
                if (kind == 0) continue;
                const unsigned long long t0 = acc.t;
                run_plan<MODE, PW>(tv, sA, st.a_lo, st.a_nw, kind, __shfl_sync(FULL, pbase, i),
                                   __shfl_sync(FULL, pb, i), __shfl_sync(FULL, pe, i),
                                   MODE == M_LOLLI ? __shfl_sync(FULL, pduv, i) : 0u, acc, vt, (j0 + i) % PW, &rs);
                if (MODE == M_VERTEX) {   // v = A[j] is at position j of A
                    unsigned long long pc = acc.t - t0;
                    for (int d = 16; d > 0; d >>= 1) pc += __shfl_xor_sync(FULL, pc, d);
                    if (lane == 0 && pc) atomicAdd(&rs.cnt[j0 + i], (uint32_t)pc);
                }
            }
            continue;
        }
        for (uint32_t i = 0; i < nb; ++i) {
            if ((j0 + i) % PW != 0) continue;   // the whole pair runs in its first unit
            const uint32_t j = (j0 + i) / PW;
            const uint32_t v = __shfl_sync(FULL, vl, i);
            const SetDesc dv = bcast_desc(mine, i);
            if (dv.len == 0) continue;
            const uint32_t duv = du.deg + dv.deg;
            unsigned long long t0 = acc.t;
            if (st.amode == 0) pair_bitmap<MODE>(tv, sA, st.a_lo, st.a_nw, dv, duv, acc, vt);
            else pair_sorted<MODE>(tv, st.A, j, dv, duv, ratio, acc, vt, rs.cnt);
            if (MODE == M_VERTEX) {
                unsigned long long pc = acc.t - t0;
                for (int d = 16; d > 0; d >>= 1) pc += __shfl_xor_sync(FULL, pc, d);
                if (lane == 0 && pc) {
                    if (rs.cnt) atomicAdd(&rs.cnt[j], (uint32_t)pc);
                    else atomicAdd(&vt[v], pc);
                }
            }
        }
    }
    if (MODE == M_VERTEX) {
        unsigned long long tu = acc.t - t_start;
        for (int d = 16; d > 0; d >>= 1) tu += __shfl_xor_sync(FULL, tu, d);
        if (lane == 0 && tu) atomicAdd(&vt[u], tu);
        if (rs.cnt) {   // the elements' counts, once each
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < st.len; i += WARPS * 32) {
                const uint32_t c = rs.cnt[i];
                if (c) atomicAdd(&vt[ldg1(&st.Ag[i])], (unsigned long long)c);
            }
        }
    }
    __syncthreads();
    return true;
}

// dynamic shared memory of k_triangle: the staged A, and for the per-vertex
// mode its elements' counters and group prefixes
constexpr int tri_smem_bytes(int mode) { return (int)(BM_CAP_WORDS + (mode == M_VERTEX ? VT_WORDS : 0)) * 4; }

// counters[0]: next heavy item, counters[1]: next light chunk
template <int MODE, int WARPS, int PW = 1>
__global__ void __launch_bounds__(WARPS * 32) k_triangle(TrieView tv, const uint32_t *__restrict__ heavy, uint32_t n_heavy,
                                                         const uint32_t *__restrict__ light, uint32_t n_light,
                                                         uint32_t ratio, unsigned long long *counters,
                                                         unsigned long long *out, uint32_t *status,
                                                         unsigned long long *vt) {
    extern __shared__ __align__(16) uint32_t sA[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_item, s_next;
    __shared__ unsigned long long s_red[MODE == M_APEX ? WARPS : 1];
    const int tid = threadIdx.x, lane = tid & 31;
    Acc acc{0, 0};
    uint32_t phase = 0;
    if (tid == 0) {
        mbar_init(&mbar, 1);
        CHK_TRIE(tv, heavy, n_heavy, light, n_light, status);
    }
    __syncthreads();

    // heavy vertices: one CTA each
    for (;;) {
        if (tid == 0) s_item = (uint32_t)min((unsigned long long)n_heavy, atomicAdd(&counters[0], 1ull));
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_heavy) break;
        const unsigned long long t0 = acc.t;
        if (!tri_heavy<MODE, WARPS, PW>(tv, ldg1(&heavy[item]), ratio, sA, &mbar, phase, &s_next, acc, status, vt,
                                        MODE == M_VERTEX ? sA + BM_CAP_WORDS : nullptr))
            return;
        if (MODE == M_APEX) {   // this vertex's triangles (as the largest id) to vt[item]
            unsigned long long d = acc.t - t0;
            for (int k = 16; k > 0; k >>= 1) d += __shfl_xor_sync(FULL, d, k);
            if (lane == 0) s_red[tid >> 5] = d;
            __syncthreads();
            if (tid == 0) {
                unsigned long long c = 0;
                for (int w = 0; w < WARPS; ++w) c += s_red[w];
                vt[item] = c;
            }
        }
    }

    // light vertices: one warp each
    const uint32_t chunk = light_chunk(n_light, WARPS);
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&counters[1], (unsigned long long)chunk);
        base = __shfl_sync(FULL, base, 0);
        if (base >= n_light) break;
        uint32_t end = (uint32_t)min((unsigned long long)n_light, base + chunk);
        for (uint32_t i = (uint32_t)base; i < end; ++i) {
            const unsigned long long t0 = acc.t;
            light_vertex<MODE>(tv, ldg1(&light[i]), ratio, acc, vt);
            if (MODE == M_APEX) {   // vt[n_heavy + i]
                unsigned long long d = acc.t - t0;
                for (int k = 16; k > 0; k >>= 1) d += __shfl_xor_sync(FULL, d, k);
                if (lane == 0) vt[n_heavy + i] = d;
            }
        }
    }

    // reduce: warp, then one atomic per warp
    unsigned long long t = acc.t, s = acc.s;
    for (int d = 16; d > 0; d >>= 1) {
        t += __shfl_xor_sync(FULL, t, d);
        s += __shfl_xor_sync(FULL, s, d);
    }
    if (lane == 0) {
        if (t) atomicAdd(&out[0], t);
        if (MODE == M_LOLLI && s) {
            unsigned long long old = atomicAdd(&out[1], s);
            if (old + s < old) atomicOr(status, DEV_ST_OVERFLOW);
        }
    }
}

// ------------------------------------------------------------------ 4-clique
//
// Table 1's 4Clique on the pruned trie with the attribute order x > y > z > w
// (a single-node GHD is optimal for it, Sec. 5.2.2):
//   for x; for y in N+(x): S = N+(x) ∩ N+(y) (materialised, sorted);
//     for z in S: K4 += |S_<z ∩ N+(z)|.
// Level 1 writes S by warp compaction (ballot / scan of per-lane match
// counts, in increasing order) into a per-warp shared buffer, or into the
// warp's slice of a global arena when |S| may exceed it.  Level 2 runs the
// same layout-dispatched intersection as the triangle on (S_<z, N+(z)).

constexpr uint32_t S_CAP = K4_S_CAP;
constexpr uint32_t K4_PAIR_BATCH = 1;   // (x, y) pairs are heavy and uneven: one at a time
constexpr uint32_t SB_CAP_WORDS = 256;    // per-warp bitmap of S: value ranges up to 8,192
constexpr uint32_t LANE_UINT_MAX = 64;    // a lane walks a uint N+(z) alone up to this length

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t x, uint32_t &total) {
    const int lane = threadIdx.x & 31;
    uint32_t incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += y;
    }
    total = __shfl_sync(FULL, incl, 31);
    return incl - x;
}

// S = A ∩ B, A an on-chip bitmap.  When B is a bitset and their overlap fits
// the warp's bitmap buffer Sbm, the AND words are also written there (words
// [lo, hi) at Sbm[0 ..)) and *bm_lo = lo, so level 2 need not rebuild S's
// bitmap; otherwise *bm_lo = EH_PAD.
__device__ uint32_t emit_bitmap(const TrieView &tv, const uint32_t *sA, uint32_t a_lo, uint32_t a_nw,
                                const SetDesc &dv, uint32_t *S, uint32_t *Sbm, uint32_t *bm_lo) {
    const int lane = threadIdx.x & 31;
    uint32_t ns = 0;
    *bm_lo = EH_PAD;
    if (dv.nwords) {
        uint32_t lo = max(a_lo, dv.lo_word), hi = min(a_lo + a_nw, dv.lo_word + dv.nwords);
        uint32_t ov = hi > lo ? hi - lo : 0;
        if (ov <= dv.len) {
            const uint32_t *bw = tv.words + dv.woff - dv.lo_word;
            const bool keep = Sbm && ov <= SB_CAP_WORDS;
            if (keep) *bm_lo = lo;
            for (uint32_t b0 = lo; b0 < hi; b0 += 128) {
                uint32_t i = b0 + lane * 4;
                uint32_t x[4] = {0, 0, 0, 0};
                if (i < hi) {
                    uint4 b = ldg4(bw + i);
                    uint4 a = *reinterpret_cast<const uint4 *>(sA + (i - a_lo));
                    x[0] = a.x & b.x; x[1] = a.y & b.y; x[2] = a.z & b.z; x[3] = a.w & b.w;
                    if (keep) *reinterpret_cast<uint4 *>(Sbm + (i - lo)) = make_uint4(x[0], x[1], x[2], x[3]);
                }
                uint32_t cnt = __popc(x[0]) + __popc(x[1]) + __popc(x[2]) + __popc(x[3]), tot;
                uint32_t pos = ns + warp_excl_scan(cnt, tot);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t w = x[k];
                    while (w) {
                        uint32_t bb = __ffs(w) - 1;
                        w &= w - 1;
                        S[pos++] = (i + k) * 32 + bb;
                    }
                }
                ns += tot;
            }
            __syncwarp();
            return ns;
        }
    }
    const uint32_t *bp = tv.nbr + dv.off;
    const uint32_t base = a_lo * 32, nbits = a_nw * 32;
    for (uint32_t c = 0; c < dv.len; c += 128) {
        uint32_t p = c + lane * 4;
        uint4 e = p < dv.len ? ldg4(bp + p) : make_uint4(EH_PAD, EH_PAD, EH_PAD, EH_PAD);
        uint32_t w[4] = {e.x, e.y, e.z, e.w};
        uint32_t f = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t x = w[k] - base;
            if (x < nbits && ((sA[x >> 5] >> (x & 31)) & 1u)) f |= 1u << k;
        }
        uint32_t tot;
        uint32_t pos = ns + warp_excl_scan(__popc(f), tot);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (f & (1u << k)) S[pos++] = w[k];
        ns += tot;
    }
    __syncwarp();
    return ns;
}

// S = A[0..j) ∩ B, A sorted (shared or global)
__device__ uint32_t emit_sorted(const TrieView &tv, const uint32_t *A, uint32_t j, const SetDesc &dv, uint32_t ratio,
                                uint32_t *S) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t ns = 0;
    const uint32_t *B = tv.nbr + dv.off;
    const bool probe = dv.nwords && j <= dv.len;
    if (probe || (uint64_t)dv.len > (uint64_t)ratio * j) {
        const uint32_t base = dv.lo_word * 32, nbits = dv.nwords * 32;
        for (uint32_t r = 0; r < j; r += 32) {
            uint32_t i = r + lane;
            bool hit = false;
            uint32_t a = 0;
            if (i < j) {
                a = ld_any(&A[i]);
                if (probe) {
                    uint32_t x = a - base;
                    hit = x < nbits && ((ldg1(&tv.words[dv.woff + (x >> 5)]) >> (x & 31)) & 1u);
                } else {
                    uint32_t pos = lower_bound(B, 0, dv.len, a);
                    hit = pos < dv.len && ldg1(&B[pos]) == a;
                }
            }
            uint32_t m = __ballot_sync(FULL, hit);
            if (hit) S[ns + __popc(m & lt)] = a;
            ns += __popc(m);
        }
        __syncwarp();
        return ns;
    }
    uint32_t wlo = 0;
    for (uint32_t c = 0; c < dv.len; c += 128) {
        uint32_t p = c + lane * 4;
        uint4 e = p < dv.len ? ldg4(B + p) : make_uint4(EH_PAD, EH_PAD, EH_PAD, EH_PAD);
        uint32_t bmin = __shfl_sync(FULL, e.x, 0);
        uint32_t mx = e.w != EH_PAD ? e.w : e.z != EH_PAD ? e.z : e.y != EH_PAD ? e.y : e.x != EH_PAD ? e.x : 0u;
        uint32_t bmax = __reduce_max_sync(FULL, mx);
        uint32_t lo = 0, hi = 0;
        if (lane == 0) lo = lower_bound(A, wlo, j, bmin);
        if (lane == 1) hi = lower_bound(A, wlo, j, bmax + 1);
        lo = __shfl_sync(FULL, lo, 0);
        hi = __shfl_sync(FULL, hi, 1);
        wlo = lo;
        uint32_t w[4] = {e.x, e.y, e.z, e.w};
        uint32_t f = 0;
        if (hi > lo) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (w[k] == EH_PAD) continue;
                uint32_t pos = lower_bound(A, lo, hi, w[k]);
                if (pos < hi && ld_any(&A[pos]) == w[k]) f |= 1u << k;
            }
        }
        uint32_t tot;
        uint32_t pos = ns + warp_excl_scan(__popc(f), tot);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (f & (1u << k)) S[pos++] = w[k];
        ns += tot;
    }
    __syncwarp();
    return ns;
}

// Level 2 over a materialised sorted S: K4 += sum_{z in S} |S_<z ∩ N+(z)|
// (= the edges of G[S]; N+(z) ⊂ [0, z) keeps S's elements >= z out).
//
// When S is dense (its value range needs at most one 32-bit word per element
// and fits the warp's bitmap buffer) it also gets a bitmap, and the warp
// takes 32 z's at a time, one per lane: a lane whose N+(z) is a bitset ANDs
// it with S's bitmap over their overlapping words (128 bits per step), a lane
// whose N+(z) is a short uint array probes S's bitmap with each element.  The
// remaining z's (and every z of a sparse S) run the warp-wide routines, z by
// z, with their descriptors loaded one per lane beforehand.

__device__ __forceinline__ void clique_level2(const TrieView &tv, const uint32_t *S, uint32_t ns, uint32_t ratio,
                                              uint32_t *Sbm, uint32_t bm_lo, Acc &acc) {
    const int lane = threadIdx.x & 31;
    uint32_t s_lo = 0, s_nw = 0;
    bool bm = false;
    if (Sbm && ns >= 32) {
        s_lo = (ld_any(&S[0]) >> 7) << 2;
        s_nw = (((ld_any(&S[ns - 1]) >> 5) + 1 - s_lo) + 3) & ~3u;
        bm = s_nw <= SB_CAP_WORDS && s_nw <= ns;
        if (bm && bm_lo != EH_PAD) {
            // level 1 left S's words [bm_lo, ...) in Sbm: S's own range starts inside it
            Sbm += s_lo - bm_lo;
        } else if (bm) {
            for (uint32_t w = lane; w < s_nw; w += 32) Sbm[w] = 0u;
            __syncwarp();
            for (uint32_t k = lane; k < ns; k += 32) {
                const uint32_t e = ld_any(&S[k]);
                atomicOr(&Sbm[(e >> 5) - s_lo], 1u << (e & 31));
            }
            __syncwarp();
        }
    }
    for (uint32_t i0 = 1; i0 < ns; i0 += 32) {
        const uint32_t il = i0 + lane;
        const SetDesc mine = il < ns ? ld_desc(&tv.desc[ld_any(&S[il])]) : empty_desc();
        const uint32_t cnt = min(32u, ns - i0);
        uint32_t coop = __ballot_sync(FULL, il < ns && mine.len > 0);
        if (bm) {
            // lane-per-z over S's bitmap
            bool mine_coop = false;
            if (il < ns && mine.len > 0) {
                uint32_t c = 0;
                if (mine.nwords) {
                    const uint32_t lo = max(s_lo, mine.lo_word), hi = min(s_lo + s_nw, mine.lo_word + mine.nwords);
                    const uint32_t *zw = tv.words + mine.woff - mine.lo_word;
                    for (uint32_t w = lo; w < hi; w += 4) {
                        const uint4 b = ldg4(zw + w);
                        const uint4 a = *reinterpret_cast<const uint4 *>(Sbm + (w - s_lo));
                        c += __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
                    }
                } else if (mine.len <= LANE_UINT_MAX) {
                    const uint32_t *zp = tv.nbr + mine.off;
                    const uint32_t base = s_lo * 32, nbits = s_nw * 32;
                    for (uint32_t p = 0; p < mine.len; p += 4) {
                        const uint4 e = ldg4(zp + p);
                        const uint32_t w4[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint32_t x = w4[q] - base;
                            if (x < nbits) c += (Sbm[x >> 5] >> (x & 31)) & 1u;
                        }
                    }
                } else {
                    mine_coop = true;
                }
                acc.t += c;
            }
            coop = __ballot_sync(FULL, mine_coop);
        }
        while (coop) {
            const uint32_t k = __ffs(coop) - 1;
            coop &= coop - 1;
            const SetDesc dz = bcast_desc(mine, k);
            pair_sorted<M_COUNT>(tv, S, i0 + k, dz, 0, ratio, acc, nullptr);
        }
        (void)cnt;
    }
    __syncwarp();
}

__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t r) {
    for (uint32_t k = 0; k < r; ++k) m &= m - 1;
    return m ? (uint32_t)(__ffs(m) - 1) : 0u;
}

template <int WARPS>
__device__ __forceinline__ bool k4_heavy(const TrieView &tv, uint32_t x, uint32_t ratio, uint32_t *sA, uint32_t *sS,
                                         uint32_t *sB, uint64_t *mbar, uint32_t &phase, uint32_t *s_next, Acc &acc,
                                         uint32_t *status, uint32_t *arena, uint64_t arena_per_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t gwarp = (uint64_t)blockIdx.x * WARPS + warp;
    const SetDesc dx = ld_desc(&tv.desc[x]);
    if (threadIdx.x == 0) *s_next = 2;
    StagedA st;
    if (!stage_set<WARPS>(tv, dx, sA, mbar, phase, st, status)) return false;
    for (;;) {
        const uint32_t j0 = next_j(s_next, K4_PAIR_BATCH);
        if (j0 >= st.len) break;
        const uint32_t jl = j0 + lane;
        SetDesc mine = empty_desc();
        if (lane < K4_PAIR_BATCH && jl < st.len) mine = ld_desc(&tv.desc[st.amode == 0 ? ldg1(&st.Ag[jl]) : ld_any(&st.A[jl])]);
        const uint32_t nbat = min(K4_PAIR_BATCH, st.len - j0);
        for (uint32_t i = 0; i < nbat; ++i) {
        const uint32_t j = j0 + i;
        const SetDesc dy = bcast_desc(mine, i);
        if (dy.len < 2) continue;
        const uint32_t bound = min(j, dy.len);
        uint32_t *S = bound <= S_CAP ? sS + warp * S_CAP : arena + gwarp * arena_per_warp;
        if (bound > S_CAP && (arena == nullptr || bound > arena_per_warp)) {
            if (lane == 0) atomicOr(status, DEV_ST_INVALID);
            continue;
        }
        uint32_t *Sbm = sB + warp * SB_CAP_WORDS;
        uint32_t bm_lo = EH_PAD;
        uint32_t ns = st.amode == 0 ? emit_bitmap(tv, sA, st.a_lo, st.a_nw, dy, S, Sbm, &bm_lo)
                                    : emit_sorted(tv, st.A, j, dy, ratio, S);
        clique_level2(tv, S, ns, ratio, Sbm, bm_lo, acc);
        __syncwarp();
        }
    }
    __syncthreads();
    return true;
}

// light vertex x: A and S held one element per lane
__device__ void k4_light(const TrieView &tv, uint32_t x, uint32_t ratio, Acc &acc) {
    const int lane = threadIdx.x & 31;
    const SetDesc dx = ld_desc(&tv.desc[x]);
    const uint32_t k = dx.len;
    const uint32_t a = lane < k ? ldg1(&tv.nbr[dx.off + lane]) : EH_PAD;
    const SetDesc mine = lane < k ? ld_desc(&tv.desc[a]) : empty_desc();
    for (uint32_t j = 2; j < k; ++j) {
        const SetDesc dy = bcast_desc(mine, j);
        if (dy.len < 2) continue;
        const uint32_t m = __ballot_sync(FULL, light_match(tv, a, j, dy, ratio));
        const uint32_t ns = __popc(m);
        if (ns < 2) continue;
        // S = the matching lanes' elements (and descriptors), compacted in order
        const uint32_t src = (uint32_t)lane < ns ? nth_set_bit(m, lane) : 0u;
        uint32_t sv = __shfl_sync(FULL, a, src);
        const SetDesc sd = bcast_desc(mine, src);
        if ((uint32_t)lane >= ns) sv = EH_PAD;
        // lane i (z = S[i]) with a bitset N+(z) probes S[0..i) itself, reading
        // S's elements from the lower lanes; the other z's run warp-wide
        const bool lane_bits = (uint32_t)lane >= 1 && (uint32_t)lane < ns && sd.len > 0 && sd.nwords;
        uint32_t c = 0;
        const uint32_t zbase = sd.lo_word * 32, znbits = sd.nwords * 32;
        for (uint32_t t2 = 0; t2 + 1 < ns; ++t2) {
            const uint32_t e = __shfl_sync(FULL, sv, t2);
            const uint32_t x = e - zbase;
            if (lane_bits && t2 < (uint32_t)lane && x < znbits)
                c += (ldg1(&tv.words[sd.woff + (x >> 5)]) >> (x & 31)) & 1u;
        }
        acc.t += c;
        uint32_t coop = __ballot_sync(FULL, (uint32_t)lane >= 1 && (uint32_t)lane < ns && sd.len > 0 && !sd.nwords);
        while (coop) {
            const uint32_t i = __ffs(coop) - 1;
            coop &= coop - 1;
            const SetDesc dz = bcast_desc(sd, i);
            if (light_match(tv, sv, i, dz, ratio)) acc.t += 1;
        }
    }
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_clique4(TrieView tv, const uint32_t *__restrict__ heavy, uint32_t n_heavy,
                                                        const uint32_t *__restrict__ light, uint32_t n_light,
                                                        uint32_t ratio, unsigned long long *counters,
                                                        unsigned long long *out, uint32_t *status, uint32_t *arena,
                                                        uint64_t arena_per_warp) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sA = smem;
    uint32_t *sS = smem + BM_CAP_WORDS;
    uint32_t *sB = sS + WARPS * S_CAP;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_item, s_next;
    const int tid = threadIdx.x, lane = tid & 31;
    Acc acc{0, 0};
    uint32_t phase = 0;
    if (tid == 0) {
        mbar_init(&mbar, 1);
        CHK_TRIE(tv, heavy, n_heavy, light, n_light, status);
        CHK_ADD(arena, arena_per_warp * gridDim.x * WARPS * 4);
    }
    __syncthreads();
    for (;;) {
        if (tid == 0) s_item = (uint32_t)min((unsigned long long)n_heavy, atomicAdd(&counters[0], 1ull));
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_heavy) break;
        if (!k4_heavy<WARPS>(tv, ldg1(&heavy[item]), ratio, sA, sS, sB, &mbar, phase, &s_next, acc, status, arena,
                             arena_per_warp))
            return;
    }
    const uint32_t chunk = light_chunk(n_light, WARPS);
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&counters[1], (unsigned long long)chunk);
        base = __shfl_sync(FULL, base, 0);
        if (base >= n_light) break;
        uint32_t end = (uint32_t)min((unsigned long long)n_light, base + chunk);
        for (uint32_t it = (uint32_t)base; it < end; ++it) k4_light(tv, ldg1(&light[it]), ratio, acc);
    }
    unsigned long long t = acc.t;
    for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(FULL, t, d);
    if (lane == 0 && t) atomicAdd(&out[0], t);
}

// ------------------------------------------------------------------- batch
//
// Many queries, each over its own induced sub-trie, in one persistent launch.
// The sub-tries of a batch are concatenated: sub-vertex s belongs to query
// q = sub_q[s] and is local vertex s - qbase[q] of it; sets hold local ids.
// Items (sub-vertices) of every query are mixed, heaviest first; each item
// runs the triangle, lollipop or 4-clique routine of its query's pattern and
// adds into out[2q] (triangles or 4-cliques) and out[2q+1] (lollipop sum).

__device__ __forceinline__ TrieView view_of(const BatchView &b, uint32_t q) {
    TrieView v;
    const uint32_t base = ldg1(&b.qbase[q]);
    v.desc = b.desc + base;
    v.nbr = b.nbr;
    v.words = b.words;
    v.deg = b.deg + base;
    v.n = ldg1(&b.qbase[q + 1]) - base;
    return v;
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_batch(BatchView bv, const uint32_t *__restrict__ heavy, uint32_t n_heavy,
                                                      const uint32_t *__restrict__ light, uint32_t n_light,
                                                      uint32_t ratio, unsigned long long *counters,
                                                      unsigned long long *out, uint32_t *status, uint32_t *arena,
                                                      uint64_t arena_per_warp) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sA = smem;
    uint32_t *sS = smem + BM_CAP_WORDS;
    uint32_t *sB = sS + WARPS * S_CAP;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_item, s_next;
    __shared__ unsigned long long red_t[WARPS], red_s[WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t phase = 0;
    if (tid == 0) {
        mbar_init(&mbar, 1);
        CHK_BATCH(bv, heavy, n_heavy, light, n_light, status);
        CHK_ADD(arena, arena_per_warp * gridDim.x * WARPS * 4);
    }
    __syncthreads();
    for (;;) {
        if (tid == 0) s_item = (uint32_t)min((unsigned long long)n_heavy, atomicAdd(&counters[0], 1ull));
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_heavy) break;
        const uint32_t sidx = ldg1(&heavy[item]);
        const uint32_t q = ldg1(&bv.sub_q[sidx]);
        const TrieView tv = view_of(bv, q);
        const uint32_t u = sidx - ldg1(&bv.qbase[q]);
        const uint32_t pat = ldg1(&bv.qpat[q]);
        Acc acc{0, 0};
        bool ok;
        if (pat == EH_CLIQUE4)
            ok = k4_heavy<WARPS>(tv, u, ratio, sA, sS, sB, &mbar, phase, &s_next, acc, status, arena, arena_per_warp);
        else if (pat == EH_TRIANGLE)
            ok = tri_heavy<M_COUNT, WARPS>(tv, u, ratio, sA, &mbar, phase, &s_next, acc, status, nullptr);
        else
            ok = tri_heavy<M_LOLLI, WARPS>(tv, u, ratio, sA, &mbar, phase, &s_next, acc, status, nullptr);
        if (!ok) return;
        unsigned long long t = acc.t, s = acc.s;
        for (int d = 16; d > 0; d >>= 1) {
            t += __shfl_xor_sync(FULL, t, d);
            s += __shfl_xor_sync(FULL, s, d);
        }
        if (lane == 0) { red_t[warp] = t; red_s[warp] = s; }
        __syncthreads();
        if (tid == 0) {
            unsigned long long T = 0, S = 0;
            for (int w = 0; w < WARPS; ++w) { T += red_t[w]; S += red_s[w]; }
            if (T) atomicAdd(&out[2 * q], T);
            if (S) atomicAdd(&out[2 * q + 1], S);
        }
    }
    const uint32_t chunk = light_chunk(n_light, WARPS);
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&counters[1], (unsigned long long)chunk);
        base = __shfl_sync(FULL, base, 0);
        if (base >= n_light) break;
        uint32_t end = (uint32_t)min((unsigned long long)n_light, base + chunk);
        for (uint32_t it = (uint32_t)base; it < end; ++it) {
            const uint32_t sidx = ldg1(&light[it]);
            const uint32_t q = ldg1(&bv.sub_q[sidx]);
            const TrieView tv = view_of(bv, q);
            const uint32_t u = sidx - ldg1(&bv.qbase[q]);
            const uint32_t pat = ldg1(&bv.qpat[q]);
            Acc acc{0, 0};
            if (pat == EH_CLIQUE4) k4_light(tv, u, ratio, acc);
            else if (pat == EH_TRIANGLE) light_vertex<M_COUNT>(tv, u, ratio, acc, nullptr);
            else light_vertex<M_LOLLI>(tv, u, ratio, acc, nullptr);
            unsigned long long t = acc.t, s = acc.s;
            for (int d = 16; d > 0; d >>= 1) {
                t += __shfl_xor_sync(FULL, t, d);
                s += __shfl_xor_sync(FULL, s, d);
            }
            if (lane == 0) {
                if (t) atomicAdd(&out[2 * q], t);
                if (s) atomicAdd(&out[2 * q + 1], s);
            }
        }
    }
}

template <int WARPS>
eh_status launch_batch(const BatchView &bv, const uint32_t *heavy, uint32_t n_heavy, const uint32_t *light,
                       uint32_t n_light, const eh_exec_opts &xo, cudaStream_t s, unsigned long long *d_out,
                       unsigned long long *d_counters, uint32_t *d_status, uint32_t *arena, uint64_t per_warp,
                       uint32_t *grid_warps) {
    auto kern = k_batch<WARPS>;
    const int smem = (BM_CAP_WORDS + WARPS * (S_CAP + SB_CAP_WORDS)) * 4;
    EH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    EH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem));
    if (per_sm < 1) per_sm = 1;
    unsigned grid = (unsigned)(eh_num_sms() * per_sm);
    if (grid_warps) { *grid_warps = grid * WARPS; return EH_OK; }
    EH_CUDA_TRY(cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned long long), s));
    kern<<<grid, WARPS * 32, smem, s>>>(bv, heavy, n_heavy, light, n_light, xo.gallop_ratio, d_counters, d_out,
                                        d_status, arena, per_warp);
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}

template <int WARPS>
eh_status launch_k4(eh_trie *t, const WorkPlan &plan, TrieView tv, const eh_exec_opts &xo, cudaStream_t s,
                    unsigned long long *d_acc, unsigned long long *d_counters, uint32_t *d_status) {
    auto kern = k_clique4<WARPS>;
    const int smem = (BM_CAP_WORDS + WARPS * (S_CAP + SB_CAP_WORDS)) * 4;
    EH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    EH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem));
    if (per_sm < 1) per_sm = 1;
    unsigned grid = (unsigned)(eh_num_sms() * per_sm);
    uint64_t per_warp = ((uint64_t)t->max_out + 3) & ~3ull;
    uint32_t *arena = nullptr;
    if (t->max_out > S_CAP) {
        std::lock_guard<std::mutex> g(t->mu);
        uint64_t need = per_warp * grid * WARPS;
        if (t->arena_words < need) {
            cudaFree(t->d_arena);
            t->d_arena = nullptr;
            t->arena_words = 0;
            if (eh_alloc_should_fail()) { eh_set_error("arena allocation failed (injected)"); return EH_ENOMEM; }
            EH_CUDA_TRY(cudaMalloc((void **)&t->d_arena, need * 4));
            t->arena_words = need;
        }
        arena = t->d_arena;
    }
    EH_CUDA_TRY(cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned long long), s));
    kern<<<grid, WARPS * 32, smem, s>>>(tv, plan.d_heavy, plan.n_heavy, plan.d_light, plan.n_light, xo.gallop_ratio,
                                        d_counters, d_acc, d_status, arena, per_warp);
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}

template <int MODE, int WARPS, int PW = 1>
eh_status launch_tri(const WorkPlan &plan, TrieView tv, const eh_exec_opts &xo, cudaStream_t s,
                     unsigned long long *d_acc, unsigned long long *d_counters, uint32_t *d_status,
                     unsigned long long *d_vt) {
    auto kern = k_triangle<MODE, WARPS, PW>;
    const int smem = tri_smem_bytes(MODE);
    static bool attr_set = false;
    if (!attr_set) {
        EH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_set = true;
    }
    int per_sm = 0;
    EH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem));
    if (per_sm < 1) per_sm = 1;
    unsigned grid = (unsigned)(eh_num_sms() * per_sm);
    EH_CUDA_TRY(cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned long long), s));
    kern<<<grid, WARPS * 32, smem, s>>>(tv, plan.d_heavy, plan.n_heavy, plan.d_light, plan.n_light,
                                        xo.gallop_ratio, d_counters, d_acc, d_status, d_vt);
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}

template <int MODE, int PW>
eh_status launch_tri_pw(const WorkPlan &plan, TrieView tv, const eh_exec_opts &xo, cudaStream_t s,
                        unsigned long long *d_acc, unsigned long long *d_counters, uint32_t *d_status,
                        unsigned long long *d_vt) {
    switch (xo.cta_warps) {
        case 4: return launch_tri<MODE, 4, PW>(plan, tv, xo, s, d_acc, d_counters, d_status, d_vt);
        case 16: return launch_tri<MODE, 16, PW>(plan, tv, xo, s, d_acc, d_counters, d_status, d_vt);
        default: return launch_tri<MODE, 8, PW>(plan, tv, xo, s, d_acc, d_counters, d_status, d_vt);
    }
}

// warps per intersection (xo.pair_warps 1, 2 or 4) for the count and the
// lollipop; the per-vertex modes take one warp per pair
template <int MODE>
eh_status launch_tri_w(const WorkPlan &plan, TrieView tv, const eh_exec_opts &xo, cudaStream_t s,
                       unsigned long long *d_acc, unsigned long long *d_counters, uint32_t *d_status,
                       unsigned long long *d_vt) {
    if (MODE == M_COUNT || MODE == M_LOLLI) {
        if (xo.pair_warps == 2) return launch_tri_pw<MODE, 2>(plan, tv, xo, s, d_acc, d_counters, d_status, d_vt);
        if (xo.pair_warps == 4) return launch_tri_pw<MODE, 4>(plan, tv, xo, s, d_acc, d_counters, d_status, d_vt);
    }
    return launch_tri_pw<MODE, 1>(plan, tv, xo, s, d_acc, d_counters, d_status, d_vt);
}

}  // namespace

eh_status eh_launch_triangle(const eh_trie *t, const WorkPlan &plan, TrieView tv, int mode, const eh_exec_opts &xo,
                             cudaStream_t s, unsigned long long *d_acc, unsigned long long *d_counters,
                             uint32_t *d_status, unsigned long long *d_vt, const uint32_t *d_qid) {
    (void)t;
    (void)d_qid;
    switch (mode) {
        case M_COUNT: return launch_tri_w<M_COUNT>(plan, tv, xo, s, d_acc, d_counters, d_status, d_vt);
        case M_LOLLI: return launch_tri_w<M_LOLLI>(plan, tv, xo, s, d_acc, d_counters, d_status, d_vt);
        case M_VERTEX: return launch_tri_w<M_VERTEX>(plan, tv, xo, s, d_acc, d_counters, d_status, d_vt);
        case M_APEX: return launch_tri_w<M_APEX>(plan, tv, xo, s, d_acc, d_counters, d_status, d_vt);
    }
    eh_set_error("unknown triangle mode %d", mode);
    return EH_EINVAL;
}

eh_status eh_launch_clique4(const eh_trie *t, const WorkPlan &plan, TrieView tv, const eh_exec_opts &xo,
                            cudaStream_t s, unsigned long long *d_acc, unsigned long long *d_counters,
                            uint32_t *d_status, uint32_t *d_arena, uint64_t arena_words_per_warp) {
    (void)d_arena;
    (void)arena_words_per_warp;
    eh_trie *tt = const_cast<eh_trie *>(t);
    switch (xo.cta_warps) {
        case 4: return launch_k4<4>(tt, plan, tv, xo, s, d_acc, d_counters, d_status);
        case 16: return launch_k4<16>(tt, plan, tv, xo, s, d_acc, d_counters, d_status);
        default: return launch_k4<8>(tt, plan, tv, xo, s, d_acc, d_counters, d_status);
    }
}

eh_status eh_launch_batch(const BatchView &bv, const uint32_t *heavy, uint32_t n_heavy, const uint32_t *light,
                          uint32_t n_light, const eh_exec_opts &xo, cudaStream_t s, unsigned long long *d_out,
                          unsigned long long *d_counters, uint32_t *d_status, uint32_t *arena,
                          uint64_t arena_words_per_warp, uint32_t *grid_warps) {
    switch (xo.cta_warps) {
        case 4: return launch_batch<4>(bv, heavy, n_heavy, light, n_light, xo, s, d_out, d_counters, d_status, arena,
                                       arena_words_per_warp, grid_warps);
        case 16: return launch_batch<16>(bv, heavy, n_heavy, light, n_light, xo, s, d_out, d_counters, d_status,
                                         arena, arena_words_per_warp, grid_warps);
        default: return launch_batch<8>(bv, heavy, n_heavy, light, n_light, xo, s, d_out, d_counters, d_status,
                                        arena, arena_words_per_warp, grid_warps);
    }
}

// ------------------------------------------ whole-graph count without allocation
//
// eh_count_noalloc runs the same count kernels as eh_count, but keeps their
// scratch (the work-distribution counters, the accumulators, the status word
// and the 4-clique spill arena) in the file-scope array below instead of
// memory it allocates.  The array is a fixed 32 MiB that every device using
// this library holds until the process exits.

namespace {

constexpr uint64_t NOALLOC_WORDS = 8ull << 20;   // 32 MiB of 32-bit words
constexpr uint64_t NOALLOC_HEAD = 64;            // 32-bit words before the arena
// in the head: the SC_* accumulators and counters (unsigned long long words
// 0 .. SC_WORDS-1), the result, the status word
constexpr uint64_t NOALLOC_RESULT = SC_WORDS;            // unsigned long long word
constexpr uint64_t NOALLOC_STATUS = 2 * (SC_WORDS + 1);  // 32-bit word
static_assert(NOALLOC_STATUS < NOALLOC_HEAD, "scratch head too small");
static __device__ __align__(256) uint32_t g_noalloc_scratch[NOALLOC_WORDS];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[256] = {};

// Device address of the array on the current device, looked up once per
// device (the name is only a host-side stand-in for it).  The lookup loads
// this file's module, which commits the array's memory.  The kernels the call
// launches are then run once on empty work lists (no item is read), so that
// whatever their first launch sets up is in place before the first call.
eh_status noalloc_scratch(uint32_t **out, cudaStream_t s) {
    int dev = 0;
    EH_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) { eh_set_error("eh_count_noalloc: device ordinal %d out of range", dev); return EH_EINVAL; }
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            eh_set_error("eh_count_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return EH_ECUDA;
        }
        uint32_t *scr = (uint32_t *)p;
        unsigned long long *sc = (unsigned long long *)scr;
        const int smem4 = (BM_CAP_WORDS + 8 * (S_CAP + SB_CAP_WORDS)) * 4;
        EH_CUDA_TRY(cudaFuncSetAttribute(k_clique4<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem4));
        TrieView none{};
        EH_CUDA_TRY(cudaMemsetAsync(scr, 0, NOALLOC_HEAD * 4, s));
        k_triangle<M_COUNT, 8><<<1, 8 * 32, BM_CAP_WORDS * 4, s>>>(none, nullptr, 0, nullptr, 0, 32, sc + SC_CNT,
                                                                    sc + SC_T, scr + NOALLOC_STATUS, nullptr);
        k_triangle<M_LOLLI, 8><<<1, 8 * 32, BM_CAP_WORDS * 4, s>>>(none, nullptr, 0, nullptr, 0, 32, sc + SC_CNT,
                                                                    sc + SC_T, scr + NOALLOC_STATUS, nullptr);
        k_clique4<8><<<1, 8 * 32, smem4, s>>>(none, nullptr, 0, nullptr, 0, 32, sc + SC_CNT2, sc + SC_K4,
                                              scr + NOALLOC_STATUS, nullptr, 0);
        EH_CUDA_TRY(cudaGetLastError());
        EH_TRY(eh_launch_finalize(sc, EH_TRIANGLE, sc + NOALLOC_RESULT, scr + NOALLOC_STATUS, s));
        EH_CUDA_TRY(cudaStreamSynchronize(s));
        g_noalloc_addr[dev] = p;
    }
    *out = (uint32_t *)g_noalloc_addr[dev];
    return EH_OK;
}

}  // namespace

eh_status eh_noalloc_setup(cudaStream_t s) {
    uint32_t *p = nullptr;
    return noalloc_scratch(&p, s);
}

extern "C" eh_status eh_count_noalloc(const eh_trie *trie, eh_pattern pattern, void *stream, uint64_t *out_count) {
    if (!trie || !out_count) { eh_set_error("eh_count_noalloc: NULL argument"); return EH_EINVAL; }
    if (pattern < EH_TRIANGLE || pattern > EH_LOLLIPOP_DISTINCT) {
        eh_set_error("eh_count_noalloc: pattern %d not supported (triangle, 4-clique and the lollipops only)",
                     (int)pattern);
        return EH_EINVAL;
    }
    eh_trie *t = const_cast<eh_trie *>(trie);
    const eh_exec_opts xo = eh_exec_defaults(nullptr);
    const WorkPlan *plan = nullptr;
    {
        std::lock_guard<std::mutex> g(t->mu);
        auto it = t->plans.find(xo.light_max);
        if (it != t->plans.end()) plan = &it->second;
    }
    if (!plan) {
        eh_set_error("eh_count_noalloc: the trie has no work plan yet; call eh_count_info_get (or any "
                     "whole-graph count) on it once first");
        return EH_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *scr = nullptr;
    EH_TRY(noalloc_scratch(&scr, s));
    unsigned long long *sc = (unsigned long long *)scr;               // SC_* layout
    unsigned long long *res = sc + NOALLOC_RESULT;
    uint32_t *status = scr + NOALLOC_STATUS;
    uint32_t *arena = scr + NOALLOC_HEAD;
    const uint64_t arena_cap = NOALLOC_WORDS - NOALLOC_HEAD;
    const TrieView tv = t->view();

    auto kern4 = k_clique4<8>;
    const int smem4 = (BM_CAP_WORDS + 8 * (S_CAP + SB_CAP_WORDS)) * 4;
    unsigned grid4 = 0;
    uint64_t per_warp = 0;
    if (pattern == EH_CLIQUE4) {
        EH_CUDA_TRY(cudaFuncSetAttribute(kern4, cudaFuncAttributeMaxDynamicSharedMemorySize, smem4));
        int per_sm = 0;
        EH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern4, 8 * 32, smem4));
        grid4 = (unsigned)(eh_num_sms() * (per_sm < 1 ? 1 : per_sm));
        if (t->max_out > S_CAP) {
            per_warp = ((uint64_t)t->max_out + 3) & ~3ull;
            const uint64_t need = per_warp * grid4 * 8;
            if (need > arena_cap) {
                eh_set_error("eh_count_noalloc: the 4-clique spill arena needs %llu bytes (max out-degree %u, %u "
                             "warps) but the static scratch holds %llu; use eh_count",
                             (unsigned long long)(need * 4), t->max_out, grid4 * 8,
                             (unsigned long long)(arena_cap * 4));
                return EH_EINVAL;
            }
        }
    }
    // the array keeps the previous call's contents: clear what must start at zero
    EH_CUDA_TRY(cudaMemsetAsync(scr, 0, NOALLOC_HEAD * 4, s));
    if (pattern == EH_CLIQUE4) {
        kern4<<<grid4, 8 * 32, smem4, s>>>(tv, plan->d_heavy, plan->n_heavy, plan->d_light, plan->n_light,
                                           xo.gallop_ratio, sc + SC_CNT2, sc + SC_K4, status,
                                           per_warp ? arena : nullptr, per_warp);
    } else {
        auto kern = pattern == EH_TRIANGLE ? k_triangle<M_COUNT, 8> : k_triangle<M_LOLLI, 8>;
        const int smem = BM_CAP_WORDS * 4;
        int per_sm = 0;
        EH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 8 * 32, smem));
        unsigned grid = (unsigned)(eh_num_sms() * (per_sm < 1 ? 1 : per_sm));
        kern<<<grid, 8 * 32, smem, s>>>(tv, plan->d_heavy, plan->n_heavy, plan->d_light, plan->n_light,
                                        xo.gallop_ratio, sc + SC_CNT, sc + SC_T, status, nullptr);
    }
    EH_CUDA_TRY(cudaGetLastError());
    EH_TRY(eh_launch_finalize(sc, (int)pattern, res, status, s));
    unsigned long long r = 0;
    uint32_t st = 0;
    EH_CUDA_TRY(cudaMemcpyAsync(&r, res, 8, cudaMemcpyDeviceToHost, s));
    EH_CUDA_TRY(cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s));
    EH_CUDA_TRY(cudaStreamSynchronize(s));
    if (st & DEV_ST_TIMEOUT) { eh_set_error("eh_count_noalloc: a bounded device wait timed out"); return EH_ETIMEOUT; }
    if (st & DEV_ST_OVERFLOW) { eh_set_error("eh_count_noalloc: count exceeds uint64"); return EH_EOVERFLOW; }
    if (st) { eh_set_error("eh_count_noalloc: device status 0x%x", st); return EH_ECUDA; }
    *out_count = r;
    return EH_OK;
}

// ------------------------------------------------------ bounded-wait self-test
//
// A kernel that waits, with the count kernels' bounded wait, on an mbarrier
// phase that nothing completes: the wait gives up after `limit_us`, the
// kernel records DEV_ST_TIMEOUT and returns, and the context stays usable.

namespace {
__global__ void k_selftest_wait(uint32_t *status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) mbar_init(&mbar, 1);
    __syncthreads();
    const bool ok = mbar_wait(&mbar, 0, limit_ns);   // no arrival, no copy: never completes
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, DEV_ST_TIMEOUT);
}
}  // namespace

extern "C" eh_status eh_selftest_wait_timeout(uint32_t limit_us, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *d = nullptr;
    EH_TRY(dev_alloc(&d, 1, s));
    uint32_t h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, 4, s);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 64, 0, s>>>(d, (uint64_t)limit_us * 1000ull);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, s);
    dev_free(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { eh_set_error("self-test: %s", cudaGetErrorString(e)); return EH_ECUDA; }
    if (h & DEV_ST_TIMEOUT) { eh_set_error("self-test: the bounded wait gave up as designed"); return EH_ETIMEOUT; }
    return EH_OK;
}
