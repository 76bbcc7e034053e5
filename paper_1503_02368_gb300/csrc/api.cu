// api.cu -- the whole-graph entry points of eh.h (counts, range counts, work-plan
// facts, per-vertex counts, selections) and shared runtime helpers.
#include "eh_internal.cuh"

#include <algorithm>
#include <atomic>
#include <vector>

namespace {
thread_local char g_err[1024] = "";

enum { M_COUNT = 0, M_LOLLI = 1, M_VERTEX = 2 };

// result of a pattern from the accumulators: T (triangles), S (sum over
// triangles of the three degrees), K (4-cliques)
__global__ void k_finalize(const unsigned long long *acc, int pattern, unsigned long long *out, uint32_t *status) {
    unsigned long long T = acc[SC_T], S = acc[SC_S], r = 0;
    switch (pattern) {
        case EH_TRIANGLE: r = T; break;
        case EH_CLIQUE4: r = acc[SC_K4]; break;
        case EH_LOLLIPOP:
            if (S >> 63) atomicOr(status, DEV_ST_OVERFLOW);
            r = 2ull * S;
            break;
        case EH_LOLLIPOP_DISTINCT: r = S - 6ull * T; break;
        case EH_BARBELL: r = acc[SC_K4]; break;
    }
    *out = r;
}

// Barbell root node: B += 4 t(x) sum_{x' in N(x)} t(x'), one warp per vertex
// over the symmetric trie (t = per-vertex triangle counts, new ids)
__global__ void k_barbell(const unsigned long long *__restrict__ vt, const uint64_t *__restrict__ soff,
                          const uint32_t *__restrict__ snbr, const uint32_t *__restrict__ deg, uint32_t n,
                          unsigned long long *acc, uint32_t *status) {
    const uint32_t x = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (x >= n) return;
    const unsigned long long tx = vt[x];
    if (tx == 0) return;
    unsigned long long sum = 0;
    const uint64_t b = soff[x];
    for (uint32_t i = lane; i < deg[x]; i += 32) sum += vt[snbr[b + i]];
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (lane == 0 && sum) {
        const unsigned long long hi = __umul64hi(4ull * tx, sum);
        const unsigned long long term = 4ull * tx * sum;
        const unsigned long long old = atomicAdd(acc, term);
        if (hi || (tx >> 61) || old + term < old) atomicOr(status, DEV_ST_OVERFLOW);
    }
}

// sum of t(x) over the symmetric set N(node) (one block)
__global__ void k_sel_sum(const unsigned long long *__restrict__ vt, const uint64_t *__restrict__ soff,
                          const uint32_t *__restrict__ snbr, const uint32_t *__restrict__ deg, uint32_t node,
                          unsigned long long *out) {
    unsigned long long sum = 0;
    for (uint32_t i = threadIdx.x; i < deg[node]; i += blockDim.x) sum += vt[snbr[soff[node] + i]];
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(out, sum);
}

__global__ void k_vt_to_old(const unsigned long long *vt, const uint32_t *new2old, uint32_t n, unsigned long long *out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[new2old[i]] = vt[i];
}

eh_status check_status(eh_trie *t, cudaStream_t s) {
    uint32_t st = 0;
    EH_CUDA_TRY(cudaMemcpyAsync(&st, t->d_status, 4, cudaMemcpyDeviceToHost, s));
    EH_CUDA_TRY(cudaStreamSynchronize(s));
    if (st) EH_CUDA_TRY(cudaMemsetAsync(t->d_status, 0, 4, s));
    if (st & DEV_ST_TIMEOUT) { eh_set_error("a bounded device wait timed out"); return EH_ETIMEOUT; }
    if (st & DEV_ST_OVERFLOW) { eh_set_error("count exceeds uint64"); return EH_EOVERFLOW; }
    if (st & DEV_ST_INVALID) { eh_set_error("invalid id on the device"); return EH_EINVAL; }
    if (st & DEV_ST_RANGE) { eh_set_error("listing: the count and write passes disagree"); return EH_ECUDA; }
    if (st & DEV_ST_BOUNDS) {
        eh_set_error("a device load fell outside its array (checked build; the load was not made)");
        return EH_ECUDA;
    }
    return EH_OK;
}

// enqueue one whole-graph count; result left in d_out (device)
eh_status enqueue_count(eh_trie *t, eh_pattern pattern, const eh_exec_opts &xo, cudaStream_t s,
                        unsigned long long *d_out) {
    NvtxRange nv("eh_count");
    WorkPlan *plan = nullptr;
    EH_TRY(eh_plan_get(t, xo.light_max, s, &plan));
    unsigned long long *sc = t->d_scratch;
    EH_CUDA_TRY(cudaMemsetAsync(sc, 0, SC_WORDS * sizeof(unsigned long long), s));
    if (pattern == EH_BARBELL) {
        // node 1 and 2 of the GHD: per-vertex triangle counts; root: the U(x,x') pass
        unsigned long long *vt = nullptr;
        EH_TRY(dev_alloc(&vt, t->n, s));
        eh_status st = EH_OK;
        if (cudaMemsetAsync(vt, 0, (uint64_t)(t->n ? t->n : 1) * 8, s) != cudaSuccess) st = EH_ECUDA;
        if (st == EH_OK)
            st = eh_launch_triangle(t, *plan, t->view(), M_VERTEX, xo, s, sc + SC_T, sc + SC_CNT, t->d_status, vt,
                                    nullptr);
        if (st == EH_OK && t->n)
            k_barbell<<<(t->n + 7) / 8, 256, 0, s>>>(vt, t->d_soff, t->d_snbr, t->d_deg, t->n, sc + SC_K4,
                                                       t->d_status);
        dev_free(vt, s);
        EH_TRY(st);
    } else if (pattern == EH_CLIQUE4) {
        EH_TRY(eh_launch_clique4(t, *plan, t->view(), xo, s, sc + SC_K4, sc + SC_CNT2, t->d_status, nullptr, 0));
    } else if (pattern == EH_TRIANGLE && t->d_boff) {
        // composite (block-level) layout
        EH_TRY(eh_launch_tri_blocks(t, *plan, s, sc + SC_T, reinterpret_cast<unsigned int *>(sc + SC_CNT)));
    } else {
        int mode = pattern == EH_TRIANGLE ? M_COUNT : M_LOLLI;
        EH_TRY(eh_launch_triangle(t, *plan, t->view(), mode, xo, s, sc + SC_T, sc + SC_CNT, t->d_status, nullptr,
                                  nullptr));
    }
    k_finalize<<<1, 1, 0, s>>>(sc, (int)pattern, d_out, t->d_status);
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}

bool valid_pattern(int p) { return p >= EH_TRIANGLE && p <= EH_BARBELL; }

}  // namespace

eh_status eh_launch_finalize(const unsigned long long *acc, int pattern, unsigned long long *out, uint32_t *status,
                             cudaStream_t s) {
    k_finalize<<<1, 1, 0, s>>>(acc, pattern, out, status);
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}

eh_status eh_enqueue_whole(eh_trie *t, eh_pattern pattern, const eh_exec_opts &xo, cudaStream_t s,
                           unsigned long long *d_out) {
    return enqueue_count(t, pattern, xo, s, d_out);
}

eh_status eh_check_status(eh_trie *t, cudaStream_t s) { return check_status(t, s); }

namespace {
std::atomic<long long> g_fail_countdown{-1};
}

bool eh_alloc_should_fail() {
    long long c = g_fail_countdown.load(std::memory_order_relaxed);
    if (c < 0) return false;
    return g_fail_countdown.fetch_sub(1) == 0;
}

extern "C" void eh_test_fail_alloc_after(long long n) { g_fail_countdown.store(n < 0 ? -1 : n); }

void eh_set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

extern "C" const char *eh_last_error(void) { return g_err; }

int eh_num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            cudaGetLastError();
            sms = 1;
        }
    }
    return sms;
}

eh_exec_opts eh_exec_defaults(const eh_exec_opts *x) {
    eh_exec_opts o;
    o.gallop_ratio = 32;
    o.light_max = 32;
    o.cta_warps = 8;
    o.flags = 0;
    o.pair_warps = 1;
    if (x) {
        if (x->gallop_ratio) o.gallop_ratio = x->gallop_ratio;
        if (x->light_max) o.light_max = std::min<uint32_t>(x->light_max, 32u);
        if (x->cta_warps == 4 || x->cta_warps == 8 || x->cta_warps == 16) o.cta_warps = x->cta_warps;
        o.flags = x->flags;
        if (x->pair_warps == 2 || x->pair_warps == 4) o.pair_warps = x->pair_warps;
    }
    return o;
}

eh_status eh_count_subset(const eh_trie *trie, eh_pattern pattern, const uint32_t *subset, uint32_t subset_len,
                          const eh_exec_opts *xopts, void *stream, uint64_t *out_count);

extern "C" eh_status eh_count_ex(const eh_trie *trie, eh_pattern pattern, const uint32_t *subset,
                                 uint32_t subset_len, const eh_exec_opts *xopts, void *stream, uint64_t *out_count) {
    if (!trie || !out_count) { eh_set_error("eh_count: NULL argument"); return EH_EINVAL; }
    if (!valid_pattern(pattern)) { eh_set_error("eh_count: unknown pattern %d", (int)pattern); return EH_EINVAL; }
    if (subset && subset_len) {
        if (pattern == EH_BARBELL) { eh_set_error("eh_count: barbell is whole-graph only"); return EH_EINVAL; }
        return eh_count_subset(trie, pattern, subset, subset_len, xopts, stream, out_count);
    }
    eh_trie *t = const_cast<eh_trie *>(trie);
    cudaStream_t s = (cudaStream_t)stream;
    eh_exec_opts xo = eh_exec_defaults(xopts);
    std::lock_guard<std::mutex> g(t->call_mu);
    unsigned long long *d_out = t->d_scratch + 15;
    EH_TRY(enqueue_count(t, pattern, xo, s, d_out));
    unsigned long long r = 0;
    EH_CUDA_TRY(cudaMemcpyAsync(&r, d_out, 8, cudaMemcpyDeviceToHost, s));
    EH_TRY(check_status(t, s));
    *out_count = r;
    return EH_OK;
}

extern "C" eh_status eh_count(const eh_trie *trie, eh_pattern pattern, const uint32_t *subset, uint32_t subset_len,
                              void *stream, uint64_t *out_count) {
    return eh_count_ex(trie, pattern, subset, subset_len, nullptr, stream, out_count);
}

extern "C" eh_status eh_count_async(const eh_trie *trie, eh_pattern pattern, const eh_exec_opts *xopts,
                                    void *stream, uint64_t *d_out_count) {
    if (!trie || !d_out_count) { eh_set_error("eh_count_async: NULL argument"); return EH_EINVAL; }
    if (!valid_pattern(pattern)) { eh_set_error("eh_count_async: unknown pattern %d", (int)pattern); return EH_EINVAL; }
    eh_trie *t = const_cast<eh_trie *>(trie);
    eh_exec_opts xo = eh_exec_defaults(xopts);
    return enqueue_count(t, pattern, xo, (cudaStream_t)stream, (unsigned long long *)d_out_count);
}

extern "C" eh_status eh_count_status(const eh_trie *trie, void *stream) {
    if (!trie) { eh_set_error("eh_count_status: NULL trie"); return EH_EINVAL; }
    return check_status(const_cast<eh_trie *>(trie), (cudaStream_t)stream);
}

// ------------------------------------------------------------- range counts
//
// One part of a whole-graph count: the plan's heavy and light lists are each
// cut into `nparts` contiguous, cost-balanced ranges (eh_split_range over the
// lists' cost prefixes) and the count kernel runs over this part's ranges
// only.  The parts' results sum to the whole count.

namespace {

bool range_pattern(int p) { return p == EH_TRIANGLE || p == EH_CLIQUE4 || p == EH_LOLLIPOP || p == EH_LOLLIPOP_DISTINCT; }

eh_status enqueue_range(eh_trie *t, eh_pattern pattern, uint32_t part, uint32_t nparts, const eh_exec_opts &xo,
                        cudaStream_t s, unsigned long long *d_out) {
    NvtxRange nv("eh_count_range");
    WorkPlan *plan = nullptr;
    EH_TRY(eh_plan_get(t, xo.light_max, s, &plan));
    EH_TRY(eh_plan_cost_prefix(t, plan, s));
    uint64_t hlo, hhi, llo, lhi;
    eh_split_range(plan->h_heavy_pre.data(), plan->n_heavy, part, nparts, &hlo, &hhi);
    eh_split_range(plan->h_light_pre.data(), plan->n_light, part, nparts, &llo, &lhi);
    WorkPlan sub;   // the part's ranges of the lists (no ownership)
    sub.light_max = plan->light_max;
    sub.d_heavy = plan->d_heavy + hlo;
    sub.n_heavy = (uint32_t)(hhi - hlo);
    sub.d_light = plan->d_light + llo;
    sub.n_light = (uint32_t)(lhi - llo);
    unsigned long long *sc = t->d_scratch;
    EH_CUDA_TRY(cudaMemsetAsync(sc, 0, SC_WORDS * sizeof(unsigned long long), s));
    if (pattern == EH_CLIQUE4) {
        EH_TRY(eh_launch_clique4(t, sub, t->view(), xo, s, sc + SC_K4, sc + SC_CNT2, t->d_status, nullptr, 0));
    } else {
        // set-level kernel also on a block-layout trie (its uint arrays and bitsets are kept)
        const int mode = pattern == EH_TRIANGLE ? M_COUNT : M_LOLLI;
        EH_TRY(eh_launch_triangle(t, sub, t->view(), mode, xo, s, sc + SC_T, sc + SC_CNT, t->d_status, nullptr,
                                  nullptr));
    }
    k_finalize<<<1, 1, 0, s>>>(sc, (int)pattern, d_out, t->d_status);
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}

eh_status check_range_args(const eh_trie *trie, int pattern, uint32_t part, uint32_t nparts, const char *who) {
    if (!trie) { eh_set_error("%s: NULL trie", who); return EH_EINVAL; }
    if (!range_pattern(pattern)) {
        eh_set_error("%s: pattern %d cannot be split (triangle, 4-clique and the lollipops only)", who, pattern);
        return EH_EINVAL;
    }
    if (nparts == 0 || part >= nparts) { eh_set_error("%s: part %u of %u parts", who, part, nparts); return EH_EINVAL; }
    return EH_OK;
}

}  // namespace

extern "C" eh_status eh_count_range(const eh_trie *trie, eh_pattern pattern, uint32_t part, uint32_t nparts,
                                    const eh_exec_opts *xopts, void *stream, uint64_t *out_count) {
    EH_TRY(check_range_args(trie, pattern, part, nparts, "eh_count_range"));
    if (!out_count) { eh_set_error("eh_count_range: NULL out_count"); return EH_EINVAL; }
    eh_trie *t = const_cast<eh_trie *>(trie);
    cudaStream_t s = (cudaStream_t)stream;
    const eh_exec_opts xo = eh_exec_defaults(xopts);
    std::lock_guard<std::mutex> g(t->call_mu);
    unsigned long long *d_out = t->d_scratch + 15;
    EH_TRY(enqueue_range(t, pattern, part, nparts, xo, s, d_out));
    unsigned long long r = 0;
    EH_CUDA_TRY(cudaMemcpyAsync(&r, d_out, 8, cudaMemcpyDeviceToHost, s));
    EH_TRY(check_status(t, s));
    *out_count = r;
    return EH_OK;
}

extern "C" eh_status eh_count_range_async(const eh_trie *trie, eh_pattern pattern, uint32_t part, uint32_t nparts,
                                          const eh_exec_opts *xopts, void *stream, uint64_t *d_out_count) {
    EH_TRY(check_range_args(trie, pattern, part, nparts, "eh_count_range_async"));
    if (!d_out_count) { eh_set_error("eh_count_range_async: NULL d_out_count"); return EH_EINVAL; }
    const eh_exec_opts xo = eh_exec_defaults(xopts);
    return enqueue_range(const_cast<eh_trie *>(trie), pattern, part, nparts, xo, (cudaStream_t)stream,
                         (unsigned long long *)d_out_count);
}

extern "C" eh_status eh_range_bounds(const uint64_t *cost, uint64_t n, uint32_t part, uint32_t nparts, uint64_t *lo,
                                     uint64_t *hi) {
    if ((n && !cost) || !lo || !hi || nparts == 0 || part >= nparts) {
        eh_set_error("eh_range_bounds: bad argument");
        return EH_EINVAL;
    }
    std::vector<uint64_t> pre((size_t)n + 1, 0);
    for (uint64_t i = 0; i < n; ++i) {
        if (pre[i] + cost[i] < pre[i]) { eh_set_error("eh_range_bounds: total cost exceeds uint64"); return EH_EOVERFLOW; }
        pre[i + 1] = pre[i] + cost[i];
    }
    eh_split_range(pre.data(), n, part, nparts, lo, hi);
    return EH_OK;
}

extern "C" eh_status eh_count_info_get(const eh_trie *trie, eh_pattern pattern, const eh_exec_opts *xopts,
                                       void *stream, eh_count_info *out) {
    if (!trie || !out) { eh_set_error("eh_count_info_get: NULL argument"); return EH_EINVAL; }
    if (!valid_pattern(pattern)) { eh_set_error("eh_count_info_get: unknown pattern"); return EH_EINVAL; }
    eh_trie *t = const_cast<eh_trie *>(trie);
    eh_exec_opts xo = eh_exec_defaults(xopts);
    WorkPlan *plan = nullptr;
    EH_TRY(eh_plan_get(t, xo.light_max, (cudaStream_t)stream, &plan));
    double alg = 0, stored = 0;
    if (pattern == EH_CLIQUE4) {
        EH_TRY(eh_plan_alg_bytes(t, plan, (cudaStream_t)stream, ALG_K4, &alg));
    } else {
        EH_TRY(eh_plan_alg_bytes(t, plan, (cudaStream_t)stream, ALG_TRI, &alg));
        EH_TRY(eh_plan_alg_bytes(t, plan, (cudaStream_t)stream, ALG_TRI_STORED, &stored));
    }
    memset(out, 0, sizeof(*out));
    out->alg_bytes = alg;
    out->alg_bytes_stored = stored;
    out->n_heavy = plan->n_heavy;
    out->n_light = plan->n_light;
    out->kernel_launches = 2;   // the count kernel and the finalize kernel
    return EH_OK;
}

extern "C" eh_status eh_vertex_triangles(const eh_trie *trie, void *stream, uint64_t *out_t) {
    if (!trie || !out_t) { eh_set_error("eh_vertex_triangles: NULL argument"); return EH_EINVAL; }
    eh_trie *t = const_cast<eh_trie *>(trie);
    cudaStream_t s = (cudaStream_t)stream;
    eh_exec_opts xo = eh_exec_defaults(nullptr);
    std::lock_guard<std::mutex> g(t->call_mu);
    WorkPlan *plan = nullptr;
    EH_TRY(eh_plan_get(t, xo.light_max, s, &plan));
    unsigned long long *vt = nullptr, *vo = nullptr;
    EH_TRY(dev_alloc(&vt, t->n, s));
    eh_status st = dev_alloc(&vo, t->n, s);
    if (st == EH_OK) {
        cudaMemsetAsync(vt, 0, (uint64_t)t->n * 8, s);
        cudaMemsetAsync(t->d_scratch, 0, SC_WORDS * sizeof(unsigned long long), s);
        st = eh_launch_triangle(t, *plan, t->view(), M_VERTEX, xo, s, t->d_scratch + SC_T, t->d_scratch + SC_CNT,
                                t->d_status, vt, nullptr);
    }
    if (st == EH_OK && t->n) {
        k_vt_to_old<<<(t->n + 255) / 256, 256, 0, s>>>(vt, t->d_new2old, t->n, vo);
        cudaError_t e = cudaMemcpyAsync(out_t, vo, (uint64_t)t->n * 8, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) { eh_set_error("eh_vertex_triangles: %s", cudaGetErrorString(e)); st = EH_ECUDA; }
    }
    if (st == EH_OK) st = check_status(t, s);
    dev_free(vt, s);
    dev_free(vo, s);
    cudaStreamSynchronize(s);
    return st;
}

extern "C" eh_status eh_count_selected(const eh_trie *trie, eh_sel_pattern pattern, uint32_t node,
                                       const eh_exec_opts *xopts, void *stream, uint64_t *out_count) {
    if (!trie || !out_count) { eh_set_error("eh_count_selected: NULL argument"); return EH_EINVAL; }
    if (pattern != EH_SEL_CLIQUE4 && pattern != EH_SEL_BARBELL) {
        eh_set_error("eh_count_selected: unknown selection pattern %d", (int)pattern);
        return EH_EINVAL;
    }
    if (node >= trie->n) { eh_set_error("eh_count_selected: node %u >= n_vertices %u", node, trie->n); return EH_EINVAL; }
    eh_trie *t = const_cast<eh_trie *>(trie);
    cudaStream_t s = (cudaStream_t)stream;
    const eh_exec_opts xo = eh_exec_defaults(xopts);
    std::lock_guard<std::mutex> g(t->call_mu);
    uint32_t node_new = 0;
    EH_CUDA_TRY(cudaMemcpyAsync(&node_new, t->d_old2new + node, 4, cudaMemcpyDeviceToHost, s));
    EH_CUDA_TRY(cudaStreamSynchronize(s));
    if (pattern == EH_SEL_CLIQUE4) {
        uint64_t k = 0;
        EH_TRY(eh_sk4_total(t, node_new, xo, s, &k));
        if (k > ~0ull / 6) { eh_set_error("SK4 count exceeds uint64"); return EH_EOVERFLOW; }
        *out_count = 6 * k;
        return EH_OK;
    }
    // SB3,1: per-vertex triangle counts (the triangle nodes of the GHD), then the
    // selection node: (sum over x in N(node) of 2 t(x))^2
    WorkPlan *plan = nullptr;
    EH_TRY(eh_plan_get(t, xo.light_max, s, &plan));
    unsigned long long *vt = nullptr;
    EH_TRY(dev_alloc(&vt, (uint64_t)t->n + 1, s));
    eh_status st = EH_OK;
    if (cudaMemsetAsync(vt, 0, ((uint64_t)t->n + 1) * 8, s) != cudaSuccess ||
        cudaMemsetAsync(t->d_scratch, 0, SC_WORDS * sizeof(unsigned long long), s) != cudaSuccess)
        st = EH_ECUDA;
    if (st == EH_OK)
        st = eh_launch_triangle(t, *plan, t->view(), M_VERTEX, xo, s, t->d_scratch + SC_T, t->d_scratch + SC_CNT,
                                t->d_status, vt, nullptr);
    unsigned long long sum = 0;
    if (st == EH_OK) {
        k_sel_sum<<<1, 1024, 0, s>>>(vt, t->d_soff, t->d_snbr, t->d_deg, node_new, vt + t->n);
        if (cudaMemcpyAsync(&sum, vt + t->n, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) st = EH_ECUDA;
    }
    if (st == EH_OK) st = check_status(t, s);
    dev_free(vt, s);
    cudaStreamSynchronize(s);
    EH_TRY(st);
    const unsigned __int128 half = (unsigned __int128)2 * sum, b = half * half;
    if ((b >> 64) != 0) { eh_set_error("SB3,1 count exceeds uint64"); return EH_EOVERFLOW; }
    *out_count = (uint64_t)b;
    return EH_OK;
}
