// batch.cu -- counts over vertex-induced subgraphs (placeholder until the
// sub-trie builder lands).
#include "eh_internal.cuh"

eh_status eh_count_subset(const eh_trie *trie, eh_pattern pattern, const uint32_t *subset, uint32_t subset_len,
                          const eh_exec_opts *xopts, void *stream, uint64_t *out_count) {
    (void)trie; (void)pattern; (void)subset; (void)subset_len; (void)xopts; (void)stream; (void)out_count;
    eh_set_error("induced-subgraph counts are not available in this build");
    return EH_EINVAL;
}

extern "C" eh_status eh_count_batch_ex(const eh_trie *trie, const eh_query *queries, uint32_t n_queries,
                                       const uint32_t *subset_pool, uint64_t pool_len, const eh_exec_opts *xopts,
                                       uint32_t mode, void *stream, uint64_t *out_counts, eh_status *out_status) {
    (void)trie; (void)queries; (void)subset_pool; (void)pool_len; (void)xopts; (void)mode; (void)stream;
    (void)out_counts;
    for (uint32_t i = 0; i < n_queries; ++i) out_status[i] = EH_EINVAL;
    eh_set_error("batched counts are not available in this build");
    return EH_EINVAL;
}

extern "C" eh_status eh_count_batch(const eh_trie *trie, const eh_query *queries, uint32_t n_queries,
                                    const uint32_t *subset_pool, uint64_t pool_len, void *stream, uint64_t *out_counts,
                                    eh_status *out_status) {
    return eh_count_batch_ex(trie, queries, n_queries, subset_pool, pool_len, nullptr, 0, stream, out_counts,
                             out_status);
}
