// serve.cpp -- the request loop over a resident trie (eh_server_*).
//
// submit() estimates a query's device footprint (membership bitmap and rank
// words over the id space, sort keys, the induced sub-trie bounded by the
// members' pruned degrees) and admits it only when the bytes admitted and not
// yet released stay within the budget (else EH_EBUSY: the caller retries).
// Admitted queries wait in a FIFO.  `max_inflight` worker threads, each with
// its own CUDA stream, repeatedly take up to `max_batch` queued queries and run
// them as one device batch (eh_count_batch_ex): queries arriving while other
// batches run are picked up by the next free worker, so batches overlap on the
// device and the queue drains continuously.  Each query's latency is measured
// from submit() to the moment its batch's results reach the host.
#include "eh_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket;
    uint32_t pattern;
    std::vector<uint32_t> subset;
    uint64_t bytes;
    Clock::time_point t_submit;
};

struct Res {
    uint64_t count = 0;
    eh_status status = EH_OK;
    double latency = 0;
};

}  // namespace

struct eh_server {
    const eh_trie *trie = nullptr;
    int device = 0;
    uint64_t budget = 0, in_use = 0, peak = 0;
    uint32_t max_batch = 1, max_inflight = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> pending;
    std::unordered_map<uint64_t, Res> done;
    std::unordered_map<uint64_t, bool> known;
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, completed = 0, rejected = 0, batches = 0, batched_queries = 0;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

uint64_t footprint(const eh_trie *t, const uint32_t *subset, uint32_t len) {
    const uint64_t W = (((uint64_t)t->n + 31) / 32 + 3) & ~3ull;
    uint64_t sets = 0;
    for (uint32_t i = 0; i < len; ++i) {
        uint32_t v = subset[i];
        if (v < t->h_out_by_old.size()) sets += std::min<uint64_t>(t->h_out_by_old[v], len);
    }
    return 8 * W + 96ull * len + 12 * sets + 65536;
}

void worker(eh_server *s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        st = nullptr;
    }
    for (;;) {
        std::vector<Req> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
            if (s->pending.empty()) break;   // stop requested and nothing left
            while (!s->pending.empty() && batch.size() < s->max_batch) {
                batch.push_back(std::move(s->pending.front()));
                s->pending.pop_front();
            }
        }
        const uint32_t k = (uint32_t)batch.size();
        std::vector<eh_query> qs(k);
        std::vector<uint32_t> pool;
        for (uint32_t i = 0; i < k; ++i) {
            qs[i].pattern = batch[i].pattern;
            qs[i].subset_len = (uint32_t)batch[i].subset.size();
            qs[i].subset_off = pool.size();
            pool.insert(pool.end(), batch[i].subset.begin(), batch[i].subset.end());
        }
        std::vector<uint64_t> counts(k, 0);
        std::vector<eh_status> sts(k, EH_OK);
        eh_count_batch_ex(s->trie, qs.data(), k, pool.data(), pool.size(), nullptr, 0, st, counts.data(), sts.data());
        const Clock::time_point now = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (uint32_t i = 0; i < k; ++i) {
                Res r;
                r.count = counts[i];
                r.status = sts[i];
                r.latency = std::chrono::duration<double>(now - batch[i].t_submit).count();
                s->done[batch[i].ticket] = r;
                s->in_use -= batch[i].bytes;
            }
            s->completed += k;
            s->batches += 1;
            s->batched_queries += k;
        }
        s->cv_done.notify_all();
    }
    if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" eh_status eh_server_create(const eh_trie *trie, uint64_t memory_budget_bytes, uint32_t max_batch,
                                      uint32_t max_inflight, eh_server **out) {
    if (!trie || !out) { eh_set_error("eh_server_create: NULL argument"); return EH_EINVAL; }
    *out = nullptr;
    EH_TRY(eh_host_out_degrees(const_cast<eh_trie *>(trie)));
    eh_server *s = new (std::nothrow) eh_server();
    if (!s) { eh_set_error("host allocation failed"); return EH_ENOMEM; }
    s->trie = trie;
    s->budget = memory_budget_bytes;
    s->max_batch = max_batch ? max_batch : 1;
    s->max_inflight = max_inflight ? std::min<uint32_t>(max_inflight, 64) : 1;
    cudaGetDevice(&s->device);
    for (uint32_t i = 0; i < s->max_inflight; ++i) s->workers.emplace_back(worker, s);
    *out = s;
    return EH_OK;
}

extern "C" eh_status eh_server_submit(eh_server *s, eh_pattern pattern, const uint32_t *subset, uint32_t subset_len,
                                      uint64_t *ticket) {
    if (!s || !ticket || (subset_len && !subset)) { eh_set_error("eh_server_submit: NULL argument"); return EH_EINVAL; }
    if (pattern < EH_TRIANGLE || pattern > EH_BARBELL || (pattern == EH_BARBELL && subset_len)) {
        eh_set_error("eh_server_submit: unknown pattern");
        return EH_EINVAL;
    }
    Req r;
    r.pattern = (uint32_t)pattern;
    r.subset.assign(subset, subset + subset_len);
    r.bytes = footprint(s->trie, subset, subset_len);
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) { eh_set_error("server is shutting down"); return EH_EINVAL; }
        if (s->in_use + r.bytes > s->budget) {
            ++s->rejected;
            eh_set_error("admission: %llu bytes in use + %llu needed > budget %llu",
                         (unsigned long long)s->in_use, (unsigned long long)r.bytes, (unsigned long long)s->budget);
            return EH_EBUSY;
        }
        s->in_use += r.bytes;
        s->peak = std::max(s->peak, s->in_use);
        r.ticket = s->next_ticket++;
        *ticket = r.ticket;
        s->known[r.ticket] = true;
        ++s->submitted;
        s->pending.push_back(std::move(r));
    }
    s->cv_work.notify_one();
    return EH_OK;
}

extern "C" eh_status eh_server_poll(eh_server *s, uint64_t ticket, int *done, uint64_t *count, eh_status *status) {
    if (!s || !done) { eh_set_error("eh_server_poll: NULL argument"); return EH_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->known.count(ticket)) { eh_set_error("unknown ticket"); return EH_EINVAL; }
    auto it = s->done.find(ticket);
    *done = it != s->done.end();
    if (*done) {
        if (count) *count = it->second.count;
        if (status) *status = it->second.status;
    }
    return EH_OK;
}

extern "C" eh_status eh_server_wait(eh_server *s, uint64_t ticket, uint32_t timeout_ms, uint64_t *count,
                                    eh_status *status) {
    if (!s) { eh_set_error("eh_server_wait: NULL argument"); return EH_EINVAL; }
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->known.count(ticket)) { eh_set_error("unknown ticket"); return EH_EINVAL; }
    auto ready = [&] { return s->done.count(ticket) > 0; };
    if (timeout_ms) {
        if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
            eh_set_error("eh_server_wait: timed out");
            return EH_ETIMEOUT;
        }
    } else {
        s->cv_done.wait(lk, ready);
    }
    const Res &r = s->done[ticket];
    if (count) *count = r.count;
    if (status) *status = r.status;
    return EH_OK;
}

extern "C" eh_status eh_server_latency(eh_server *s, uint64_t ticket, double *seconds) {
    if (!s || !seconds) { eh_set_error("eh_server_latency: NULL argument"); return EH_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) { eh_set_error("ticket not complete or unknown"); return EH_EINVAL; }
    *seconds = it->second.latency;
    return EH_OK;
}

extern "C" eh_status eh_server_stats_get(eh_server *s, eh_server_stats *o) {
    if (!s || !o) { eh_set_error("eh_server_stats_get: NULL argument"); return EH_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    o->submitted = s->submitted;
    o->completed = s->completed;
    o->rejected = s->rejected;
    o->batches = s->batches;
    o->bytes_in_use = s->in_use;
    o->peak_bytes = s->peak;
    o->mean_batch = s->batches ? (double)s->batched_queries / (double)s->batches : 0.0;
    return EH_OK;
}

extern "C" void eh_server_destroy(eh_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &th : s->workers) th.join();
    delete s;
}
