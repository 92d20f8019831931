// Serving loop: the graph stays resident; a scheduler thread admits queries while
// a slot is free and their weight tables fit in the scratch budget, runs every
// admitted query together in epochs (one persistent sampler launch over all of
// their next tiles, replayed from a captured epoch graph), retires each query at
// its first converged Alg. 1 checkpoint and admits waiting ones as slots and memory
// free up (continuous batching).  Two epochs are kept in flight on the context's
// stream, each with its own launch buffers: while one runs, the next one is staged
// and enqueued from the sums absorbed so far (a query whose checkpoint is still in
// flight gets one more chunk), so the GPU does not wait for the host between
// epochs.  Tiles issued after a query's stopping checkpoint are discarded unread,
// so a query's result depends only on its own trials and checkpoint schedule: it is
// the same alone, batched or served.
#include <algorithm>
#include <cstring>
#include <new>

#include "agis_internal.h"

namespace {

struct Served {
    uint64_t ticket = 0;
    agis_pattern pat;
    agis_opts opts{};
    agis::QueryRun run;
    double t_submit = 0.0, t_done = 0.0;
    int status = AGIS_OK;
    bool done = false;
    bool released = false;          // polled while an epoch still held it: freed by the scheduler
    int refs = 0;                   // in-flight epochs that carry tiles of this query
    uint64_t admit_epoch = 0;       // index of the first epoch with tiles of this query
    uint64_t finish_epoch = 0;      // index of the epoch whose sums finished it
    bool started = false;
    agis_result res{};
    std::vector<uint64_t> pinned;   // table keys this query holds
};

struct Epoch {
    int slot = 0;
    uint64_t index = 0;
    std::vector<agis::QueryRun *> runs;
    std::vector<uint64_t> ntiles;
    std::vector<Served *> owners;
};

}  // namespace

struct agis_server {
    agis_graph *g = nullptr;
    size_t scratch_bytes = 0;
    int max_slots = 1;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Served *> waiting;
    std::vector<Served *> active;
    std::unordered_map<uint64_t, Served *> by_ticket;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    uint64_t completed = 0, epochs = 0, launched = 0;
    int peak_slots = 0;
    double gpu_busy_s = 0.0;        // summed epoch durations (events around each launch)
    double busy_span_s = 0.0;       // wall time with at least one epoch in flight
    // two launch-buffer sets (slot 1 borrows slot 0's candidate-list scratch: both run
    // in order on the context's stream) and their events
    agis::LaunchBuffers lb[2];
    cudaEvent_t ev_start[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
};

namespace agis {
namespace {

constexpr size_t kMaxWaiting = 65536;

// Device bytes a query would add: the parts of the tables its f_approx steps read that are
// not resident yet (q per vertex; a vertex prefix for step 1; a row prefix for
// single-backward steps while the graph's row-prefix budget allows one).
size_t extra_bytes(agis_graph *g, const agis_pattern &p, const agis_opts &o)
{
    uint8_t use[kMaxK];
    agis_pattern_decide(&p, o.mode, o.beta, use);
    std::map<uint64_t, std::pair<bool, bool>> need;   // cfg -> (vertex prefix, row prefix)
    // a row prefix of every row, or of the highest-degree rows within the budget
    const size_t rowp_bytes = rowp_full_fits(g) ? sizeof(uint64_t) * (size_t)g->nnz
                                                 : std::min<size_t>(g->rowp_budget, sizeof(uint64_t) * (size_t)g->nnz);
    for (int i = 0; i < p.k; ++i) {
        if (!step_uses_table(&p, i, &o, g->oriented, use)) continue;
        int32_t cfg[4];
        effective_cfg(&p, i, o.terms, g->oriented, cfg);
        auto &f = need[cfg_key(cfg)];
        f.first = f.first || i == 0;
        f.second = f.second || (i > 0 && (p.nback[i] == 1 || o.anchor));
    }
    size_t extra = 0;
    for (const auto &kv : need) {
        auto it = g->tables.find(kv.first);
        const bool have = it != g->tables.end();
        if (!have) extra += sizeof(uint64_t) * (size_t)g->nv;
        if (kv.second.first && !(have && it->second.pref)) extra += sizeof(uint64_t) * (size_t)g->nv;
        if (kv.second.second && !(have && it->second.rowp)) extra += rowp_bytes;
    }
    return extra;
}

size_t resident_bytes(agis_graph *g)
{
    size_t b = 0;
    for (const auto &kv : g->tables) b += kv.second.bytes;
    return b;
}

// Frees unpinned tables, least recently used first, until `need` more bytes fit.
void evict_for(agis_graph *g, size_t budget, size_t need)
{
    while (resident_bytes(g) + need > budget) {
        auto victim = g->tables.end();
        for (auto it = g->tables.begin(); it != g->tables.end(); ++it)
            if (it->second.pins == 0 && (victim == g->tables.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == g->tables.end()) return;
        cudaStreamSynchronize(g->ctx->stream);
        free_table(victim->second);
        g->tables.erase(victim);
    }
}

void finish(agis_server *s, Served *q, int status)
{
    q->status = status;
    if (status == AGIS_OK) fill_result(q->run, &q->res);
    q->t_done = now_s();
    q->res.t_sample_s = q->t_done - q->t_submit;
    for (uint64_t key : q->pinned) {
        auto it = s->g->tables.find(key);
        if (it != s->g->tables.end() && it->second.pins > 0) it->second.pins--;
    }
    q->pinned.clear();
    q->done = true;
    s->completed++;
}

// Admission (under s->mu and g->mu): queries enter while a slot is free and their
// tables fit the scratch budget (unpinned tables are evicted least recently used
// first); a query that cannot fit even alone fails with NOMEM.
void admit(agis_server *s)
{
    agis_graph *g = s->g;
    while ((int)s->active.size() < s->max_slots && !s->waiting.empty()) {
        Served *q = s->waiting.front();
        const size_t need = extra_bytes(g, q->pat, q->opts);
        if (resident_bytes(g) + need > s->scratch_bytes) evict_for(g, s->scratch_bytes, need);
        if (resident_bytes(g) + need > s->scratch_bytes) {
            if (s->active.empty()) {          // can never fit: fail it
                s->waiting.pop_front();
                finish(s, q, AGIS_ERR_NOMEM);
                continue;
            }
            break;                            // wait for running queries to free tables
        }
        s->waiting.pop_front();
        int rc = init_run(g, &q->pat, &q->opts, q->run);
        if (rc != AGIS_OK) {
            finish(s, q, rc);
            continue;
        }
        uint8_t use[kMaxK];
        agis_pattern_decide(&q->pat, q->opts.mode, q->opts.beta, use);
        for (int i = 0; i < q->pat.k; ++i) {
            if (!step_uses_table(&q->pat, i, &q->opts, g->oriented, use)) continue;
            int32_t cfg[4];
            effective_cfg(&q->pat, i, q->opts.terms, g->oriented, cfg);
            const uint64_t key = cfg_key(cfg);
            if (std::find(q->pinned.begin(), q->pinned.end(), key) != q->pinned.end()) continue;
            g->tables[key].pins++;
            q->pinned.push_back(key);
        }
        s->active.push_back(q);
    }
    s->peak_slots = std::max(s->peak_slots, (int)s->active.size());
}

// Plans and enqueues the next epoch (under s->mu and g->mu): every admitted query
// gets its next tiles, capped so that an epoch stays short enough for new
// arrivals to join soon.  Returns false when no query has tiles to issue.
bool launch_epoch(agis_server *s, std::deque<Epoch> &inflight, int &rc)
{
    agis_graph *g = s->g;
    int per_sm = g->ctx->blocks_per_sm;
    if (per_sm <= 0) sampler_occupancy(&per_sm);
    const int grid = g->ctx->sm_count * std::max(1, per_sm);
    const uint64_t cap = std::max<uint64_t>(64, (uint64_t)grid * 2 / std::max<size_t>(1, s->active.size()));
    Epoch e;
    size_t total = 0;
    for (Served *q : s->active) {
        uint64_t n = ahead_tiles(q->run);
        const uint64_t tpc = q->run.tiles_per_chunk;
        if (n > cap) n = std::max<uint64_t>(tpc, cap / tpc * tpc);
        n = std::min<uint64_t>(n, q->run.max_tiles - q->run.issued_tiles);
        if (n == 0) continue;
        e.runs.push_back(&q->run);
        e.ntiles.push_back(n);
        e.owners.push_back(q);
        total += n;
    }
    if (e.runs.empty()) return false;
    e.slot = (int)(s->launched & 1);
    e.index = s->launched;
    rc = ensure_scratch(g, s->lb[0], 2 * grid);
    if (rc == AGIS_OK)
        rc = enqueue_epoch_graph(g, s->lb[e.slot], s->lb[0], e.runs, e.ntiles, total, s->ev_start[e.slot],
                                 s->ev_done[e.slot]);
    if (rc != AGIS_OK) return false;
    s->launched++;
    for (Served *q : e.owners) {
        q->refs++;
        if (!q->started) {
            q->started = true;
            q->admit_epoch = e.index;
        }
    }
    inflight.push_back(std::move(e));
    return true;
}

void release_if_unused(agis_server *s, Served *q)
{
    if (q->released && q->refs == 0) {
        (void)s;
        delete q;
    }
}

// Waits for the oldest in-flight epoch, folds its tile sums into its queries and
// retires the finished ones (takes s->mu and g->mu after the wait).
void complete_epoch(agis_server *s, std::deque<Epoch> &inflight, double &span_t0)
{
    agis_graph *g = s->g;
    Epoch e = std::move(inflight.front());
    inflight.pop_front();
    const cudaError_t err = cudaEventSynchronize(s->ev_done[e.slot]);
    float ms = 0.0f;
    if (err == cudaSuccess) cudaEventElapsedTime(&ms, s->ev_start[e.slot], s->ev_done[e.slot]);
    std::lock_guard<std::mutex> lk(s->mu);
    std::lock_guard<std::recursive_mutex> gl(g->mu);
    s->epochs++;
    s->gpu_busy_s += ms / 1000.0;
    const uint64_t *out = s->lb[e.slot].h_out;
    size_t k = 0;
    for (size_t i = 0; i < e.runs.size(); ++i) {
        Served *q = e.owners[i];
        if (err == cudaSuccess && !q->done) {
            e.runs[i]->launches++;
            absorb(*e.runs[i], out + kTileWords * k, e.ntiles[i]);
        }
        k += e.ntiles[i];
    }
    std::vector<Served *> still;
    for (Served *q : s->active) {
        if (err != cudaSuccess || q->run.finished) {
            q->finish_epoch = e.index;
            finish(s, q, err != cudaSuccess ? AGIS_ERR_CUDA : AGIS_OK);
        } else {
            still.push_back(q);
        }
    }
    s->active.swap(still);
    for (Served *q : e.owners) {
        q->refs--;
        release_if_unused(s, q);
    }
    if (inflight.empty()) s->busy_span_s += now_s() - span_t0;
}

void scheduler(agis_server *s)
{
    agis_graph *g = s->g;
    cudaSetDevice(g->ctx->device);
    std::deque<Epoch> inflight;
    double span_t0 = 0.0;
    for (;;) {
        bool queued = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (inflight.empty())
                s->cv.wait(lk, [&] { return s->stop || !s->waiting.empty() || !s->active.empty(); });
            if (s->stop) break;
            std::lock_guard<std::recursive_mutex> gl(g->mu);
            admit(s);
            if (inflight.size() < 2) {
                int rc = AGIS_OK;
                const bool was_idle = inflight.empty();
                const double t_enqueue = now_s();
                queued = launch_epoch(s, inflight, rc);
                if (queued && was_idle) span_t0 = t_enqueue;
                if (rc != AGIS_OK) {
                    for (Served *q : s->active) finish(s, q, rc);
                    s->active.clear();
                }
            }
        }
        if (queued && inflight.size() < 2) continue;      // stage a second epoch behind it
        if (!inflight.empty()) complete_epoch(s, inflight, span_t0);
    }
    while (!inflight.empty()) complete_epoch(s, inflight, span_t0);
}

}  // namespace
}  // namespace agis

using namespace agis;

extern "C" int agis_server_create(agis_graph *g, size_t scratch_bytes, int max_slots, agis_server **out)
{
    if (!g || !out || max_slots < 1) return AGIS_ERR_ARG;
    if (!g->prepped) return AGIS_ERR_STATE;
    agis_server *s = new (std::nothrow) agis_server();
    if (!s) return AGIS_ERR_NOMEM;
    s->g = g;
    graph_retain(g);
    s->scratch_bytes = scratch_bytes;
    s->max_slots = max_slots;
    cudaSetDevice(g->ctx->device);
    for (int i = 0; i < 2; ++i) {
        if (cudaEventCreate(&s->ev_start[i]) != cudaSuccess || cudaEventCreate(&s->ev_done[i]) != cudaSuccess) {
            for (int j = 0; j < 2; ++j) {
                if (s->ev_start[j]) cudaEventDestroy(s->ev_start[j]);
                if (s->ev_done[j]) cudaEventDestroy(s->ev_done[j]);
            }
            graph_release(g);
            delete s;
            return AGIS_ERR_CUDA;
        }
    }
    try {
        s->worker = std::thread(scheduler, s);
    } catch (...) {
        graph_release(g);
        delete s;
        return AGIS_ERR_NOMEM;
    }
    *out = s;
    return AGIS_OK;
}

extern "C" int agis_server_submit(agis_server *s, const agis_pattern *p, const agis_opts *opts, uint64_t *ticket)
{
    if (!s || !p || !opts || !ticket) return AGIS_ERR_ARG;
    int rc = check_opts(opts);
    if (rc != AGIS_OK) return rc;
    Served *q = new (std::nothrow) Served();
    if (!q) return AGIS_ERR_NOMEM;
    q->pat = *p;
    q->opts = *opts;
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->waiting.size() >= kMaxWaiting) {
            delete q;
            return AGIS_ERR_BUSY;
        }
        q->ticket = s->next_ticket++;
        s->by_ticket[q->ticket] = q;
        s->waiting.push_back(q);
        *ticket = q->ticket;
    }
    s->cv.notify_one();
    return AGIS_OK;
}

extern "C" int agis_server_poll(agis_server *s, uint64_t ticket, agis_result *out, double *latency_s,
                                uint64_t *epochs)
{
    if (!s || !out) return AGIS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->by_ticket.find(ticket);
    if (it == s->by_ticket.end()) return AGIS_ERR_ARG;
    Served *q = it->second;
    if (!q->done) return AGIS_ERR_BUSY;
    const int status = q->status;
    *out = q->res;
    if (latency_s) *latency_s = q->t_done - q->t_submit;
    if (epochs) {
        epochs[0] = q->admit_epoch;
        epochs[1] = q->finish_epoch;
    }
    s->by_ticket.erase(it);
    // an epoch still in flight may carry tiles of it: the scheduler frees it then
    q->released = true;
    release_if_unused(s, q);
    return status;
}

extern "C" int agis_server_stats(agis_server *s, uint64_t *completed, uint64_t *epochs, int32_t *peak_slots,
                                 double *gpu_busy_s, double *busy_span_s)
{
    if (!s) return AGIS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (epochs) *epochs = s->epochs;
    if (peak_slots) *peak_slots = s->peak_slots;
    if (gpu_busy_s) *gpu_busy_s = s->gpu_busy_s;
    if (busy_span_s) *busy_span_s = s->busy_span_s;
    return AGIS_OK;
}

extern "C" int agis_server_destroy(agis_server *s)
{
    if (!s) return AGIS_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    {
        std::lock_guard<std::recursive_mutex> gl(s->g->mu);
        for (Served *q : s->active) {
            for (uint64_t key : q->pinned) {
                auto it = s->g->tables.find(key);
                if (it != s->g->tables.end() && it->second.pins > 0) it->second.pins--;
            }
        }
    }
    for (auto &kv : s->by_ticket) delete kv.second;
    agis_graph *g = s->g;
    {
        std::lock_guard<std::recursive_mutex> gl(g->mu);
        cudaSetDevice(g->ctx->device);
        cudaStreamSynchronize(g->ctx->stream);
        free_buffers(s->lb[1]);
        free_buffers(s->lb[0]);
        for (int i = 0; i < 2; ++i) {
            cudaEventDestroy(s->ev_start[i]);
            cudaEventDestroy(s->ev_done[i]);
        }
    }
    delete s;
    graph_release(g);
    return AGIS_OK;
}
