// Serving loop: the graph stays resident; a scheduler thread admits queries while
// a slot is free and their weight tables fit in the scratch budget, runs every
// admitted query together in epochs (one persistent sampler launch over all of
// their next tiles, replayed from the captured epoch graph), retires each query at
// its first converged Alg. 1 checkpoint and admits waiting ones between epochs.
// A query's result depends only on its own trials and checkpoint schedule, so it is
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
    agis_result res{};
    std::vector<uint64_t> pinned;   // table keys this query holds
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
    uint64_t completed = 0, epochs = 0;
    int peak_slots = 0;
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

void scheduler(agis_server *s)
{
    agis_graph *g = s->g;
    cudaSetDevice(g->ctx->device);
    for (;;) {
        std::vector<Served *> admitted;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->waiting.empty() || !s->active.empty(); });
            if (s->stop) break;
            std::lock_guard<std::recursive_mutex> gl(g->mu);
            // admission by slot and by scratch memory (weight tables)
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
            admitted = s->active;
        }
        if (admitted.empty()) continue;
        // one epoch over every admitted query; each gets its next tiles, capped so
        // an epoch stays short enough for new arrivals to join soon
        std::vector<QueryRun *> runs;
        std::vector<uint64_t> ntiles;
        std::vector<Served *> owners;
        size_t total = 0;
        int per_sm = 1;
        sampler_occupancy(&per_sm);
        const uint64_t cap = std::max<uint64_t>(64, (uint64_t)g->ctx->sm_count * (uint64_t)std::max(1, per_sm) * 2 /
                                                        std::max<size_t>(1, admitted.size()));
        for (Served *q : admitted) {
            uint64_t n = next_tiles(q->run);
            const uint64_t tpc = q->run.tiles_per_chunk;
            if (n > cap) n = std::max<uint64_t>(tpc, cap / tpc * tpc);
            n = std::min<uint64_t>(n, q->run.max_tiles - q->run.done_tiles);
            if (n == 0) { q->run.finished = true; continue; }
            runs.push_back(&q->run);
            ntiles.push_back(n);
            owners.push_back(q);
            total += n;
        }
        int rc = AGIS_OK;
        std::vector<std::vector<uint64_t>> outs(runs.size());
        if (!runs.empty()) {
            std::lock_guard<std::recursive_mutex> gl(g->mu);
            rc = run_epoch_graph(g, runs, ntiles, total);
            if (rc == AGIS_OK) {
                size_t k = 0;
                for (size_t i = 0; i < runs.size(); ++i) {
                    outs[i].assign(g->lb.h_out + 4 * k, g->lb.h_out + 4 * (k + ntiles[i]));
                    k += ntiles[i];
                }
            }
        }
        std::lock_guard<std::mutex> lk(s->mu);
        std::lock_guard<std::recursive_mutex> gl(g->mu);
        s->epochs++;
        for (size_t i = 0; i < runs.size(); ++i) {
            if (rc == AGIS_OK) {
                runs[i]->launches++;
                absorb(*runs[i], outs[i].data(), ntiles[i]);
            }
        }
        std::vector<Served *> still;
        for (Served *q : s->active) {
            if (rc != AGIS_OK) finish(s, q, rc);
            else if (q->run.finished) finish(s, q, AGIS_OK);
            else still.push_back(q);
        }
        s->active.swap(still);
    }
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

extern "C" int agis_server_poll(agis_server *s, uint64_t ticket, agis_result *out, double *latency_s)
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
    s->by_ticket.erase(it);
    delete q;
    return status;
}

extern "C" int agis_server_stats(agis_server *s, uint64_t *completed, uint64_t *epochs, int32_t *peak_slots)
{
    if (!s) return AGIS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (epochs) *epochs = s->epochs;
    if (peak_slots) *peak_slots = s->peak_slots;
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
    delete s;
    graph_release(g);
    return AGIS_OK;
}
