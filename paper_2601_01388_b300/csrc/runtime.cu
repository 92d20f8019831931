// Host runtime: contexts, query compilation into device descriptors, the adaptive
// Alg. 1 loop (plain per-query launches), the batched loop that replays one captured
// CUDA graph per epoch, per-trial dumps, and device-resident fixed-budget sampling.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include "agis_internal.h"

// Tiles per work item of agis_sample_device's implicit items (at most kMaxSpan).
#ifndef AGIS_SAMPLE_SPAN
#define AGIS_SAMPLE_SPAN 1
#endif
// Tail of an epoch, in grids' worth of tiles (see tail_tiles); 1 / 2 / 4 / 8 / 16 grids
// measured, eight kept.
#ifndef AGIS_TAIL_GRIDS
#define AGIS_TAIL_GRIDS 8
#endif

namespace agis {

std::atomic<uint64_t> g_launches{0};

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

namespace {

template <typename T>
int grow_device(T **p, size_t *cap, size_t need, uint64_t *generation)
{
    if (need <= *cap) return AGIS_OK;
    size_t n = std::max<size_t>(need, *cap * 2);
    n = std::max<size_t>(n, 64);
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    AGIS_CUDA_TRY(cudaMalloc(p, sizeof(T) * n));
    *cap = n;
    ++*generation;
    return AGIS_OK;
}

template <typename T>
int grow_pinned(T **p, size_t *cap, size_t need, uint64_t *generation)
{
    if (need <= *cap) return AGIS_OK;
    size_t n = std::max<size_t>(need, *cap * 2);
    n = std::max<size_t>(n, 64);
    cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    AGIS_CUDA_TRY(cudaMallocHost(p, sizeof(T) * n));
    *cap = n;
    ++*generation;
    return AGIS_OK;
}

}  // namespace

void free_buffers(LaunchBuffers &lb)
{
    if (lb.exec) cudaGraphExecDestroy(lb.exec);
    if (lb.graph) cudaGraphDestroy(lb.graph);
    if (lb.sexec) cudaGraphExecDestroy(lb.sexec);
    if (lb.sgraph) cudaGraphDestroy(lb.sgraph);
    cudaFree(lb.d_sx);
    cudaFree(lb.d_shit);
    cudaFree(lb.d_ssec);
    cudaFree(lb.d_queries);
    cudaFree(lb.d_items);
    cudaFree(lb.d_out);
    cudaFree(lb.d_counter);
    if (!lb.scratch_borrowed) cudaFree(lb.d_scratch);
    cudaFreeHost(lb.h_queries);
    cudaFreeHost(lb.h_items);
    cudaFreeHost(lb.h_out);
    cudaFreeHost(lb.h_counter);
    if (lb.ev_fork) cudaEventDestroy(lb.ev_fork);
    if (lb.ev_join) cudaEventDestroy(lb.ev_join);
    if (lb.aux) cudaStreamDestroy(lb.aux);
    lb = LaunchBuffers();
}

namespace {

// Alg. 1: mu, population sigma^2 (clamped at 0) and eps_hat from N trials.
void alg1(double n, double sx, double sx2, double z, double *mu, double *var, double *eps_hat)
{
    const double m = sx / n;
    double s2 = sx2 / n - m * m;
    if (s2 < 0.0) s2 = 0.0;
    *mu = m;
    *var = s2;
    *eps_hat = m > 0.0 ? z * std::sqrt(s2) / std::sqrt(n) / m : INFINITY;
}

}  // namespace

int check_opts(const agis_opts *o)
{
    if (!o) return AGIS_ERR_ARG;
    if (o->mode < 0 || o->mode > 2) return AGIS_ERR_ARG;
    // T[F1] stays in every version (Sec. 6.2 adds terms to it): without it a vertex of
    // degree 0 would reach the nsum/d factor of T[F2]
    if (o->terms < 0 || o->terms > 7 || (o->terms != 0 && !(o->terms & 1))) return AGIS_ERR_ARG;
    if ((o->anchor != 0 && o->anchor != 1) || o->reserved != 0) return AGIS_ERR_ARG;
    if (o->chunk_trials == 0 || o->chunk_trials % 1024 != 0) return AGIS_ERR_ARG;
    if (o->max_trials == 0) return AGIS_ERR_ARG;
    if (o->eps > 0.0 && !(o->delta > 0.0 && o->delta < 1.0)) return AGIS_ERR_ARG;
    return AGIS_OK;
}

int ensure_buffers(LaunchBuffers &lb, size_t n_queries, size_t n_items)
{
    int rc;
    if ((rc = grow_device(&lb.d_queries, &lb.cap_queries, n_queries, &lb.generation))) return rc;
    if ((rc = grow_device(&lb.d_items, &lb.cap_items, n_items, &lb.generation))) return rc;
    if ((rc = grow_device(&lb.d_out, &lb.cap_out, kTileWords * n_items, &lb.generation))) return rc;
    if (!lb.d_counter) {
        AGIS_CUDA_TRY(cudaMalloc(&lb.d_counter, 4 * sizeof(uint32_t)));
        AGIS_CUDA_TRY(cudaMallocHost(&lb.h_counter, 4 * sizeof(uint32_t)));
        ++lb.generation;
    }
    if ((rc = grow_pinned(&lb.h_queries, &lb.hcap_queries, n_queries, &lb.generation))) return rc;
    if ((rc = grow_pinned(&lb.h_items, &lb.hcap_items, n_items, &lb.generation))) return rc;
    if ((rc = grow_pinned(&lb.h_out, &lb.hcap_out, kTileWords * n_items, &lb.generation))) return rc;
    return AGIS_OK;
}

// The last tiles of an epoch -- AGIS_TAIL_GRIDS times as many as a full grid has
// CTAs, or all of a smaller epoch -- run on the scatter kernel, where every warp of
// the grid takes single trials.  The main kernel gives a CTA whole tiles, 32 trials
// back to back on each warp, so an epoch of few tiles leaves most of the GPU idle,
// and in a larger one the CTAs that run out of tiles wait up to a tile's time for
// the last ones.  Launched beside the main kernel at a lower priority, the scatter
// kernel's CTAs take the SM slots that the main kernel's CTAs free as they run out,
// and its single trials level the end of the epoch.  Measured on the benchmark
// graph (all of an epoch in scatter mode): a 4-clique query to +-1% (20,480
// trials) 26.3 -> 5.9 ms, a 5-clique (45,056) 56 -> 12.5 ms.
size_t tail_capacity(int grid)
{
    return (size_t)(std::max(1.0, (double)AGIS_TAIL_GRIDS) * (double)std::max(grid, 0));
}

size_t tail_tiles(size_t tiles, int grid)
{
    const size_t full = (size_t)std::max(grid, 0);
    if (tiles <= full) return tiles;
    return std::min(tiles, (size_t)(AGIS_TAIL_GRIDS * (double)full));
}

// Per-trial output buffers of scatter epochs for `tiles` tiles.
int ensure_scatter(LaunchBuffers &lb, size_t tiles)
{
    const size_t trials = tiles * (size_t)kTile;
    if (trials <= lb.cap_scatter) return AGIS_OK;
    const size_t n = std::max<size_t>(trials, lb.cap_scatter * 2);
    cudaFree(lb.d_sx);
    cudaFree(lb.d_shit);
    cudaFree(lb.d_ssec);
    lb.d_sx = nullptr;
    lb.d_shit = nullptr;
    lb.d_ssec = nullptr;
    lb.cap_scatter = 0;
    ++lb.generation;
    AGIS_CUDA_TRY(cudaMalloc(&lb.d_sx, sizeof(double) * n));
    AGIS_CUDA_TRY(cudaMalloc(&lb.d_shit, n));
    AGIS_CUDA_TRY(cudaMalloc(&lb.d_ssec, 3 * sizeof(uint64_t) * n));
    lb.cap_scatter = n;
    return AGIS_OK;
}

// Persistent grid: resident CTAs on every SM (the autotuned count if set), never
// more than there are items.
int grid_for(agis_graph *g, size_t n_items)
{
    agis_ctx *c = g->ctx;
    int per_sm = c->blocks_per_sm;
    if (per_sm <= 0) {
        int occ = 1;
        sampler_occupancy(&occ);
        per_sm = std::max(1, occ);
    }
    size_t grid = (size_t)c->sm_count * (size_t)per_sm;
    grid = std::min(grid, std::max<size_t>(n_items, 1));
    return (int)grid;
}

// Bytes of one warp's candidate lists: two lists of cap ids and cap running weights.
size_t scratch_stride(uint32_t cap)
{
    const size_t b = (size_t)cap * 2 * (sizeof(int32_t) + sizeof(uint64_t));
    return (b + 255) / 256 * 256;
}

// Per-warp candidate-list scratch for a launch of `grid` CTAs: lists as long as
// the largest row, at most 65536 entries and within an eighth of device memory
// (a step whose survivors overflow takes the sampler's list-free path).  The
// allocation is padded so that 16-byte list loads may read past a list's end.
int ensure_scratch(agis_graph *g, LaunchBuffers &lb, int grid)
{
    const uint64_t want = ((uint64_t)std::min<int64_t>(std::max<int64_t>(g->max_deg, 64), (int64_t)g->list_cap) + 63) / 64 * 64;
    if (lb.d_scratch && lb.scratch_grid >= grid && lb.scratch_cap <= want && lb.scratch_cap + 64 > want) return AGIS_OK;
    size_t free_b = 0, total_b = 0;
    AGIS_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    const size_t warps = (size_t)grid * kWarps;
    uint64_t cap = (uint64_t)std::min<int64_t>(std::max<int64_t>(g->max_deg, 64), (int64_t)g->list_cap);
    cap = (cap + 63) / 64 * 64;
    const size_t budget = total_b / 8;
    while (cap > 64 && scratch_stride((uint32_t)cap) * warps > budget) cap = (cap / 2 + 63) / 64 * 64;
    cudaFree(lb.d_scratch);
    lb.d_scratch = nullptr;
    lb.scratch_bytes = 0;
    AGIS_CUDA_TRY(cudaMalloc(&lb.d_scratch, scratch_stride((uint32_t)cap) * warps + 256));
    lb.scratch_bytes = scratch_stride((uint32_t)cap) * warps;
    lb.scratch_cap = (uint32_t)cap;
    lb.scratch_grid = grid;
    ++lb.generation;
    return AGIS_OK;
}

void effective_cfg(const agis_pattern *p, int i, int32_t terms, bool oriented, int32_t out[4])
{
    out[0] = oriented ? 0 : p->cfg[i][0];
    out[1] = (terms == 0 || (terms & 1)) ? p->cfg[i][1] : 0;
    out[2] = (terms == 0 || (terms & 2)) ? p->cfg[i][2] : 0;
    out[3] = (terms == 0 || (terms & 4)) ? p->cfg[i][3] : 0;
}

// With |F1| = |I_eff| = |F2| = 0 in the effective configuration, Eq.
// probability_function is binom(d - |B|, 0) = 1 for d >= |B| and an intended zero
// below.  Every candidate of a later step's S_tau is adjacent to the |B| distinct
// backward vertices, so d >= |B| (on an orientation |B| is 0): the quantised weight
// is one constant c on all of S_tau.  The draw r = floor(U * |S| c / 2^128) then
// picks position floor(r / c) = floor(U * |S| / 2^128), the position draw, and
// W / q = |S| exactly, so such a step runs as f_uniform with identical results and
// no weight reads.  Step 1 is excluded (f_uniform is edge-uniform there), and so is
// an anchor draw, whose proposal row may hold vertices of degree below |B|.
bool step_weights_flat(const agis_pattern *p, int i, const agis_opts *o, bool oriented)
{
    if (i == 0) return false;
    if (o->anchor && p->nback[i] >= 2) return false;
    int32_t cfg[4];
    effective_cfg(p, i, o->terms, oriented, cfg);
    return cfg[1] == 0 && cfg[2] == 0 && cfg[3] == 0;
}

bool step_uses_table(const agis_pattern *p, int i, const agis_opts *o, bool oriented, const uint8_t *use)
{
    return use[i] && !step_weights_flat(p, i, o, oriented);
}

int make_dev_query(agis_graph *g, const agis_pattern *p, const agis_opts *o, DevQuery *dq,
                   double *t_prep)
{
    if (!g->prepped) return AGIS_ERR_STATE;
    if (g->oriented)
        for (int i = 0; i < p->k; ++i)
            if (p->nback[i] != i) return AGIS_ERR_PATTERN;   // an orientation serves cliques only
    uint8_t use[kMaxK];
    int rc = agis_pattern_decide(p, o->mode, o->beta, use);
    if (rc != AGIS_OK) return rc;
    std::memset(dq, 0, sizeof(*dq));
    dq->k = p->k;
    dq->flags = o->anchor ? kFlagAnchor : 0;
    dq->seed = o->seed;
    const double t0 = now_s();
    bool built = false;
    for (int i = 0; i < p->k; ++i) {
        DevStep &s = dq->step[i];
        s.nb = p->nback[i];
        s.approx = step_uses_table(p, i, o, g->oriented, use);
        s.dapprox = use[i] ? 1 : 0;
        for (int j = 0; j < p->nback[i] && j < kMaxK; ++j) s.back[j] = (int8_t)p->back[i][j];
        if (i >= 2) {
            // back(i) == back(i-1) + {i-1}?
            unsigned mi = 0, mp = 0;
            for (int j = 0; j < p->nback[i]; ++j) mi |= 1u << p->back[i][j];
            for (int j = 0; j < p->nback[i - 1]; ++j) mp |= 1u << p->back[i - 1][j];
            s.inc = (int8_t)(mi == (mp | (1u << (i - 1))) ? 1 : 0);
        }
        if (!s.approx) continue;
        const size_t before = g->tables.size();
        WeightTable *t = nullptr;
        // a row-prefix table makes single-backward draws a search; when the full table
        // (8 B per CSR entry) is past the budget only the highest-degree rows get one
        // and the sampler scans the other anchor rows
        const bool rowp = i > 0 && (p->nback[i] == 1 || o->anchor);
        int32_t cfg[4];
        effective_cfg(p, i, o->terms, g->oriented, cfg);
        rc = build_weight_table(g, cfg, i == 0, rowp, &t);
        if (rc != AGIS_OK) return rc;
        built |= g->tables.size() != before;
        s.q = t->q;
        if (i == 0) {
            s.pref = t->pref;
            dq->W1 = t->total;
        } else if (rowp && t->rowp) {
            s.pref = t->rowp;
            s.rp_mode = t->rowp_partial ? 2 : 1;
        }
    }
    if (!use[0]) dq->W1 = (uint64_t)g->nnz;
    // a step draws from a candidate list when it has several backward vertices, or
    // one without a row prefix for every row; if none of those lists is weighted,
    // the sampler filters survivor ids only
    bool weighted_lists = false;
    for (int i = 1; i < p->k; ++i) {
        const DevStep &s = dq->step[i];
        if (s.approx && (s.nb >= 2 || s.rp_mode != 1)) weighted_lists = true;
    }
    if (!weighted_lists) dq->flags |= kFlagPlainLists;
    if (built) AGIS_CUDA_TRY(cudaStreamSynchronize(g->ctx->stream));
    if (t_prep) *t_prep += now_s() - t0;
    return AGIS_OK;
}

int init_run(agis_graph *g, const agis_pattern *p, const agis_opts *o, QueryRun &r)
{
    int rc = check_opts(o);
    if (rc != AGIS_OK) return rc;
    if (!p) return AGIS_ERR_ARG;
    r.p = p;
    r.o = *o;
    r.z = o->eps > 0.0 ? agis_z_of_delta(o->delta) : 0.0;
    r.max_tiles = (o->max_trials + kTile - 1) / kTile;
    r.tiles_per_chunk = o->chunk_trials / kTile;
    r.oriented = g->oriented;
    return make_dev_query(g, p, o, &r.dq, &r.t_prep);
}

// Tiles to run after the first `from` tiles of one query: the first epoch covers
// min_trials (whole chunks); later ones aim at the trial count Alg. 1's own formula
// predicts from the sums absorbed so far, N ~ (z sigma / (eps mu))^2, between one
// chunk and four times the work so far.  Tiles already issued but not absorbed
// count as work done; with some in flight (a server staging its next epoch) a query
// gets more only when the prediction exceeds them, since tiles past its stopping
// checkpoint would be computed and discarded.
static uint64_t tiles_after(const QueryRun &r, uint64_t from)
{
    const uint64_t left = r.max_tiles > from ? r.max_tiles - from : 0;
    if (r.o.eps <= 0.0) return left;
    const uint64_t tpc = r.tiles_per_chunk;
    uint64_t want;
    if (from == 0) {
        const uint64_t min_tiles = (r.o.min_trials + kTile - 1) / kTile;
        want = std::max<uint64_t>(tpc, (min_tiles + tpc - 1) / tpc * tpc);
    } else if (r.trials_done == 0) {
        want = tpc;               // nothing absorbed yet: one more chunk
    } else {
        const double n = (double)r.trials_done;
        const double issued = (double)(from * kTile);
        const double mu = r.sx / n;
        double var = r.sx2 / n - mu * mu;
        if (var < 0) var = 0;
        double need = mu > 0 ? (r.z * r.z * var) / (r.o.eps * r.o.eps * mu * mu) : 4.0 * issued;
        need = std::min(need, 4.0 * issued + 1.0);
        if (from > r.done_tiles && need <= issued) return 0;   // the tiles in flight may suffice
        const double more = std::max(need - issued, (double)r.o.chunk_trials);
        want = (uint64_t)std::ceil(more / kTile);
        want = (want + tpc - 1) / tpc * tpc;
    }
    return std::min(want, left);
}

uint64_t next_tiles(const QueryRun &r) { return tiles_after(r, r.done_tiles); }

uint64_t ahead_tiles(const QueryRun &r) { return r.finished ? 0 : tiles_after(r, r.issued_tiles); }

// Folds the tile sums of tiles [done_tiles, done_tiles + n) (in index order) into
// the run, evaluating Alg. 1 at each chunk checkpoint.  Stops at the first
// converged checkpoint.
void absorb(QueryRun &r, const uint64_t *tiles, uint64_t n)
{
    for (uint64_t j = 0; j < n && !r.finished; ++j) {
        const uint64_t *o = tiles + kTileWords * j;
        const uint64_t tile_idx = r.done_tiles;
        const uint64_t first = tile_idx * kTile;
        const uint64_t cnt = std::min<uint64_t>(kTile, r.o.max_trials > first ? r.o.max_trials - first : 0);
        double s, s2;
        std::memcpy(&s, &o[2], 8);
        std::memcpy(&s2, &o[3], 8);
        r.hits += o[0];
        r.sectors += o[1];
        r.streamed += o[4];
        r.survey += o[5];
        r.sx += s;
        r.sx2 += s2;
        r.trials_done += cnt;
        r.done_tiles++;
        const bool at_ck = (r.done_tiles % r.tiles_per_chunk == 0) || r.done_tiles == r.max_tiles;
        if (!at_ck) continue;
        r.ck_trials = r.trials_done;
        r.ck_hits = r.hits;
        r.ck_sectors = r.sectors;
        r.ck_streamed = r.streamed;
        r.ck_survey = r.survey;
        r.ck_sx = r.sx;
        r.ck_sx2 = r.sx2;
        if (r.o.eps > 0.0 && r.trials_done >= r.o.min_trials) {
            double mu, var, eh;
            alg1((double)r.trials_done, r.sx, r.sx2, r.z, &mu, &var, &eh);
            if (mu > 0.0 && eh <= r.o.eps) {
                r.converged = true;
                r.finished = true;
            }
        }
        if (r.done_tiles == r.max_tiles) r.finished = true;
    }
}

void fill_result(const QueryRun &r, agis_result *out)
{
    std::memset(out, 0, sizeof(*out));
    const double n = (double)r.ck_trials;
    double mu = 0, var = 0, eh = INFINITY;
    if (r.ck_trials > 0) alg1(n, r.ck_sx, r.ck_sx2, r.z > 0 ? r.z : agis_z_of_delta(r.o.delta > 0 && r.o.delta < 1 ? r.o.delta : 0.05), &mu, &var, &eh);
    // on an orientation every clique is one trajectory, so mu estimates the cliques
    // themselves and the embedding count is mu * |Aut| = mu * k!
    const double aut = r.p && r.p->aut ? (double)r.p->aut : 0.0;
    out->estimate = r.oriented ? mu * aut : mu;
    out->subgraphs = r.oriented ? mu : (aut > 0 ? mu / aut : 0.0);
    out->mean = mu;
    out->var = var;
    out->eps_hat = eh;
    out->sum_x = r.ck_sx;
    out->sum_x2 = r.ck_sx2;
    out->trials = r.ck_trials;
    out->hits = r.ck_hits;
    out->sectors = r.ck_sectors;
    out->sectors_streamed = r.ck_streamed;
    out->sectors_survey = r.ck_survey;
    out->converged = r.converged ? 1 : 0;
    out->launches = r.launches;
    out->t_prep_s = r.t_prep;
}

// Tiles per work item for an epoch of `tiles` tiles on `grid` CTAs: the autotuned
// span (else kMaxSpan), halved while the CTAs would get fewer than two items each,
// so that short epochs (a query's first checkpoint) still spread over every SM.
int span_for(const agis_graph *g, size_t tiles, int grid)
{
    int span = g->ctx->span > 0 ? g->ctx->span : kMaxSpan;
    while (span > 1 && tiles < (size_t)span * (size_t)grid * 2) span >>= 1;
    return span;
}

// Stages the epoch's work items for the given runs (tile ranges) into lb's pinned
// buffers and fills lb.h_counter: first the last `tail` tiles (in query then tile
// order) as single-tile items for the scatter kernel, then the others as items of up
// to `span` tiles for the main kernel.  Tile output slots run 0, 1, ... in query then
// tile order.  Returns the number of items.
size_t stage_items(LaunchBuffers &lb, std::vector<QueryRun *> &runs, const std::vector<uint64_t> &ntiles, int span,
                   size_t tail)
{
    size_t total = 0;
    for (uint64_t n : ntiles) total += n;
    const uint64_t head = total - std::min(tail, total);
    size_t m = 0;
    auto emit = [&](size_t q, uint64_t j, uint64_t nt, uint64_t slot) {
        const QueryRun &r = *runs[q];
        const uint64_t first = (r.issued_tiles + j) * kTile;
        WorkItem &w = lb.h_items[m++];
        w.query = (uint32_t)q;
        w.count = (uint32_t)std::min<uint64_t>(nt * kTile, r.o.max_trials - first);
        w.first = first;
        w.slot = slot;
    };
    uint64_t g0 = 0;            // epoch tile index of the query's first tile
    for (size_t q = 0; q < runs.size(); ++q) {
        const uint64_t from = head > g0 ? std::min<uint64_t>(head - g0, ntiles[q]) : 0;
        for (uint64_t j = from; j < ntiles[q]; ++j) emit(q, j, 1, g0 + j);
        g0 += ntiles[q];
    }
    const size_t n_tail = m;
    g0 = 0;
    for (size_t q = 0; q < runs.size(); ++q) {
        const uint64_t nh = head > g0 ? std::min<uint64_t>(head - g0, ntiles[q]) : 0;
        for (uint64_t j = 0; j < nh; j += (uint64_t)span) emit(q, j, std::min<uint64_t>((uint64_t)span, nh - j), g0 + j);
        g0 += ntiles[q];
    }
    for (size_t q = 0; q < runs.size(); ++q) {
        lb.h_queries[q] = runs[q]->dq;
        runs[q]->issued_tiles += ntiles[q];
    }
    lb.h_counter[0] = (uint32_t)n_tail;
    lb.h_counter[1] = (uint32_t)m;
    lb.h_counter[2] = 0;
    lb.h_counter[3] = (uint32_t)n_tail;
    return m;
}

static bool any_anchor(const std::vector<QueryRun *> &runs)
{
    for (const QueryRun *r : runs)
        if (r->dq.flags & kFlagAnchor) return true;
    return false;
}

// The aux stream and fork/join events of lb's tail launches, created on first use.
static int ensure_aux(LaunchBuffers &lb)
{
    if (!lb.aux) AGIS_CUDA_TRY(cudaStreamCreateWithFlags(&lb.aux, cudaStreamNonBlocking));
    if (!lb.ev_fork) AGIS_CUDA_TRY(cudaEventCreateWithFlags(&lb.ev_fork, cudaEventDisableTiming));
    if (!lb.ev_join) AGIS_CUDA_TRY(cudaEventCreateWithFlags(&lb.ev_join, cudaEventDisableTiming));
    return AGIS_OK;
}

// One epoch by plain stream launches: the main kernel over the head items (urgent),
// the scatter kernel and tile reduction over the tail on lb.aux beside it.
int run_epoch_direct(agis_graph *g, std::vector<QueryRun *> &runs, const std::vector<uint64_t> &ntiles,
                     size_t total)
{
    agis::NvtxRange nvtx_range("agis:epoch");
    LaunchBuffers &lb = g->lb;
    cudaStream_t st = g->ctx->stream;
    int rc = ensure_buffers(lb, runs.size(), total);
    if (rc != AGIS_OK) return rc;
    const int full = grid_for(g, (size_t)g->ctx->sm_count * 64);
    const size_t tail = tail_tiles(total, full);
    const size_t head = total - tail;
    const int hgrid = grid_for(g, head);
    if ((rc = ensure_scratch(g, lb, 2 * full)) != AGIS_OK) return rc;
    if ((rc = ensure_scatter(lb, tail)) != AGIS_OK) return rc;
    const size_t n = stage_items(lb, runs, ntiles, head ? span_for(g, head, hgrid) : 1, tail);
    const size_t n_tail = lb.h_counter[3];
    AGIS_CUDA_TRY(cudaMemcpyAsync(lb.d_queries, lb.h_queries, sizeof(DevQuery) * runs.size(), cudaMemcpyHostToDevice, st));
    AGIS_CUDA_TRY(cudaMemcpyAsync(lb.d_items, lb.h_items, sizeof(WorkItem) * n, cudaMemcpyHostToDevice, st));
    AGIS_CUDA_TRY(cudaMemcpyAsync(lb.d_counter, lb.h_counter, 4 * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    const bool anchor = any_anchor(runs);
    if (head == 0) {
        rc = launch_scatter(g, lb, full, full, n_tail, st, anchor);
    } else {
        if ((rc = ensure_aux(lb)) != AGIS_OK) return rc;
        AGIS_CUDA_TRY(cudaEventRecord(lb.ev_fork, st));
        rc = launch_sampler(g, lb, grid_for(g, n - n_tail), nullptr, st, 0, 0, 1, nullptr, anchor, true);
        if (rc != AGIS_OK) return rc;
        AGIS_CUDA_TRY(cudaStreamWaitEvent(lb.aux, lb.ev_fork, 0));
        rc = launch_scatter(g, lb, full, full, n_tail, lb.aux, anchor);
        if (rc != AGIS_OK) return rc;
        AGIS_CUDA_TRY(cudaEventRecord(lb.ev_join, lb.aux));
        AGIS_CUDA_TRY(cudaStreamWaitEvent(st, lb.ev_join, 0));
    }
    if (rc != AGIS_OK) return rc;
    AGIS_CUDA_TRY(cudaMemcpyAsync(lb.h_out, lb.d_out, sizeof(uint64_t) * kTileWords * total, cudaMemcpyDeviceToHost, st));
    AGIS_CUDA_TRY(cudaStreamSynchronize(st));
    return AGIS_OK;
}

// The batched epoch as a CUDA graph: H2D of queries, items and counters, then the
// main kernel (urgent) beside the scatter kernel and tile reduction of the tail, D2H
// of the tile sums; an epoch of no more tiles than the grid has CTAs uses a graph
// without the main kernel.  Each is built once per buffer generation and grid;
// sizes are patched per epoch.  `start` and `done` (either may be null) are recorded
// around the graph launch.  The scratch (per-warp candidate lists) of scratch_lb
// must cover twice the full grid: the main kernel's CTAs use the first half, the
// scatter kernel's the second.
int enqueue_epoch_graph(agis_graph *g, LaunchBuffers &lb, const LaunchBuffers &scratch_lb,
                        std::vector<QueryRun *> &runs, const std::vector<uint64_t> &ntiles, size_t total,
                        cudaEvent_t start, cudaEvent_t done)
{
    agis::NvtxRange nvtx_range("agis:epoch");
    cudaStream_t st = g->ctx->stream;
    int rc = ensure_buffers(lb, runs.size(), total);
    if (rc != AGIS_OK) return rc;
    const int grid = std::min(grid_for(g, (size_t)g->ctx->sm_count * 64), scratch_lb.scratch_grid / 2);
    if (grid <= 0) return AGIS_ERR_ARG;
    if (&lb != &scratch_lb && (lb.d_scratch != scratch_lb.d_scratch || lb.scratch_cap != scratch_lb.scratch_cap)) {
        lb.d_scratch = scratch_lb.d_scratch;
        lb.scratch_cap = scratch_lb.scratch_cap;
        lb.scratch_grid = scratch_lb.scratch_grid;
        lb.scratch_borrowed = true;
        ++lb.generation;
    }
    if ((rc = ensure_scatter(lb, tail_capacity(grid))) != AGIS_OK) return rc;
    const bool anchor = any_anchor(runs);
    const size_t tail = tail_tiles(total, grid);
    const size_t head = total - tail;
    const size_t n = stage_items(lb, runs, ntiles, head ? span_for(g, head, grid) : 1, tail);
    const bool mixed = head > 0;
    cudaGraph_t &graph = mixed ? lb.graph : lb.sgraph;
    cudaGraphExec_t &exec = mixed ? lb.exec : lb.sexec;
    cudaGraphNode_t &h2d_q = mixed ? lb.n_h2d_q : lb.s_h2d_q;
    cudaGraphNode_t &h2d_i = mixed ? lb.n_h2d_i : lb.s_h2d_i;
    cudaGraphNode_t &h2d_c = mixed ? lb.n_h2d_c : lb.s_h2d_c;
    cudaGraphNode_t &d2h = mixed ? lb.n_d2h : lb.s_d2h;
    uint64_t &gen = mixed ? lb.graph_generation : lb.sgraph_generation;
    int &ggrid = mixed ? lb.graph_grid : lb.sgraph_grid;
    bool &ganchor = mixed ? lb.graph_anchor : lb.sgraph_anchor;
    uint64_t &gl2 = mixed ? lb.graph_l2 : lb.sgraph_l2;
    if (!exec || gen != lb.generation || ggrid != grid || ganchor != anchor || gl2 != g->l2_window_bytes) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        AGIS_CUDA_TRY(cudaGraphCreate(&graph, 0));
        AGIS_CUDA_TRY(cudaGraphAddMemcpyNode1D(&h2d_q, graph, nullptr, 0, lb.d_queries, lb.h_queries,
                                               sizeof(DevQuery), cudaMemcpyHostToDevice));
        AGIS_CUDA_TRY(cudaGraphAddMemcpyNode1D(&h2d_i, graph, &h2d_q, 1, lb.d_items, lb.h_items, sizeof(WorkItem),
                                               cudaMemcpyHostToDevice));
        AGIS_CUDA_TRY(cudaGraphAddMemcpyNode1D(&h2d_c, graph, &h2d_i, 1, lb.d_counter, lb.h_counter,
                                               4 * sizeof(uint32_t), cudaMemcpyHostToDevice));
        cudaGraphNode_t ends[2];
        size_t nends = 0;
        if (mixed) {
            rc = add_sampler_node(g, lb, grid, graph, &h2d_c, 1, &lb.n_kernel, anchor, true);
            if (rc != AGIS_OK) return rc;
            ends[nends++] = lb.n_kernel;
        }
        cudaGraphNode_t &skernel = mixed ? lb.n_scatter : lb.s_kernel;
        cudaGraphNode_t &reduce = mixed ? lb.n_reduce : lb.s_reduce;
        rc = add_scatter_nodes(g, lb, grid, grid, tail_capacity(grid), graph, &h2d_c, 1, &skernel, &reduce, anchor);
        if (rc != AGIS_OK) return rc;
        ends[nends++] = reduce;
        AGIS_CUDA_TRY(cudaGraphAddMemcpyNode1D(&d2h, graph, ends, nends, lb.h_out, lb.d_out,
                                               kTileWords * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        AGIS_CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
        gen = lb.generation;
        ganchor = anchor;
        ggrid = grid;
        gl2 = g->l2_window_bytes;
    }
    AGIS_CUDA_TRY(cudaGraphExecMemcpyNodeSetParams1D(exec, h2d_q, lb.d_queries, lb.h_queries,
                                                     sizeof(DevQuery) * runs.size(), cudaMemcpyHostToDevice));
    AGIS_CUDA_TRY(cudaGraphExecMemcpyNodeSetParams1D(exec, h2d_i, lb.d_items, lb.h_items,
                                                     sizeof(WorkItem) * std::max<size_t>(n, 1), cudaMemcpyHostToDevice));
    AGIS_CUDA_TRY(cudaGraphExecMemcpyNodeSetParams1D(exec, d2h, lb.h_out, lb.d_out,
                                                     sizeof(uint64_t) * kTileWords * std::max<size_t>(total, 1),
                                                     cudaMemcpyDeviceToHost));
    if (start) AGIS_CUDA_TRY(cudaEventRecord(start, st));
    count_launch(mixed ? 3 : 2);
    AGIS_CUDA_TRY(cudaGraphLaunch(exec, st));
    if (done) AGIS_CUDA_TRY(cudaEventRecord(done, st));
    return AGIS_OK;
}

int run_epoch_graph(agis_graph *g, std::vector<QueryRun *> &runs, const std::vector<uint64_t> &ntiles,
                    size_t total)
{
    LaunchBuffers &lb = g->lb;
    const int grid = grid_for(g, (size_t)g->ctx->sm_count * 64);
    int rc = ensure_scratch(g, lb, 2 * grid);
    if (rc != AGIS_OK) return rc;
    rc = enqueue_epoch_graph(g, lb, lb, runs, ntiles, total, nullptr, nullptr);
    if (rc != AGIS_OK) return rc;
    AGIS_CUDA_TRY(cudaStreamSynchronize(g->ctx->stream));
    return AGIS_OK;
}

// Drives a set of queries to completion; each epoch is one launch over the next
// tiles of every unfinished query.  `use_graph` selects the captured-graph epoch.
int drive(agis_graph *g, std::vector<QueryRun *> &runs, bool use_graph, size_t max_items_per_epoch)
{
    const double t0 = now_s();
    for (;;) {
        std::vector<QueryRun *> active;
        std::vector<uint64_t> ntiles;
        size_t total = 0;
        for (QueryRun *r : runs) {
            if (r->finished) continue;
            uint64_t n = next_tiles(*r);
            if (n == 0) { r->finished = true; continue; }
            active.push_back(r);
            ntiles.push_back(n);
            total += n;
        }
        if (active.empty()) break;
        if (max_items_per_epoch && total > max_items_per_epoch) {
            // shrink proportionally, keeping whole chunks and at least one chunk each
            const double f = (double)max_items_per_epoch / (double)total;
            total = 0;
            for (size_t q = 0; q < active.size(); ++q) {
                const uint64_t tpc = active[q]->tiles_per_chunk;
                uint64_t n = (uint64_t)((double)ntiles[q] * f) / tpc * tpc;
                n = std::max<uint64_t>(n, std::min<uint64_t>(tpc, ntiles[q]));
                ntiles[q] = n;
                total += n;
            }
        }
        int rc = use_graph ? run_epoch_graph(g, active, ntiles, total) : run_epoch_direct(g, active, ntiles, total);
        if (rc != AGIS_OK) return rc;
        size_t k = 0;
        for (size_t q = 0; q < active.size(); ++q) {
            active[q]->launches++;
            absorb(*active[q], g->lb.h_out + kTileWords * k, ntiles[q]);
            k += ntiles[q];
        }
    }
    const double dt = now_s() - t0;
    (void)dt;
    return AGIS_OK;
}

}  // namespace agis

using namespace agis;

extern "C" const char *agis_status_str(int s)
{
    switch (s) {
    case AGIS_OK: return "ok";
    case AGIS_ERR_ARG: return "invalid argument";
    case AGIS_ERR_NOMEM: return "out of memory";
    case AGIS_ERR_CUDA: return "CUDA error";
    case AGIS_ERR_GRAPH: return "invalid graph";
    case AGIS_ERR_PATTERN: return "invalid pattern";
    case AGIS_ERR_TIMEOUT: return "timeout";
    case AGIS_ERR_BUSY: return "busy";
    case AGIS_ERR_STATE: return "invalid state";
    case AGIS_ERR_IO: return "file error";
    default: return "unknown status";
    }
}

extern "C" int agis_tile_trials(void)
{
    return kTile;
}

extern "C" void agis_default_opts(agis_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->eps = 0.1;
    o->delta = 0.01;
    o->beta = 0.8;
    o->mode = AGIS_MODE_AUTO;
    o->seed = 1;
    o->min_trials = 65536;
    o->max_trials = 1ull << 32;
    o->chunk_trials = 65536;
}

// Phi^{-1}(1 - delta/2): bisection on the upper tail 0.5 erfc(z / sqrt 2) = delta / 2.
extern "C" double agis_z_of_delta(double delta)
{
    if (!(delta > 0.0 && delta < 1.0)) return NAN;
    double lo = 0.0, hi = 64.0;
    for (int it = 0; it < 256 && hi - lo > 0.0; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        const double tail = 0.5 * std::erfc(mid / std::sqrt(2.0));
        if (tail > 0.5 * delta) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

extern "C" int agis_create(int device, void *cuda_stream, agis_ctx **out)
{
    if (!out) return AGIS_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return AGIS_ERR_CUDA;
    if (device < 0 || device >= ndev) return AGIS_ERR_ARG;
    AGIS_CUDA_TRY(cudaSetDevice(device));
    agis_ctx *c = new (std::nothrow) agis_ctx();
    if (!c) return AGIS_ERR_NOMEM;
    c->device = device;
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return AGIS_ERR_CUDA;
    }
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return AGIS_ERR_CUDA;
        }
        c->own_stream = true;
    }
    *out = c;
    return AGIS_OK;
}

namespace agis {

void ctx_retain(agis_ctx *c) { c->refs.fetch_add(1); }

void ctx_release(agis_ctx *c)
{
    if (c->refs.fetch_sub(1) != 1) return;
    cudaSetDevice(c->device);
    if (c->l2_limit_set) {
        // the persisting-L2 set-aside as it was before the first windowed launch
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, c->l2_limit_before);
        cudaGetLastError();
    }
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

void graph_retain(agis_graph *g) { g->refs.fetch_add(1); }

void graph_release(agis_graph *g)
{
    if (g->refs.fetch_sub(1) != 1) return;
    agis_ctx *c = g->ctx;
    {
        std::lock_guard<std::recursive_mutex> lk(g->mu);
        cudaSetDevice(c->device);
        cudaStreamSynchronize(c->stream);
        // lines of the bitmaps marked persisting go back to normal before their memory does
        if (c->l2_limit_set && g->hub_bits) cudaCtxResetPersistingL2Cache();
        for (auto &kv : g->tables) free_table(kv.second);
        g->tables.clear();
        free_buffers(g->lb);
        cudaFree(g->off);
        cudaFree(g->cols);
        cudaFree(g->nsum);
        cudaFree(g->hits);
        cudaFree(g->hub_id);
        cudaFree(g->hub_bits);
        cudaFree(g->rp_base);
        cudaFree(g->rp_rows);
    }
    delete g;
    ctx_release(c);
}

}  // namespace agis

// Releases the caller's reference; the context goes away once its last graph does.
extern "C" int agis_destroy(agis_ctx *c)
{
    if (!c) return AGIS_ERR_ARG;
    ctx_release(c);
    return AGIS_OK;
}

// Releases the caller's reference; the graph goes away once no server uses it.
extern "C" int agis_graph_free(agis_graph *g)
{
    if (!g) return AGIS_ERR_ARG;
    graph_release(g);
    return AGIS_OK;
}

extern "C" int agis_estimate(agis_graph *g, const agis_pattern *p, const agis_opts *opts, agis_result *out)
{
    if (!g || !p || !opts || !out) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    QueryRun r;
    int rc = init_run(g, p, opts, r);
    if (rc != AGIS_OK) return rc;
    const double t0 = now_s();
    std::vector<QueryRun *> runs{&r};
    rc = drive(g, runs, false, 0);
    if (rc != AGIS_OK) return rc;
    fill_result(r, out);
    out->t_sample_s = now_s() - t0;
    return AGIS_OK;
}

extern "C" int agis_estimate_batch(agis_graph *g, int n, const agis_pattern *const *patterns,
                                   const agis_opts *opts, agis_result *out)
{
    if (!g || n < 0 || (n > 0 && (!patterns || !opts || !out))) return AGIS_ERR_ARG;
    if (n == 0) return AGIS_OK;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    std::vector<QueryRun> rs((size_t)n);
    for (int i = 0; i < n; ++i) {
        int rc = init_run(g, patterns[i], &opts[i], rs[(size_t)i]);
        if (rc != AGIS_OK) return rc;
    }
    const double t0 = now_s();
    std::vector<QueryRun *> runs;
    for (auto &r : rs) runs.push_back(&r);
    int rc = drive(g, runs, true, 0);
    if (rc != AGIS_OK) return rc;
    const double dt = now_s() - t0;
    for (int i = 0; i < n; ++i) {
        fill_result(rs[(size_t)i], &out[i]);
        out[i].t_sample_s = dt;
    }
    return AGIS_OK;
}

extern "C" int agis_dump_trials(agis_graph *g, const agis_pattern *p, const agis_opts *opts, uint64_t first,
                                uint64_t count, int32_t *emb, uint8_t *hit, double *x, uint64_t *sectors)
{
    agis::NvtxRange nvtx_range("agis:dump");
    if (!g || !p || !opts) return AGIS_ERR_ARG;
    if (count == 0) return AGIS_OK;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    DevQuery dq;
    int rc = make_dev_query(g, p, opts, &dq, nullptr);
    if (rc != AGIS_OK) return rc;
    const uint64_t ntiles = (count + kTile - 1) / kTile;
    LaunchBuffers &lb = g->lb;
    rc = ensure_buffers(lb, 1, ntiles);
    if (rc != AGIS_OK) return rc;
    DumpView dv{nullptr, nullptr, nullptr, nullptr, first};
    const size_t c = (size_t)count;
    auto cleanup = [&]() { cudaFree(dv.emb); cudaFree(dv.hit); cudaFree(dv.x); cudaFree(dv.sectors); };
    if ((emb && cudaMalloc(&dv.emb, sizeof(int32_t) * kMaxK * c) != cudaSuccess) ||
        (hit && cudaMalloc(&dv.hit, c) != cudaSuccess) ||
        (x && cudaMalloc(&dv.x, sizeof(double) * c) != cudaSuccess) ||
        (sectors && cudaMalloc(&dv.sectors, 3 * sizeof(uint64_t) * c) != cudaSuccess)) {
        cleanup();
        return AGIS_ERR_NOMEM;
    }
    lb.h_queries[0] = dq;
    lb.h_counter[0] = 0;
    lb.h_counter[1] = (uint32_t)ntiles;
    cudaMemcpyAsync(lb.d_queries, lb.h_queries, sizeof(DevQuery), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(lb.d_counter, lb.h_counter, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    const int grid = grid_for(g, ntiles);
    if (rc == AGIS_OK) rc = ensure_scratch(g, lb, grid);
    if (rc == AGIS_OK) rc = launch_sampler(g, lb, grid, &dv, st, first, count, 1, nullptr, true);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == AGIS_OK && e != cudaSuccess) rc = AGIS_ERR_CUDA;
    if (rc == AGIS_OK && emb && cudaMemcpy(emb, dv.emb, sizeof(int32_t) * kMaxK * c, cudaMemcpyDeviceToHost) != cudaSuccess) rc = AGIS_ERR_CUDA;
    if (rc == AGIS_OK && hit && cudaMemcpy(hit, dv.hit, c, cudaMemcpyDeviceToHost) != cudaSuccess) rc = AGIS_ERR_CUDA;
    if (rc == AGIS_OK && x && cudaMemcpy(x, dv.x, sizeof(double) * c, cudaMemcpyDeviceToHost) != cudaSuccess) rc = AGIS_ERR_CUDA;
    if (rc == AGIS_OK && sectors && cudaMemcpy(sectors, dv.sectors, 3 * sizeof(uint64_t) * c, cudaMemcpyDeviceToHost) != cudaSuccess) rc = AGIS_ERR_CUDA;
    cleanup();
    return rc;
}

extern "C" int agis_sample_device(agis_graph *g, const agis_pattern *p, const agis_opts *opts, uint64_t first,
                                  uint64_t ntiles, uint64_t *tile_out)
{
    agis::NvtxRange nvtx_range("agis:sample");
    if (!g || !p || !opts || !tile_out || ntiles == 0 || ntiles > 0xffffffffull) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    int rc = check_opts(opts);
    if (rc != AGIS_OK) return rc;
    LaunchBuffers &lb = g->lb;
    rc = ensure_buffers(lb, 1, 1);
    if (rc != AGIS_OK) return rc;
    DevQuery dq;
    rc = make_dev_query(g, p, opts, &dq, nullptr);
    if (rc != AGIS_OK) return rc;
    // pageable sources: the runtime stages them before the call returns, so back to
    // back calls never wait for the device (the copies are stream-ordered after the
    // previous launch, which is what keeps the shared device slots safe)
    // items of up to AGIS_SAMPLE_SPAN tiles (fewer CTA barriers), smaller while that
    // would leave CTAs without work; each tile keeps its own sums and slot
    const int grid = grid_for(g, ntiles);
    const int span = std::min(AGIS_SAMPLE_SPAN, span_for(g, ntiles, grid));
    const uint32_t counter[2] = {0u, (uint32_t)((ntiles + span - 1) / span)};
    AGIS_CUDA_TRY(cudaMemcpyAsync(lb.d_queries, &dq, sizeof(DevQuery), cudaMemcpyHostToDevice, st));
    AGIS_CUDA_TRY(cudaMemcpyAsync(lb.d_counter, counter, sizeof(counter), cudaMemcpyHostToDevice, st));
    if ((rc = ensure_scratch(g, lb, grid)) != AGIS_OK) return rc;
    return launch_sampler(g, lb, grid, nullptr, st, first, ntiles * kTile, (uint32_t)span, tile_out,
                          (dq.flags & kFlagAnchor) != 0);
}

extern "C" int agis_prepare(agis_graph *g, const agis_pattern *p, const agis_opts *opts)
{
    if (!g || !p || !opts) return AGIS_ERR_ARG;
    int rc = check_opts(opts);
    if (rc != AGIS_OK) return rc;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    DevQuery dq;
    rc = make_dev_query(g, p, opts, &dq, nullptr);
    if (rc != AGIS_OK) return rc;
    return cuda_status(cudaStreamSynchronize(g->ctx->stream));
}

extern "C" uint64_t agis_kernel_launches(void) { return g_launches.load(); }

extern "C" int agis_autotune(agis_graph *g, int n, const agis_pattern *const *patterns, const agis_opts *opts,
                             uint64_t trials_per_query, int32_t *blocks_per_sm, int32_t *tiles_per_item)
{
    agis::NvtxRange nvtx_range("agis:autotune");
    if (!g || n <= 0 || !patterns || !opts || trials_per_query == 0) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    int occ = 1;
    int rc = sampler_occupancy(&occ);
    if (rc != AGIS_OK) return rc;
    occ = std::max(1, occ);
    const uint64_t ntiles = (trials_per_query + kTile - 1) / kTile;
    std::vector<DevQuery> dqs((size_t)n);
    bool anchor = false;
    for (int i = 0; i < n; ++i) {
        if ((rc = check_opts(&opts[i])) != AGIS_OK) return rc;
        if ((rc = make_dev_query(g, patterns[i], &opts[i], &dqs[(size_t)i], nullptr)) != AGIS_OK) return rc;
        anchor = anchor || (dqs[(size_t)i].flags & kFlagAnchor);
    }
    LaunchBuffers &lb = g->lb;
    const size_t tiles = (size_t)n * ntiles;
    if ((rc = ensure_buffers(lb, (size_t)n, tiles)) != AGIS_OK) return rc;
    if ((rc = ensure_scratch(g, lb, g->ctx->sm_count * occ)) != AGIS_OK) return rc;
    AGIS_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) lb.h_queries[i] = dqs[(size_t)i];
    AGIS_CUDA_TRY(cudaMemcpyAsync(lb.d_queries, lb.h_queries, sizeof(DevQuery) * (size_t)n, cudaMemcpyHostToDevice, st));
    cudaEvent_t e0, e1;
    AGIS_CUDA_TRY(cudaEventCreate(&e0));
    AGIS_CUDA_TRY(cudaEventCreate(&e1));
    // every (CTAs per SM, tiles per item) pair on the same trials; the first launch
    // only warms the caches
    int best_c = occ, best_s = 1;
    float best_ms = -1.0f;
    for (int trial = -1; trial < occ * 3 && rc == AGIS_OK; ++trial) {
        const int c = trial < 0 ? occ : 1 + trial / 3;
        const int span = trial < 0 ? 1 : 1 << (trial % 3);
        size_t m = 0;
        for (int i = 0; i < n; ++i) {
            for (uint64_t j = 0; j < ntiles; j += (uint64_t)span) {
                WorkItem &w = lb.h_items[m++];
                w.query = (uint32_t)i;
                w.count = (uint32_t)(std::min<uint64_t>((uint64_t)span, ntiles - j) * kTile);
                w.first = j * kTile;
                w.slot = (uint64_t)i * ntiles + j;
            }
        }
        const uint32_t counter[2] = {0u, (uint32_t)m};
        cudaMemcpyAsync(lb.d_items, lb.h_items, sizeof(WorkItem) * m, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(lb.d_counter, counter, sizeof(counter), cudaMemcpyHostToDevice, st);
        const int grid = (int)std::min<size_t>((size_t)g->ctx->sm_count * (size_t)c, m);
        cudaEventRecord(e0, st);
        rc = launch_sampler(g, lb, grid, nullptr, st, 0, 0, 1, nullptr, anchor);
        cudaEventRecord(e1, st);
        if (rc != AGIS_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = AGIS_ERR_CUDA; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (trial >= 0 && (best_ms < 0.0f || ms < best_ms)) {
            best_ms = ms;
            best_c = c;
            best_s = span;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != AGIS_OK) return rc;
    g->ctx->blocks_per_sm = best_c;
    g->ctx->span = best_s;
    if (blocks_per_sm) *blocks_per_sm = best_c;
    if (tiles_per_item) *tiles_per_item = best_s;
    return AGIS_OK;
}
