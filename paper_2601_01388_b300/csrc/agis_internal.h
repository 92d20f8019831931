// Internal types shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/agis.h"
#include "agis_device.h"

namespace agis {

// An NVTX range for the scope (header-only NVTX 3: without a profiler attached a
// push/pop costs a check of one function pointer).  Range names start with "agis:"
// so that a profiler's launch list can be attributed to the phases of the path.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct WeightTable {
    int32_t cfg[4];
    int32_t shift = 0;
    uint64_t *q = nullptr;      // nv
    uint64_t *pref = nullptr;   // nv, inclusive prefix over vertices (|B| = 0 configs)
    uint64_t *rowp = nullptr;   // inclusive prefix inside each row (|B| = 1 configs): nnz
                                // entries, or only the rows of g->rp_base when rowp_partial
    bool rowp_partial = false;
    uint64_t total = 0;
    size_t bytes = 0;
    uint64_t last_use = 0;
    int pins = 0;               // queries of a running server that use it
};

// Launch-side scratch: device buffers grown on demand and reused across launches.
struct LaunchBuffers {
    DevQuery *d_queries = nullptr;
    size_t cap_queries = 0;
    WorkItem *d_items = nullptr;
    size_t cap_items = 0;
    uint64_t *d_out = nullptr;  // kTileWords words per tile slot
    size_t cap_out = 0;
    // [0] the main kernel's item counter (starts at the number of tail items), [1] the
    // end of its items; [2] the scatter kernel's trial counter, [3] its number of items
    uint32_t *d_counter = nullptr;
    // per-trial outputs of scatter launches (trials of up to cap_scatter)
    double *d_sx = nullptr;
    uint8_t *d_shit = nullptr;
    uint64_t *d_ssec = nullptr;
    size_t cap_scatter = 0;
    void *d_scratch = nullptr;     // per-warp candidate lists of the sampler
    bool scratch_borrowed = false; // d_scratch belongs to another LaunchBuffers (not freed here)
    size_t scratch_bytes = 0;
    uint32_t scratch_cap = 0;      // entries per list
    int scratch_grid = 0;          // CTAs the scratch was sized for
    // pinned host mirrors
    DevQuery *h_queries = nullptr;
    WorkItem *h_items = nullptr;
    uint64_t *h_out = nullptr;
    uint32_t *h_counter = nullptr;
    size_t hcap_queries = 0, hcap_items = 0, hcap_out = 0;
    // captured epoch graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t n_h2d_q = nullptr, n_h2d_i = nullptr, n_h2d_c = nullptr, n_kernel = nullptr,
                    n_scatter = nullptr, n_reduce = nullptr, n_d2h = nullptr;
    int graph_grid = 0;
    uint64_t generation = 0;       // bumps when device buffers move (graph must be rebuilt)
    uint64_t graph_generation = ~0ull;
    bool graph_anchor = false;  // the cached graph's kernel node is the anchor-capable instance
    // the captured scatter epoch: H2D, scatter kernel, tile reduction, D2H
    cudaGraph_t sgraph = nullptr;
    cudaGraphExec_t sexec = nullptr;
    cudaGraphNode_t s_h2d_q = nullptr, s_h2d_i = nullptr, s_h2d_c = nullptr, s_kernel = nullptr, s_reduce = nullptr,
                    s_d2h = nullptr;
    int sgraph_grid = 0;
    uint64_t sgraph_generation = ~0ull;
    bool sgraph_anchor = false;
    uint64_t graph_l2 = ~0ull, sgraph_l2 = ~0ull;  // the L2 window the cached graphs were built with
    // stream and events of the tail's scatter launch in epochs of stream launches
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

}  // namespace agis

struct agis_ctx {
    std::atomic<int> refs{1};   // the creator plus every live graph of this context
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    int blocks_per_sm = 0;      // sampler CTAs per SM chosen by the autotuner (0 = not tuned)
    bool l2_limit_set = false;  // the persisting-L2 set-aside was raised (restored at release)
    size_t l2_limit_before = 0;
    int span = 0;               // tiles per work item chosen by the autotuner (0 = not tuned)
};

struct agis_pattern {
    int k = 0;
    int order[agis::kMaxK] = {0};
    int nback[agis::kMaxK] = {0};
    int back[agis::kMaxK][agis::kMaxK] = {{0}};
    int cfg[agis::kMaxK][4] = {{0}};
    double certainty[agis::kMaxK] = {0};
    uint64_t aut = 0;
};

struct agis_graph {
    std::atomic<int> refs{1};   // the creator plus every live server on this graph
    agis_ctx *ctx = nullptr;
    int64_t nv = 0, nnz = 0, max_deg = 0;
    int64_t *off = nullptr;
    int32_t *cols = nullptr;
    uint64_t *nsum = nullptr;
    uint32_t *hits = nullptr;
    bool prepped = false;
    bool oriented = false;      // degree-ordered orientation (agis_graph_orient): out-rows only
    double c_min = 0.0;
    uint64_t prep_seed = 0;
    std::map<uint64_t, agis::WeightTable> tables;
    uint64_t use_clock = 0;
    std::recursive_mutex mu;
    agis::LaunchBuffers lb;     // used by estimate/batch/dump (under mu)
    // memory policy (agis_graph_set_memory_policy)
    size_t rowp_budget = 0;     // largest row-prefix table built in full; beyond it only high-degree rows
    size_t bitmap_budget = 0;   // total bytes of hub neighbour bitmaps (0: a sixteenth of device memory)
    int64_t bitmap_min_degree = 1024;
    uint32_t list_cap = 65536;  // per-warp candidate-list capacity
    // partial row-prefix layout shared by every configuration (built on demand)
    int64_t *rp_base = nullptr; // per vertex, -1 if its row has no prefix
    int32_t *rp_rows = nullptr; // the vertices whose rows have one
    int64_t rp_nrows = 0, rp_entries = 0, rp_min_degree = 0;
    // neighbour bitmaps of the highest-degree vertices (built by preprocessing)
    int32_t *hub_id = nullptr;
    uint32_t *hub_bits = nullptr;
    int64_t hub_words = 0;
    int64_t n_hubs = 0;
    int64_t hub_min_degree = 0;
    // bytes of hub bitmaps (highest degrees first) kept persisting in L2 by sampler
    // launches (agis_graph_set_l2_window)
    uint64_t l2_window_bytes = 48ull << 20;
};

namespace agis {

// graph.cu
int build_hub_bitmaps(agis_graph *g);
int build_partial_rowp_layout(agis_graph *g);
bool rowp_full_fits(const agis_graph *g);
int inclusive_scan_u64(agis_ctx *ctx, const uint64_t *in, int64_t n, uint64_t *out);
int build_weight_table(agis_graph *g, const int32_t cfg[4], bool need_pref, bool need_rowp,
                       WeightTable **out);
uint64_t cfg_key(const int32_t cfg[4]);
size_t table_bytes(const agis_graph *g, const int32_t cfg[4], bool need_pref, bool need_rowp);
void free_table(WeightTable &t);

// sample.cu
// sample.cu: the kernel instance for dumps, or for launches with (anchor) or
// without anchor-draw queries
const void *sampler_function(bool dump, bool anchor);
// launch.cu.  anchor: some staged query uses the anchor draw (selects the instance);
// urgent: launch at the device's greatest stream priority
int launch_sampler(agis_graph *g, LaunchBuffers &lb, int grid, const DumpView *dump,
                   cudaStream_t stream, uint64_t implicit_first, uint64_t implicit_count,
                   uint32_t implicit_span, uint64_t *tile_out, bool anchor, bool urgent = false);
// tiles per work item for an epoch of `tiles` tiles on `grid` CTAs (runtime.cu)
int span_for(const agis_graph *g, size_t tiles, int grid);
int add_sampler_node(agis_graph *g, LaunchBuffers &lb, int grid, cudaGraph_t graph,
                     const cudaGraphNode_t *deps, size_t ndeps, cudaGraphNode_t *node, bool anchor,
                     bool urgent = false);
int sampler_occupancy(int *blocks_per_sm);
// the scatter kernel instance and the tile reduction of scatter epochs (sample.cu)
const void *scatter_function(bool anchor);
const void *tile_reduce_function();
// launch.cu: the scatter kernel on `grid` CTAs over lb's staged tail items (the
// first lb.d_counter[3] items), its warps' candidate lists after those of the first
// `scratch_skip` CTAs, then the tile reduction on `rgrid` CTAs (at least one per item)
int launch_scatter(agis_graph *g, LaunchBuffers &lb, int grid, int scratch_skip, size_t rgrid, cudaStream_t stream,
                   bool anchor);
int add_scatter_nodes(agis_graph *g, LaunchBuffers &lb, int grid, int scratch_skip, size_t rgrid, cudaGraph_t graph,
                      const cudaGraphNode_t *deps, size_t ndeps, cudaGraphNode_t *kernel, cudaGraphNode_t *reduce,
                      bool anchor);
// the tiles of an epoch of `tiles` tiles on a full grid of `grid` CTAs that the
// scatter kernel runs (runtime.cu)
size_t tail_tiles(size_t tiles, int grid);
// the most tiles tail_tiles returns for that grid
size_t tail_capacity(int grid);
int ensure_scatter(LaunchBuffers &lb, size_t tiles);

// runtime.cu
int make_dev_query(agis_graph *g, const agis_pattern *p, const agis_opts *o, DevQuery *dq,
                   double *t_prep);
// weight configuration of step i: the factors that `terms` drops get exponent 0, and
// on an oriented graph |B| is 0 (no backward vertex lies in a later vertex's out-row)
void effective_cfg(const agis_pattern *p, int i, int32_t terms, bool oriented, int32_t out[4]);
// true when step i's f_approx weight is the same for every candidate of its S_tau
// build, so the step draws by position with no table (see runtime.cu)
bool step_weights_flat(const agis_pattern *p, int i, const agis_opts *o, bool oriented);
// true when step i reads an f_approx weight table: D(i) chose f_approx and the
// weights are not flat
bool step_uses_table(const agis_pattern *p, int i, const agis_opts *o, bool oriented, const uint8_t *use);
int ensure_buffers(LaunchBuffers &lb, size_t n_queries, size_t n_items);
int grid_for(agis_graph *g, size_t n_items);
int ensure_scratch(agis_graph *g, LaunchBuffers &lb, int grid);
size_t scratch_stride(uint32_t cap);

// Per-query progress of the adaptive loop (Alg. 1 at chunk checkpoints).
struct QueryRun {
    const agis_pattern *p = nullptr;
    agis_opts o{};
    DevQuery dq{};
    double z = 0.0;
    uint64_t max_tiles = 0;       // ceil(max_trials / 1024)
    uint64_t tiles_per_chunk = 0;
    uint64_t done_tiles = 0;      // tiles whose sums are in
    uint64_t issued_tiles = 0;    // tiles staged for launches so far (>= done_tiles; more
                                  // while a server's epochs are in flight)
    uint64_t trials_done = 0;
    uint64_t hits = 0, sectors = 0, streamed = 0, survey = 0;
    double sx = 0.0, sx2 = 0.0;
    uint64_t ck_trials = 0, ck_hits = 0, ck_sectors = 0;   // at the last checkpoint
    uint64_t ck_streamed = 0, ck_survey = 0;
    double ck_sx = 0.0, ck_sx2 = 0.0;
    bool finished = false;
    bool converged = false;
    bool oriented = false;        // sampled on a degree-ordered orientation: X counts cliques once
    int launches = 0;
    double t_prep = 0.0;
};
int check_opts(const agis_opts *o);
int init_run(agis_graph *g, const agis_pattern *p, const agis_opts *o, QueryRun &r);
uint64_t next_tiles(const QueryRun &r);
// tiles to issue next while issued_tiles - done_tiles are still in flight
uint64_t ahead_tiles(const QueryRun &r);
void absorb(QueryRun &r, const uint64_t *tiles, uint64_t n);
void fill_result(const QueryRun &r, agis_result *out);
int run_epoch_graph(agis_graph *g, std::vector<QueryRun *> &runs, const std::vector<uint64_t> &ntiles,
                    size_t total);
// Stages an epoch into lb (its own pinned and device buffers, the scratch of
// scratch_lb) and enqueues its captured graph on the context's stream, recording
// `done` after the tile sums' copy to lb.h_out; no host synchronisation.
int enqueue_epoch_graph(agis_graph *g, LaunchBuffers &lb, const LaunchBuffers &scratch_lb,
                        std::vector<QueryRun *> &runs, const std::vector<uint64_t> &ntiles, size_t total,
                        cudaEvent_t start, cudaEvent_t done);
void free_buffers(LaunchBuffers &lb);
double now_s();

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? AGIS_OK : AGIS_ERR_CUDA; }

// Lifetimes: a graph keeps its context alive and a server its graph, whatever
// order the caller releases them in.
void ctx_retain(agis_ctx *c);
void ctx_release(agis_ctx *c);
void graph_retain(agis_graph *g);
void graph_release(agis_graph *g);

// process-wide count of kernel launches (diagnostics)
extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace agis

#define AGIS_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) {                              \
            return _e == cudaErrorMemoryAllocation ? AGIS_ERR_NOMEM : AGIS_ERR_CUDA; \
        }                                                     \
    } while (0)
