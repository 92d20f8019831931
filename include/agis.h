/*
 * agis.h -- C ABI of the B300 (sm_103a) implementation of AGIS's approximate
 * graph-pattern counting (Lee & Lee, "AGIS: Fast Approximate Graph Pattern Mining
 * with Structure-Informed Sampling", PVLDB 19(2), arXiv 2601.01388).
 *
 * The problem (Sec. 2.1): given an undirected data graph G, a pattern P, an error
 * bound eps and a confidence 1 - delta, return a (1 +- eps) estimate of C(G,P), the
 * number of embeddings (injective maps V_P -> V_G that keep every pattern edge;
 * automorphic copies are counted separately).  The estimate is the mean of
 * independent sampler outputs of Alg. 3 (structure-informed neighbour sampling),
 * each the inverse probability of its trajectory or 0, stopped by Alg. 1.
 *
 * Conventions for every call:
 *   - The return value is an agis_status; nothing else signals errors, and no C++
 *     exception or abort crosses this boundary.
 *   - Handles (agis_ctx, agis_graph, agis_pattern, agis_server) are owned by the
 *     library and released by the matching _destroy / _free call.
 *   - Input arrays are copied before the call returns; output arrays are owned by
 *     the caller and must hold the stated number of elements.
 *   - "device" pointers are CUDA global-memory addresses of the context's device;
 *     "host" pointers are ordinary (pageable or pinned) host memory.
 *   - The graph is undirected and stored in CSR with both directions: int64 row
 *     offsets off[nv+1] (off[0] = 0, non-decreasing) and int32 column ids
 *     cols[nnz]; every row is sorted strictly ascending, has no self-loop, and every
 *     entry (u, v) has its reverse (v, u) (Sec. 2: both graphs undirected).
 *   - Patterns have 2..8 vertices, are connected (Alg. 2 grows the order along
 *     edges) and have no self-loops or repeated edges.
 *   - One agis_ctx may be used from one host thread at a time; an agis_server is
 *     internally synchronised.
 */
#ifndef AGIS_H
#define AGIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AGIS_OK = 0,
    AGIS_ERR_ARG = -1,      /* a null handle/pointer or an out-of-range argument      */
    AGIS_ERR_NOMEM = -2,    /* device or host allocation failed                         */
    AGIS_ERR_CUDA = -3,     /* a CUDA runtime call failed (no device, launch error ...) */
    AGIS_ERR_GRAPH = -4,    /* CSR violates the conventions above                       */
    AGIS_ERR_PATTERN = -5,  /* pattern violates the conventions above                   */
    AGIS_ERR_TIMEOUT = -6,  /* reserved: no device loop of this library waits on another agent */
    AGIS_ERR_BUSY = -7,     /* server: result not ready yet, or admission refused       */
    AGIS_ERR_STATE = -8,    /* call not valid in the handle's current state             */
    AGIS_ERR_IO = -9        /* a file could not be read or written, or is not a table file */
} agis_status;

/* Distribution per step: AUTO = the decision function D^pi with threshold beta
 * (Def. decision function); APPROX = f_approx at every step (beta = -inf in the
 * Sec. 6 beta sweep); UNIFORM = f_uniform at every step (beta = +inf, which is
 * ScaleGPM's NS-prune without symmetry breaking, Sec. 5.3). */
typedef enum { AGIS_MODE_AUTO = 0, AGIS_MODE_APPROX = 1, AGIS_MODE_UNIFORM = 2 } agis_mode;

typedef struct agis_ctx agis_ctx;
typedef struct agis_graph agis_graph;
typedef struct agis_pattern agis_pattern;
typedef struct agis_server agis_server;

/* Per-query options.  agis_default_opts fills eps = 0.1, delta = 0.01 (the paper's
 * defaults, Sec. 6.1), beta = 0.8 (Def. decision function), mode AUTO, seed 1,
 * chunk_trials = 65536, min_trials = 65536, max_trials = 2^32. */
typedef struct {
    double eps;             /* target relative error of Alg. 1                         */
    double delta;           /* 1 - confidence; z = Phi^{-1}(1 - delta/2)               */
    double beta;            /* decision threshold (AUTO mode)                          */
    int32_t mode;           /* agis_mode                                               */
    int32_t terms;          /* factors of Eq. probability_function kept: bit 0 T[F1],
                               bit 1 T[I1], bit 2 T[F2]; 0 = all (the method).  1, 3, 5
                               give the incremental versions of the Sec. 6.2 ablation;
                               T[F1] must be kept (else ARG)                           */
    uint64_t seed;          /* Philox key of this query's trials                       */
    uint64_t min_trials;    /* Alg. 1 is not consulted before this many trials         */
    uint64_t max_trials;    /* hard budget; with eps <= 0 exactly this many run        */
    uint64_t chunk_trials;  /* checkpoint spacing for Alg. 1; multiple of 1024         */
    int32_t anchor;         /* 1: a step with several backward vertices draws from the
                               shortest backward row (minus tau) with the step's weights
                               and the trial fails unless the drawn vertex closes every
                               other backward edge, instead of building S_tau (Alg. 3);
                               still unbiased by Thm. 2.  0 (default): S_tau as in Alg. 3 */
    int32_t reserved;       /* must be 0                                               */
} agis_opts;

/* Words of one tile's output in agis_sample_device: hits, sectors, the FP64 sum X
 * and sum X^2 bit patterns, sectors_streamed, sectors_survey (see agis_result). */
#define AGIS_TILE_WORDS 6

typedef struct {
    double estimate;        /* mean sampler output = estimate of C(G,P) (embeddings)    */
    double subgraphs;       /* estimate / |Aut(P)|                                      */
    double mean, var;       /* Alg. 1: mu and population sigma^2 of the outputs         */
    double eps_hat;         /* Alg. 1 estimated relative error at the stopping point    */
    double sum_x, sum_x2;   /* FP64 sums over the trials used                           */
    uint64_t trials;        /* trials used (a multiple of chunk_trials unless capped)   */
    uint64_t hits;          /* successful trajectories among them                       */
    uint64_t sectors;       /* algorithmic 32-byte sectors of those trials (the cost
                               model: the sectors Alg. 3 must touch with no reuse)     */
    int32_t converged;      /* 1 if Alg. 1 accepted eps at a checkpoint                 */
    int32_t launches;       /* sampler kernel launches used                             */
    double t_prep_s;        /* weight-table builds done for this call                  */
    double t_sample_s;      /* wall time of the sampling loop                           */
    uint64_t sectors_streamed; /* the part of `sectors` read as consecutive runs: scans
                               of the shortest backward row and rows read once by a
                               merge; the rest are random accesses                      */
    uint64_t sectors_survey;   /* the plain count: one membership search per scanned
                               entry in every other backward row, and weight reads on
                               every step D(i) puts under f_approx                       */
} agis_result;

const char *agis_status_str(int status);
void agis_default_opts(agis_opts *opts);

/* ---- context -------------------------------------------------------------
 * agis_create: binds CUDA device `device` and the CUDA stream `cuda_stream`
 * (a cudaStream_t; NULL = the library's own non-blocking stream).  Every kernel
 * of this context runs on that stream.  Errors: ARG (out is NULL), CUDA. */
int agis_create(int device, void *cuda_stream, agis_ctx **out);
int agis_destroy(agis_ctx *ctx);

/* ---- graph ---------------------------------------------------------------
 * agis_graph_load_csr: copies a CSR graph to the device (Sec. 5.4 "the graph is
 * read and loaded in CSR format").  offsets: nv+1 entries, int64 if
 * offsets_are_64bit else int32; cols: nnz int32 entries.  on_device = 1 means both
 * pointers are device addresses of ctx's device, 0 means host memory.  validate = 1
 * checks the CSR conventions on the device and returns GRAPH on a violation.
 * The graph keeps a reference to ctx; free the graph before the ctx.
 * Errors: ARG, NOMEM, CUDA, GRAPH. */
int agis_graph_load_csr(agis_ctx *ctx, const void *offsets, int offsets_are_64bit,
                        const int32_t *cols, int64_t nv, int64_t nnz, int on_device,
                        int validate, agis_graph **out);

/* agis_graph_preprocess: Sec. 4.4 -- for every vertex v the neighbour-degree sum
 * nsum(v) = sum_{x in N(v)} d(x) (numerator of the average neighbour degree) and the
 * sampled clustering coefficient C_v = max(c_min, hits(v)/d(v)) from d(v) probes of
 * uniform ordered distinct neighbour pairs, probe j of v keyed by Philox4x64-10
 * counter (v, j, 2, 0) and key (seed, 0); d(v) < 2 gives c_min.  Must precede any
 * estimate; calling it again with new values drops cached weight tables.
 * Errors: ARG (c_min outside (0, 1]), NOMEM, CUDA. */
int agis_graph_preprocess(agis_graph *g, uint64_t seed, double c_min);

/* agis_graph_info: nv, nnz (directed entries), max degree, device bytes held. */
int agis_graph_info(const agis_graph *g, int64_t *nv, int64_t *nnz, int64_t *max_degree,
                    uint64_t *device_bytes);

/* agis_graph_stats_copy: copies nsum (uint64[nv]) and hits (uint32[nv]) of the last
 * preprocess to caller-owned host arrays (either may be NULL).  Errors: ARG, STATE. */
int agis_graph_stats_copy(const agis_graph *g, uint64_t *nsum, uint32_t *hits);

/* agis_graph_weight_table: builds (or reuses) the quantised f_approx weight table
 * of step configuration cfg = (|B|, |F1|, |I_eff|, |F2|) (Eq. probability_function)
 * and copies it out: q[nv] uint64 weights, prefix[nv] uint64 inclusive running sums
 * over v (either may be NULL), *shift = the power-of-two scale applied before
 * flooring.  Used to check the tables bit for bit.  Errors: ARG, STATE, NOMEM, CUDA. */
int agis_graph_weight_table(agis_graph *g, const int32_t cfg[4], uint64_t *q,
                            uint64_t *prefix, int32_t *shift);

/* agis_graph_row_prefix: copies the per-row inclusive running sums of q over each
 * row's neighbours for configuration cfg (nnz uint64, caller-owned host array).
 * STATE when the memory policy only allows a partial table. */
int agis_graph_row_prefix(agis_graph *g, const int32_t cfg[4], uint64_t *row_prefix);

/* agis_graph_validate: re-checks the CSR conventions above on the device (e.g. for a
 * generated graph); on an oriented graph (agis_graph_orient) the reverse of every
 * entry must be absent instead of present.  Returns OK or GRAPH. */
int agis_graph_validate(agis_graph *g);

/* agis_graph_copy_csr: copies the device CSR to caller-owned host arrays off[nv+1]
 * (int64) and cols[nnz] (int32); either may be NULL. */
int agis_graph_copy_csr(const agis_graph *g, int64_t *off, int32_t *cols);

/* agis_graph_orient: the degree-ordered orientation that Sec. 5.4 applies to clique
 * patterns (the graph turned into a DAG by dropping every edge that points from a
 * higher- to a lower-degree vertex).  Row u of *out keeps v when (d(u), u) < (d(v), v)
 * lexicographically, degrees taken in g, in g's ascending order; so each k-clique is
 * exactly one chain v1 -> ... -> vk with every later vertex in the out-rows of all
 * earlier ones, and a row holds at most about sqrt(2|E|) entries.  *out is a new
 * device graph with half of g's entries and g's memory policy; it needs
 * agis_graph_preprocess (the Sec. 4.4 statistics over out-rows) and agis_graph_free,
 * and g stays valid.  Queries on it take clique patterns only (others: PATTERN); their
 * f_approx weight uses |B| = 0 in T[F1] (no earlier vertex is in a later one's
 * out-row), and results report estimate = cliques * k! (embeddings, as on g) and
 * subgraphs = cliques, with mean/var/sum_x the per-trial moments (cliques).
 * Errors: ARG, STATE (g is itself oriented), NOMEM, CUDA. */
int agis_graph_orient(agis_graph *g, agis_graph **out);

/* agis_graph_is_oriented: 1 for a graph made by agis_graph_orient, 0 for a loaded
 * or generated one, ARG for NULL. */
int agis_graph_is_oriented(const agis_graph *g);

/* agis_graph_set_memory_policy: device-memory budgets of the optional structures
 * that speed up sampling (0 keeps a setting): row_prefix_bytes -- the largest
 * per-configuration row-prefix table built in full (default a quarter of device
 * memory); past it only the highest-degree rows that fit get a prefix and the
 * other single-backward draws scan their row; bitmap_bytes -- total for hub
 * neighbour bitmaps (default a sixteenth), built for vertices of degree at least
 * bitmap_min_degree (default 1024) at the next agis_graph_preprocess;
 * list_entries (>= 64) -- per-warp candidate-list capacity (default 65536), whose
 * overflow makes a step take the list-free scan.  Results never depend on these
 * settings.  Cached weight tables not in use are dropped.  Errors: ARG. */
int agis_graph_set_memory_policy(agis_graph *g, uint64_t row_prefix_bytes, uint64_t bitmap_bytes,
                                 int64_t bitmap_min_degree, uint32_t list_entries);

/* agis_graph_set_l2_window: bytes of g's hub neighbour bitmaps that sampler launches
 * on g mark as persisting in L2 (a CUDA access-policy window over the bitmaps, which
 * are laid out in decreasing degree order, so the window holds the most probed
 * ones); default 48 MiB, limited by the device's largest window and persisting
 * set-aside (79 MiB on a B300); 0 turns the window off.  The first windowed launch
 * raises the context's persisting-L2 set-aside to the window's size, which leaves
 * other kernels of the process that much less L2 while the agis_ctx lives; its
 * release restores the previous set-aside.  No effect without hub bitmaps.
 * Results never depend on this setting.  Errors: ARG (NULL). */
int agis_graph_set_l2_window(agis_graph *g, uint64_t bytes);

/* ---- preprocessing cache ---------------------------------------------------
 * The System Overview runs the preprocessor only for a graph that has not been
 * preprocessed yet; these calls keep that work across processes.
 * agis_graph_save_tables: writes the graph's Sec. 4.4 statistics (nsum, hits, the
 * probe seed and c_min of the last agis_graph_preprocess) and every cached f_approx
 * weight table (q, the vertex prefix, the full row prefix; a row prefix of only the
 * highest-degree rows is left out) to the file `path` (written to path.tmp, then
 * renamed).  Layout: the magic "AGISTAB1", uint32 version 1, uint32 table count,
 * int64 nv, int64 nnz, uint64 fingerprint (agis_graph_fingerprint), uint64 seed,
 * double c_min, nsum[nv] uint64, hits[nv] uint32, then per table int32 cfg[4], int32
 * shift, uint32 flags (bit 0 vertex prefix, bit 1 row prefix), uint64 total, q[nv],
 * then prefix[nv] and row_prefix[nnz] as flagged; all little-endian uint64 arrays.
 * Errors: ARG, STATE (not preprocessed), NOMEM, CUDA, IO. */
int agis_graph_save_tables(agis_graph *g, const char *path);

/* agis_graph_load_tables: reads such a file into g, which must hold the same CSR
 * (same nv, nnz and fingerprint, else GRAPH and g is unchanged): the statistics
 * replace any earlier preprocessing (hub bitmaps are rebuilt from the graph), cached
 * tables are replaced by the file's, and estimates then give exactly the results of
 * the graph the file was saved from.  A saved row prefix that the current memory
 * policy does not allow in full is skipped (rebuilt on demand as a partial one).  If
 * a table cannot be read the statistics stay loaded and no table is kept.
 * Errors: ARG, GRAPH, NOMEM, CUDA, IO. */
int agis_graph_load_tables(agis_graph *g, const char *path);

/* agis_graph_fingerprint: the 64-bit CSR fingerprint that ties a table file to its
 * graph: the wrapping sum over entries i < nnz of m(i * G XOR cols[i]) plus the sum
 * over v <= nv of m(v * G XOR off[v] XOR S), with m SplitMix64's output function,
 * G = 0x9E3779B97F4A7C15 and S = 0xD1B54A32D192ED03 (uint64 arithmetic, cols[i]
 * taken as an unsigned 32-bit value).  Errors: ARG, CUDA. */
int agis_graph_fingerprint(agis_graph *g, uint64_t *fingerprint);

/* agis_tables_file_info: reads only the header of a table file (host only, no
 * device needed).  Any output pointer may be NULL.  Errors: ARG, IO. */
int agis_tables_file_info(const char *path, int64_t *nv, int64_t *nnz, uint64_t *fingerprint,
                          int32_t *n_tables);

/* agis_graph_drop_tables: frees every cached weight table (they are rebuilt on
 * demand). */
int agis_graph_drop_tables(agis_graph *g);
int agis_graph_free(agis_graph *g);

/* ---- synthetic graphs on the device ---------------------------------------
 * agis_graph_generate_rmat: R-MAT (Chakrabarti et al., SDM'04) with 2^scale
 * vertices and edge_factor * 2^scale edge draws, quadrant probabilities (a, b, c,
 * 1-a-b-c), symmetrised, self-loops and duplicates removed, ids permuted by a
 * seeded bijection; built on the device in chunks.  Errors: ARG, NOMEM, CUDA. */
int agis_graph_generate_rmat(agis_ctx *ctx, int scale, int edge_factor, double a, double b,
                             double c, uint64_t seed, agis_graph **out);

/* agis_graph_generate_chunglu: Chung-Lu graph (Chung & Lu, PNAS 2002) on n
 * vertices with expected degrees proportional to (i + i0)^(-1/(gamma-1)), scaled
 * to mean_degree (i0 keeps the largest below sqrt(n * mean_degree)); n*mean/2
 * edge draws with both endpoints drawn in proportion to the weights, symmetrised,
 * loops and duplicates removed, ids permuted by a seeded bijection; built on the
 * device.  Errors: ARG, NOMEM, CUDA. */
int agis_graph_generate_chunglu(agis_ctx *ctx, int64_t n, double gamma, double mean_degree,
                                uint64_t seed, agis_graph **out);

/* ---- pattern -------------------------------------------------------------
 * agis_pattern_create: k vertices (2..8), ne undirected edges as pairs
 * edge_pairs[2*ne] (host).  Computes the matching order pi (Alg. 2, ties to the
 * smallest id), the auxiliary arrays B, F1, I_eff, F2 per step (Def. auxiliary
 * arrays), Certainty per step (Def. decision function, E^{>=2hop} over E_P) and
 * |Aut(P)|.  Errors: ARG, PATTERN. */
int agis_pattern_create(int k, int ne, const int32_t *edge_pairs, agis_pattern **out);

/* agis_pattern_info: order[8] (pattern vertex of step i), cfg[8][4] = (|B|, |F1|,
 * |I_eff|, |F2|) per step, certainty[8], back[8] = bitmask over earlier steps of the
 * backward neighbours, *automorphisms = |Aut(P)|.  Entries past k are zero.  Any
 * output pointer may be NULL. */
int agis_pattern_info(const agis_pattern *p, int32_t *k, int32_t order[8], int32_t cfg[8][4],
                      double certainty[8], uint8_t back[8], uint64_t *automorphisms);

/* agis_pattern_decide: D^pi per step for (mode, beta) into use_approx[8]. */
int agis_pattern_decide(const agis_pattern *p, int32_t mode, double beta, uint8_t use_approx[8]);
int agis_pattern_free(agis_pattern *p);

/* ---- estimation ------------------------------------------------------------
 * agis_estimate: one query, plain per-query launches.  Runs Alg. 3 trials
 * 0, 1, 2, ... (trial t draws step i from Philox4x64-10 counter (t, i, 1, 0), key
 * (seed, 0)) in tiles of agis_tile_trials() trials on the device, and evaluates Alg. 1 on host at every
 * chunk_trials checkpoint once min_trials trials are in.  The result is that of the
 * first converged checkpoint, or of max_trials; it is a deterministic function of
 * (graph, pattern, opts).  eps <= 0 runs exactly max_trials trials.
 * Errors: ARG, STATE (graph not preprocessed), NOMEM, CUDA. */
int agis_estimate(agis_graph *g, const agis_pattern *p, const agis_opts *opts,
                  agis_result *out);

/* agis_estimate_batch: n queries (patterns[i], opts[i]) in one replayed CUDA graph
 * per epoch: a persistent, work-stealing sampler launch, with the epoch's last
 * tiles (all of a short epoch) on a launch where every warp takes single trials;
 * tiles of all unconverged queries share each epoch.  Each out[i] equals what
 * agis_estimate(g, patterns[i], &opts[i]) returns.  Errors: as agis_estimate. */
int agis_estimate_batch(agis_graph *g, int n, const agis_pattern *const *patterns,
                        const agis_opts *opts, agis_result *out);

/* agis_dump_trials: per-trial record of trials [first, first+count) of the query:
 * emb[count*8] int32 trajectory (step order; -1 after a failed step), hit[count]
 * (1 = the trajectory is an embedding), x[count] FP64 sampler output (Alg. 3:
 * 1/p or 0), sectors[count*3] the trial's sector counts (sectors, sectors_streamed,
 * sectors_survey as in agis_result).  Host arrays; any may be NULL.
 * Errors: ARG, STATE, NOMEM, CUDA. */
int agis_dump_trials(agis_graph *g, const agis_pattern *p, const agis_opts *opts,
                     uint64_t first, uint64_t count, int32_t *emb, uint8_t *hit, double *x,
                     uint64_t *sectors);

/* agis_tile_trials: trials per tile, the unit of work and of the fixed-order FP64
 * reduction (a power of two dividing 1024; set when the library is built). */
int agis_tile_trials(void);

/* agis_sample_device: fixed-budget sampling with all buffers on the device:
 * trials [first, first + ntiles*T) of the query, T = agis_tile_trials(), per-tile sums written to
 * tile_out (device, AGIS_TILE_WORDS uint64 words per tile: hits, sectors, the FP64
 * sum X and sum X^2 bit patterns, sectors_streamed, sectors_survey).  Enqueued on
 * ctx's stream, no host sync.
 * Errors: ARG, STATE, NOMEM, CUDA. */
int agis_sample_device(agis_graph *g, const agis_pattern *p, const agis_opts *opts,
                       uint64_t first, uint64_t ntiles, uint64_t *tile_out);

/* agis_autotune: picks the sampler's launch shape for this graph and query mix --
 * resident CTAs per SM (1 up to the occupancy limit) and tiles per work item (1, 2
 * or 4 tiles of agis_tile_trials() trials each) -- by timing a fixed budget of
 * trials_per_query trials of every query at each pair (CUDA events on the
 * context's stream), and keeps the fastest in the context for later launches.
 * Short epochs still split into single tiles so that every SM gets work.  Results
 * never depend on the choice: tiles and their fixed-order sums stay the same.
 * *blocks_per_sm and *tiles_per_item (either may be NULL) receive the choice.
 * Errors: ARG, STATE, NOMEM, CUDA. */
int agis_autotune(agis_graph *g, int n, const agis_pattern *const *patterns, const agis_opts *opts,
                  uint64_t trials_per_query, int32_t *blocks_per_sm, int32_t *tiles_per_item);

/* agis_prepare: builds, for the query's f_approx steps, the quantised weight tables
 * of Eq. probability_function and their prefix sums (Sec. 4.4 / Sec. 5.1: f_approx
 * needs the per-vertex weights of every candidate); later calls reuse them.  Blocks
 * until the tables are ready.  Errors: ARG, STATE, NOMEM, CUDA. */
int agis_prepare(agis_graph *g, const agis_pattern *p, const agis_opts *opts);

/* agis_prefix_sum_u64_noalloc: out[i] = in[0] + ... + in[i] for i < n (uint64,
 * wrapping), the same scan that builds the weight tables' prefix sums, for callers
 * that cannot call cudaMalloc: a custom device allocator or memory-pool hook that
 * must not re-enter the CUDA allocator, a service whose device memory a pool already
 * holds in full, or latency-critical code that avoids cudaMalloc because it can
 * block and synchronise the device.  The paper has no counterpart; this is a
 * library service.
 * in and out are device pointers of the context current on the calling thread
 * (they may not overlap); the work is enqueued on cuda_stream (NULL = legacy default
 * stream) and nothing is allocated or freed: the tile-sum scratch is a file-scope
 * device array of 65536 uint64 (512 KiB), held by every device that loads the
 * library until the process exits.  So n is at most 65536 * 2048 = 134217728;
 * larger n returns ARG.
 * The first call in a CUDA context looks up the array's device address (once per
 * context; a reset device or another context is looked up again); make that first
 * call before any stream capture.  All calls share the one array, which keeps the
 * last call's tile sums (each call writes every entry it reads first): calls whose
 * work overlaps on the GPU (other streams, or other host threads) race on it and
 * must be serialised by the caller.  A launch error, or an error still pending from
 * earlier work on this thread, is returned as CUDA.
 * Errors: ARG (n < 0, n too large, null pointer), CUDA. */
int agis_prefix_sum_u64_noalloc(const uint64_t *in, int64_t n, uint64_t *out, void *cuda_stream);

/* agis_probe_random_read: enqueues (on cuda_stream) about `reads` independent reads,
 * each of the first 8 bytes of a random 32-byte sector among the first 2^k sectors
 * of the device buffer buf (bytes long, 2^k*32 <= bytes; choose it far larger than L2), as a measure of the random-access
 * bandwidth that bounds the sampler's gathers and searches (the roofline of
 * Alg. 3's memory pattern).  The exact count issued is a multiple of
 * 8 * 2048 * (number of SMs) >= reads; sink is a device uint64 the kernel may
 * write.  Time it with events on the same stream.  Errors: ARG, CUDA. */
int agis_probe_random_read(const void *buf, uint64_t bytes, uint64_t reads, uint64_t seed,
                           void *cuda_stream, void *sink);

/* agis_step_timers: reads (and with reset != 0 clears) the sampler's per-step-kind
 * cycle counters of the current device: out16[2k] = summed SM cycles, out16[2k+1]
 * = number of steps, for kinds k = 0 step 1, 1 single-backward search, 2 listed
 * intersection, 3 listed reuse of the previous list, 4 list-free scan.  They are
 * only counted in a build with -DAGIS_STEP_TIMERS (zeros otherwise).  A profiling
 * aid.  Errors: ARG, CUDA. */
int agis_step_timers(uint64_t *out16, int reset);

/* agis_kernel_launches: number of this library's CUDA kernel launches so far in
 * the process (all contexts); a diagnostic for counting device work. */
uint64_t agis_kernel_launches(void);

/* agis_z_of_delta: Phi^{-1}(1 - delta/2) as Alg. 1 uses it. */
double agis_z_of_delta(double delta);

/* ---- serving -------------------------------------------------------------
 * A server keeps the graph resident and runs a scheduler thread that admits
 * queries while a slot is free and their weight tables fit in scratch_bytes of
 * device memory, runs all admitted queries together in epochs (each epoch one
 * replayed CUDA graph over every admitted query's next tiles), retires queries at
 * their first converged checkpoint and admits waiting ones as slots and memory
 * free up (continuous batching).  Two epochs are in flight at a time: the next one
 * is staged and enqueued while the current one runs, so queries that arrive while
 * others are on the GPU join the next epoch and their work overlaps.  Results
 * equal agis_estimate's.  The server allocates its own launch buffers and one
 * candidate-list scratch (as large as an estimate call's) on the graph's device. */
int agis_server_create(agis_graph *g, size_t scratch_bytes, int max_slots, agis_server **out);
/* agis_server_submit: copies the pattern and options; *ticket identifies the query.
 * Errors: ARG, BUSY (more than 65536 queries waiting). */
int agis_server_submit(agis_server *s, const agis_pattern *p, const agis_opts *opts,
                       uint64_t *ticket);
/* agis_server_poll: AGIS_OK and *out filled when done (the ticket is then
 * released), AGIS_ERR_BUSY while queued or running, ARG for an unknown ticket, or
 * the query's own error status.  latency_s (may be NULL) = completion - submit.
 * epochs (may be NULL; 2 entries) = the index of the first epoch that ran tiles of
 * this query and of the epoch whose sums finished it (epochs are numbered from 0
 * in launch order): two queries whose ranges overlap shared the GPU. */
int agis_server_poll(agis_server *s, uint64_t ticket, agis_result *out, double *latency_s,
                     uint64_t *epochs);
/* agis_server_stats: queries completed, epochs completed, peak admitted slots,
 * gpu_busy_s = summed device time of the epochs (events around each launch) and
 * busy_span_s = wall time during which at least one epoch was in flight; their
 * ratio is the fraction of that time the GPU was not idle.  Any pointer may be
 * NULL. */
int agis_server_stats(agis_server *s, uint64_t *completed, uint64_t *epochs, int32_t *peak_slots,
                      double *gpu_busy_s, double *busy_span_s);
int agis_server_destroy(agis_server *s);

#ifdef __cplusplus
}
#endif
#endif /* AGIS_H */
