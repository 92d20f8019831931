// The preprocessing cache: a graph's Sec. 4.4 statistics (neighbour-degree sums,
// clustering hits, the probe seed and c_min) and its quantised f_approx weight
// tables (q, the vertex prefix, the full row prefix) written to a file and read back
// into another handle of the same graph, so that a later process skips the
// preprocessing and table builds (System Overview: the preprocessor runs only for a
// graph that has not been preprocessed yet).  A file is tied to its graph by the vertex and
// entry counts and a 64-bit fingerprint of the CSR.  Row prefixes of only the
// highest-degree rows (a memory policy below the full table) are not saved; they
// are rebuilt on demand after a load.  Hub bitmaps are derived from the graph and
// rebuilt at load.
//
// File layout (little-endian): an 8-byte magic "AGISTAB1", then uint32 version (1),
// uint32 table count, int64 nv, int64 nnz, uint64 fingerprint, uint64 probe seed,
// double c_min; nsum (nv uint64) and hits (nv uint32); then per table: int32 cfg[4],
// int32 shift, uint32 flags (bit 0: vertex prefix follows, bit 1: full row prefix
// follows), uint64 total, q (nv uint64), the vertex prefix (nv uint64) and the row
// prefix (nnz uint64) when flagged.
#include <cstdio>
#include <cstring>
#include <memory>

#include "agis_internal.h"

namespace agis {
namespace {

constexpr char kMagic[8] = {'A', 'G', 'I', 'S', 'T', 'A', 'B', '1'};
constexpr uint32_t kVersion = 1;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kOffSalt = 0xD1B54A32D192ED03ull;

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t n_tables;
    int64_t nv, nnz;
    uint64_t fingerprint;
    uint64_t prep_seed;
    double c_min;
};
static_assert(sizeof(FileHeader) == 56, "file header layout");

struct TableHeader {
    int32_t cfg[4];
    int32_t shift;
    uint32_t flags;
    uint64_t total;
};
static_assert(sizeof(TableHeader) == 32, "table header layout");

// SplitMix64's output function (Steele, Lea & Flood, OOPSLA'14).
__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Order-free CSR fingerprint: the wrapping sum over entries i of
// mix64(i * golden XOR cols[i]) plus the sum over v <= nv of
// mix64(v * golden XOR off[v] XOR salt).
__global__ void k_fingerprint(const int64_t *__restrict__ off, const int32_t *__restrict__ cols, int64_t nv,
                              int64_t nnz, unsigned long long *out)
{
    uint64_t s = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride)
        s += mix64(((uint64_t)i * kGolden) ^ (uint64_t)(uint32_t)cols[i]);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= nv; v += stride)
        s += mix64(((uint64_t)v * kGolden) ^ (uint64_t)off[v] ^ kOffSalt);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, (unsigned long long)s);
}

struct FileCloser {
    void operator()(FILE *f) const { if (f) fclose(f); }
};
using File = std::unique_ptr<FILE, FileCloser>;

// Streams `bytes` between a device buffer and a file through a pinned staging buffer.
int device_to_file(FILE *f, const void *dev, size_t bytes, void *stage, size_t stage_bytes, cudaStream_t st)
{
    for (size_t o = 0; o < bytes; o += stage_bytes) {
        const size_t n = std::min(stage_bytes, bytes - o);
        AGIS_CUDA_TRY(cudaMemcpyAsync(stage, (const char *)dev + o, n, cudaMemcpyDeviceToHost, st));
        AGIS_CUDA_TRY(cudaStreamSynchronize(st));
        if (fwrite(stage, 1, n, f) != n) return AGIS_ERR_IO;
    }
    return AGIS_OK;
}

int file_to_device(FILE *f, void *dev, size_t bytes, void *stage, size_t stage_bytes, cudaStream_t st)
{
    for (size_t o = 0; o < bytes; o += stage_bytes) {
        const size_t n = std::min(stage_bytes, bytes - o);
        AGIS_CUDA_TRY(cudaStreamSynchronize(st));
        if (fread(stage, 1, n, f) != n) return AGIS_ERR_IO;
        AGIS_CUDA_TRY(cudaMemcpyAsync((char *)dev + o, stage, n, cudaMemcpyHostToDevice, st));
    }
    return cuda_status(cudaStreamSynchronize(st));
}

struct PinnedStage {
    void *p = nullptr;
    size_t bytes = 0;
    int alloc(size_t b)
    {
        bytes = b;
        return cudaMallocHost(&p, b) == cudaSuccess ? AGIS_OK : AGIS_ERR_NOMEM;
    }
    ~PinnedStage() { if (p) cudaFreeHost(p); }
};

constexpr size_t kStageBytes = 64u << 20;

int read_header(FILE *f, FileHeader *h)
{
    if (fread(h, sizeof(*h), 1, f) != 1) return AGIS_ERR_IO;
    if (std::memcmp(h->magic, kMagic, sizeof(kMagic)) != 0 || h->version != kVersion || h->nv < 0 || h->nnz < 0)
        return AGIS_ERR_IO;
    return AGIS_OK;
}

}  // namespace

int graph_fingerprint(agis_graph *g, uint64_t *out)
{
    cudaStream_t st = g->ctx->stream;
    unsigned long long *d = nullptr;
    AGIS_CUDA_TRY(cudaMallocAsync(&d, sizeof(*d), st));
    AGIS_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(*d), st));
    const int blocks = std::max(1, g->ctx->sm_count * 8);
    count_launch();
    k_fingerprint<<<blocks, 256, 0, st>>>(g->off, g->cols, g->nv, g->nnz, d);
    AGIS_CUDA_TRY(cudaGetLastError());
    unsigned long long h = 0;
    AGIS_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    AGIS_CUDA_TRY(cudaFreeAsync(d, st));
    AGIS_CUDA_TRY(cudaStreamSynchronize(st));
    *out = (uint64_t)h;
    return AGIS_OK;
}

}  // namespace agis

namespace agis {
namespace {

int load_tables_body(agis_graph *g, FILE *f, const FileHeader &h, const PinnedStage &stage, cudaStream_t st)
{
    int rc = AGIS_OK;
    const size_t nv = (size_t)g->nv, nnz = (size_t)g->nnz;
    for (uint32_t k = 0; k < h.n_tables; ++k) {
        TableHeader th;
        if (fread(&th, sizeof(th), 1, f) != 1) return AGIS_ERR_IO;
        WeightTable t;
        std::memcpy(t.cfg, th.cfg, sizeof(t.cfg));
        t.shift = th.shift;
        t.total = th.total;
        const uint64_t key = cfg_key(th.cfg);
        auto &slot = g->tables[key];
        free_table(slot);
        slot = t;
        WeightTable &w = slot;
        AGIS_CUDA_TRY(cudaMalloc(&w.q, sizeof(uint64_t) * std::max<size_t>(nv, 1)));
        w.bytes = sizeof(uint64_t) * nv;
        if ((rc = file_to_device(f, w.q, nv * sizeof(uint64_t), stage.p, stage.bytes, st)) != AGIS_OK) return rc;
        if (th.flags & 1u) {
            AGIS_CUDA_TRY(cudaMalloc(&w.pref, sizeof(uint64_t) * std::max<size_t>(nv, 1)));
            w.bytes += sizeof(uint64_t) * nv;
            if ((rc = file_to_device(f, w.pref, nv * sizeof(uint64_t), stage.p, stage.bytes, st)) != AGIS_OK)
                return rc;
        }
        if (th.flags & 2u) {
            if (rowp_full_fits(g)) {
                AGIS_CUDA_TRY(cudaMalloc(&w.rowp, sizeof(uint64_t) * std::max<size_t>(nnz, 1)));
                w.bytes += sizeof(uint64_t) * nnz;
                if ((rc = file_to_device(f, w.rowp, nnz * sizeof(uint64_t), stage.p, stage.bytes, st)) !=
                    AGIS_OK)
                    return rc;
            } else if (fseeko(f, (off_t)(nnz * sizeof(uint64_t)), SEEK_CUR) != 0) {
                return AGIS_ERR_IO;   // the current policy keeps partial row prefixes: rebuilt on demand
            }
        }
        w.last_use = ++g->use_clock;
    }
    return AGIS_OK;
}

}  // namespace
}  // namespace agis

using namespace agis;

extern "C" int agis_graph_fingerprint(agis_graph *g, uint64_t *fingerprint)
{
    if (!g || !fingerprint) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    return graph_fingerprint(g, fingerprint);
}

extern "C" int agis_tables_file_info(const char *path, int64_t *nv, int64_t *nnz, uint64_t *fingerprint,
                                     int32_t *n_tables)
{
    if (!path) return AGIS_ERR_ARG;
    File f(fopen(path, "rb"));
    if (!f) return AGIS_ERR_IO;
    FileHeader h;
    int rc = read_header(f.get(), &h);
    if (rc != AGIS_OK) return rc;
    if (nv) *nv = h.nv;
    if (nnz) *nnz = h.nnz;
    if (fingerprint) *fingerprint = h.fingerprint;
    if (n_tables) *n_tables = (int32_t)h.n_tables;
    return AGIS_OK;
}

extern "C" int agis_graph_save_tables(agis_graph *g, const char *path)
{
    agis::NvtxRange nvtx_range("agis:save_tables");
    if (!g || !path) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    if (!g->prepped) return AGIS_ERR_STATE;
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    AGIS_CUDA_TRY(cudaStreamSynchronize(st));
    FileHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, sizeof(kMagic));
    h.version = kVersion;
    h.n_tables = (uint32_t)g->tables.size();
    h.nv = g->nv;
    h.nnz = g->nnz;
    int rc = graph_fingerprint(g, &h.fingerprint);
    if (rc != AGIS_OK) return rc;
    h.prep_seed = g->prep_seed;
    h.c_min = g->c_min;
    PinnedStage stage;
    if ((rc = stage.alloc(kStageBytes)) != AGIS_OK) return rc;
    const std::string tmp = std::string(path) + ".tmp";
    {
        File f(fopen(tmp.c_str(), "wb"));
        if (!f) return AGIS_ERR_IO;
        if (fwrite(&h, sizeof(h), 1, f.get()) != 1) return AGIS_ERR_IO;
        const size_t nv = (size_t)g->nv, nnz = (size_t)g->nnz;
        if ((rc = device_to_file(f.get(), g->nsum, nv * sizeof(uint64_t), stage.p, stage.bytes, st)) != AGIS_OK ||
            (rc = device_to_file(f.get(), g->hits, nv * sizeof(uint32_t), stage.p, stage.bytes, st)) != AGIS_OK)
            return rc;
        for (const auto &kv : g->tables) {
            const WeightTable &t = kv.second;
            TableHeader th;
            std::memset(&th, 0, sizeof(th));
            std::memcpy(th.cfg, t.cfg, sizeof(th.cfg));
            th.shift = t.shift;
            th.flags = (t.pref ? 1u : 0u) | ((t.rowp && !t.rowp_partial) ? 2u : 0u);
            th.total = t.total;
            if (fwrite(&th, sizeof(th), 1, f.get()) != 1) return AGIS_ERR_IO;
            if ((rc = device_to_file(f.get(), t.q, nv * sizeof(uint64_t), stage.p, stage.bytes, st)) != AGIS_OK)
                return rc;
            if ((th.flags & 1u) &&
                (rc = device_to_file(f.get(), t.pref, nv * sizeof(uint64_t), stage.p, stage.bytes, st)) != AGIS_OK)
                return rc;
            if ((th.flags & 2u) &&
                (rc = device_to_file(f.get(), t.rowp, nnz * sizeof(uint64_t), stage.p, stage.bytes, st)) != AGIS_OK)
                return rc;
        }
        if (fflush(f.get()) != 0) return AGIS_ERR_IO;
    }
    if (std::rename(tmp.c_str(), path) != 0) return AGIS_ERR_IO;
    return AGIS_OK;
}

extern "C" int agis_graph_load_tables(agis_graph *g, const char *path)
{
    agis::NvtxRange nvtx_range("agis:load_tables");
    if (!g || !path) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    File f(fopen(path, "rb"));
    if (!f) return AGIS_ERR_IO;
    FileHeader h;
    int rc = read_header(f.get(), &h);
    if (rc != AGIS_OK) return rc;
    if (h.nv != g->nv || h.nnz != g->nnz || !(h.c_min > 0.0 && h.c_min <= 1.0)) return AGIS_ERR_GRAPH;
    uint64_t fp = 0;
    if ((rc = graph_fingerprint(g, &fp)) != AGIS_OK) return rc;
    if (fp != h.fingerprint) return AGIS_ERR_GRAPH;
    AGIS_CUDA_TRY(cudaStreamSynchronize(st));
    for (auto &kv : g->tables) free_table(kv.second);
    g->tables.clear();
    g->prepped = false;
    const size_t nv = (size_t)g->nv;
    if (!g->nsum) AGIS_CUDA_TRY(cudaMalloc(&g->nsum, sizeof(uint64_t) * std::max<size_t>(nv, 1)));
    if (!g->hits) AGIS_CUDA_TRY(cudaMalloc(&g->hits, sizeof(uint32_t) * std::max<size_t>(nv, 1)));
    PinnedStage stage;
    if ((rc = stage.alloc(kStageBytes)) != AGIS_OK) return rc;
    if ((rc = file_to_device(f.get(), g->nsum, nv * sizeof(uint64_t), stage.p, stage.bytes, st)) != AGIS_OK ||
        (rc = file_to_device(f.get(), g->hits, nv * sizeof(uint32_t), stage.p, stage.bytes, st)) != AGIS_OK)
        return rc;
    if ((rc = build_hub_bitmaps(g)) != AGIS_OK) return rc;
    g->c_min = h.c_min;
    g->prep_seed = h.prep_seed;
    g->prepped = true;
    rc = load_tables_body(g, f.get(), h, stage, st);
    if (rc != AGIS_OK) {
        // the statistics stay loaded; a table that did not load completely is dropped
        cudaStreamSynchronize(st);
        for (auto &kv : g->tables) free_table(kv.second);
        g->tables.clear();
    }
    g->lb.generation++;
    return rc;
}
