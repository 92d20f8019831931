// Device-side synthetic graphs: R-MAT (Chakrabarti, Zhan & Faloutsos, SDM'04) built
// straight into device CSR.  Edge e draws one quadrant per level from Philox4x64-10
// at counter (e, level / 2, 3, 0), key (seed, 0) (one 64-bit word per level), then
// ids pass through a seeded bijection of [0, 2^scale) so hubs are spread.  The
// symmetrised entries are built in row-range chunks (sort, unique, append), which
// keeps the peak footprint at one chunk of keys plus the final CSR.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>

#include <algorithm>
#include <new>

#include "agis_internal.h"
#include "philox.cuh"

namespace agis {
namespace {

constexpr uint64_t kStreamRmat = 3;
constexpr uint64_t kSentinel = ~0ull;

struct RmatParams {
    int scale;
    uint64_t m;              // edge draws
    uint64_t ta, tab, tabc;  // cumulative quadrant thresholds as 64-bit fractions
    uint64_t seed;
    uint64_t mix[3];         // bijection keys
};

// A bijection of [0, 2^scale): odd multiplies, xor-shifts and adds modulo 2^scale.
__device__ __forceinline__ uint64_t scramble(uint64_t x, const RmatParams &p)
{
    const uint64_t mask = (p.scale >= 64) ? ~0ull : ((1ull << p.scale) - 1);
    const int sh = (p.scale + 1) / 2;
    for (int r = 0; r < 3; ++r) {
        x = (x * (p.mix[r] | 1ull)) & mask;
        x ^= x >> sh;
        x = (x + p.mix[r]) & mask;
    }
    return x;
}

__device__ __forceinline__ void rmat_edge(uint64_t e, const RmatParams &p, uint64_t &u, uint64_t &v)
{
    u = 0;
    v = 0;
    uint64_t w0 = 0, w1 = 0;
    for (int level = 0; level < p.scale; ++level) {
        // level l uses word (l & 1) of the block at counter (e, l >> 1, 3, 0)
        if ((level & 1) == 0) philox4x64_10(e, (uint64_t)(level >> 1), kStreamRmat, 0, p.seed, 0, w0, w1);
        const uint64_t r = (level & 1) ? w1 : w0;
        const uint64_t bit = 1ull << (p.scale - 1 - level);
        if (r >= p.tab) u |= bit;                              // quadrants c, d
        if ((r >= p.ta && r < p.tab) || r >= p.tabc) v |= bit; // quadrants b, d
    }
    u = scramble(u, p);
    v = scramble(v, p);
}

// Emits both directions of every non-loop edge whose row falls in [lo, hi).
__global__ void k_rmat_keys(RmatParams p, uint64_t lo, uint64_t hi, uint64_t *keys,
                            unsigned long long *count, uint64_t cap)
{
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < p.m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t u, v;
        rmat_edge(e, p, u, v);
        if (u == v) continue;
        if (u >= lo && u < hi) {
            const unsigned long long i = atomicAdd(count, 1ull);
            if (i < cap) keys[i] = (u << 32) | v;
        }
        if (v >= lo && v < hi) {
            const unsigned long long i = atomicAdd(count, 1ull);
            if (i < cap) keys[i] = (v << 32) | u;
        }
    }
}

__global__ void k_rmat_count(RmatParams p, uint64_t nchunks, uint64_t rows_per_chunk,
                             unsigned long long *per_chunk)
{
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < p.m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t u, v;
        rmat_edge(e, p, u, v);
        if (u == v) continue;
        atomicAdd(per_chunk + u / rows_per_chunk, 1ull);
        atomicAdd(per_chunk + v / rows_per_chunk, 1ull);
    }
    (void)nchunks;
}

__global__ void k_keys_to_cols(const uint64_t *keys, uint64_t n, int32_t *cols)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        cols[i] = (int32_t)(keys[i] & 0xffffffffull);
}

// off[v] for v in [lo, hi): base + first position of row v in the chunk's sorted keys
__global__ void k_row_offsets(const uint64_t *keys, uint64_t n, uint64_t lo, uint64_t hi, int64_t base,
                              int64_t *off)
{
    for (uint64_t v = lo + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < hi;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t target = v << 32;
        uint64_t a = 0, b = n;
        while (a < b) {
            const uint64_t mid = (a + b) >> 1;
            if (keys[mid] < target) a = mid + 1; else b = mid;
        }
        off[v] = base + (int64_t)a;
    }
}

}  // namespace
}  // namespace agis

using namespace agis;

extern "C" int agis_graph_generate_rmat(agis_ctx *ctx, int scale, int edge_factor, double a, double b, double c,
                                        uint64_t seed, agis_graph **out)
{
    if (!ctx || !out || scale < 1 || scale > 30 || edge_factor < 1 || !(a >= 0 && b >= 0 && c >= 0) ||
        a + b + c > 1.0)
        return AGIS_ERR_ARG;
    *out = nullptr;
    AGIS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    RmatParams p;
    p.scale = scale;
    p.m = (uint64_t)edge_factor << scale;
    auto frac = [](double x) -> uint64_t { return x >= 1.0 ? ~0ull : (uint64_t)(x * 18446744073709551616.0); };
    p.ta = frac(a);
    p.tab = frac(a + b);
    p.tabc = frac(a + b + c);
    p.seed = seed;
    p.mix[0] = 0x9E3779B97F4A7C15ull ^ (seed * 0xD1B54A32D192ED03ull);
    p.mix[1] = 0xC2B2AE3D27D4EB4Full ^ (seed * 0x94D049BB133111EBull);
    p.mix[2] = 0x165667B19E3779F9ull ^ (seed * 0xBF58476D1CE4E5B9ull);
    const uint64_t nv = 1ull << scale;
    const int gen_blocks = ctx->sm_count * 8;

    // row chunks small enough that each holds at most 2^30 keys (CUB's int sizes)
    uint64_t nchunks = 1;
    while ((2 * p.m) / nchunks > (1ull << 30) && nchunks < nv) nchunks *= 2;
    std::vector<unsigned long long> per_chunk;
    uint64_t rows_per_chunk = 0;
    for (;;) {
        rows_per_chunk = nv / nchunks;
        per_chunk.assign(nchunks, 0);
        unsigned long long *d_pc = nullptr;
        AGIS_CUDA_TRY(cudaMalloc(&d_pc, sizeof(unsigned long long) * nchunks));
        cudaMemsetAsync(d_pc, 0, sizeof(unsigned long long) * nchunks, st);
        count_launch();
        k_rmat_count<<<gen_blocks, 256, 0, st>>>(p, nchunks, rows_per_chunk, d_pc);
        cudaMemcpyAsync(per_chunk.data(), d_pc, sizeof(unsigned long long) * nchunks, cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        cudaFree(d_pc);
        if (e != cudaSuccess) return AGIS_ERR_CUDA;
        uint64_t mx = 0;
        for (auto x : per_chunk) mx = std::max<uint64_t>(mx, x);
        if (mx <= (1ull << 30) || nchunks >= nv) break;
        nchunks *= 2;
    }
    uint64_t cap = 0, upper = 0;
    for (auto x : per_chunk) { cap = std::max<uint64_t>(cap, x); upper += x; }
    if (cap >= (1ull << 31)) return AGIS_ERR_NOMEM;

    agis_graph *g = new (std::nothrow) agis_graph();
    if (!g) return AGIS_ERR_NOMEM;
    g->ctx = ctx;
    g->nv = (int64_t)nv;
    uint64_t *keys = nullptr, *keys2 = nullptr;
    unsigned long long *d_count = nullptr;
    void *temp = nullptr;
    int32_t *cols_tmp = nullptr;
    auto fail = [&](int rc) {
        cudaFree(keys); cudaFree(keys2); cudaFree(d_count); cudaFree(temp); cudaFree(cols_tmp);
        cudaFree(g->off); cudaFree(g->cols); delete g;
        return rc;
    };
    if (cudaMalloc(&g->off, sizeof(int64_t) * (nv + 1)) != cudaSuccess) return fail(AGIS_ERR_NOMEM);
    // cols sized to the duplicate-inclusive upper bound, trimmed at the end
    if (cudaMalloc(&cols_tmp, sizeof(int32_t) * std::max<uint64_t>(upper, 1)) != cudaSuccess) return fail(AGIS_ERR_NOMEM);
    if (cudaMalloc(&keys, sizeof(uint64_t) * std::max<uint64_t>(cap, 1)) != cudaSuccess ||
        cudaMalloc(&keys2, sizeof(uint64_t) * std::max<uint64_t>(cap, 1)) != cudaSuccess ||
        cudaMalloc(&d_count, 2 * sizeof(unsigned long long)) != cudaSuccess)
        return fail(AGIS_ERR_NOMEM);
    size_t sort_bytes = 0, uniq_bytes = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, sort_bytes, keys, keys2, (int)std::max<uint64_t>(cap, 1), 0, 32 + scale, st);
    cub::DeviceSelect::Unique(nullptr, uniq_bytes, keys2, keys, d_count + 1, (int)std::max<uint64_t>(cap, 1), st);
    if (cudaMalloc(&temp, std::max(sort_bytes, uniq_bytes)) != cudaSuccess) return fail(AGIS_ERR_NOMEM);

    int64_t written = 0;
    for (uint64_t ch = 0; ch < nchunks; ++ch) {
        const uint64_t lo = ch * rows_per_chunk, hi = (ch + 1 == nchunks) ? nv : lo + rows_per_chunk;
        cudaMemsetAsync(d_count, 0, 2 * sizeof(unsigned long long), st);
        count_launch();
        k_rmat_keys<<<gen_blocks, 256, 0, st>>>(p, lo, hi, keys, d_count, cap);
        unsigned long long n = 0;
        cudaMemcpyAsync(&n, d_count, sizeof(n), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail(AGIS_ERR_CUDA);
        if (n > cap) return fail(AGIS_ERR_CUDA);
        size_t tb = sort_bytes;
        if (cub::DeviceRadixSort::SortKeys(temp, tb, keys, keys2, (int)n, 0, 32 + scale, st) != cudaSuccess)
            return fail(AGIS_ERR_CUDA);
        tb = uniq_bytes;
        if (cub::DeviceSelect::Unique(temp, tb, keys2, keys, d_count + 1, (int)n, st) != cudaSuccess)
            return fail(AGIS_ERR_CUDA);
        unsigned long long u = 0;
        cudaMemcpyAsync(&u, d_count + 1, sizeof(u), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail(AGIS_ERR_CUDA);
        count_launch();
        k_keys_to_cols<<<gen_blocks, 256, 0, st>>>(keys, u, cols_tmp + written);
        count_launch();
        k_row_offsets<<<gen_blocks, 256, 0, st>>>(keys, u, lo, hi, written, g->off);
        written += (int64_t)u;
    }
    cudaMemcpyAsync(g->off + nv, &written, sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(AGIS_ERR_CUDA);
    cudaFree(keys); keys = nullptr;
    cudaFree(keys2); keys2 = nullptr;
    cudaFree(temp); temp = nullptr;
    // trim cols to the exact size
    if (cudaMalloc(&g->cols, sizeof(int32_t) * std::max<int64_t>(written, 1)) != cudaSuccess) return fail(AGIS_ERR_NOMEM);
    if (written > 0 && cudaMemcpyAsync(g->cols, cols_tmp, sizeof(int32_t) * written, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return fail(AGIS_ERR_CUDA);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(AGIS_ERR_CUDA);
    cudaFree(cols_tmp); cols_tmp = nullptr;
    cudaFree(d_count); d_count = nullptr;
    g->nnz = written;
    {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) g->rowp_budget = total_b / 4;
    }
    // max degree from the offsets
    {
        std::vector<int64_t> h(nv + 1);
        if (cudaMemcpy(h.data(), g->off, sizeof(int64_t) * (nv + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(AGIS_ERR_CUDA);
        int64_t m = 0;
        for (uint64_t v = 0; v < nv; ++v) m = std::max(m, h[v + 1] - h[v]);
        g->max_deg = m;
    }
    ctx_retain(ctx);
    *out = g;
    return AGIS_OK;
}
