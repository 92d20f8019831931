// Device-side synthetic graphs built straight into device CSR:
//  * R-MAT (Chakrabarti, Zhan & Faloutsos, SDM'04): edge e draws one quadrant per
//    level from Philox4x64-10 at counter (e, level / 2, 3, 0), key (seed, 0) (one
//    64-bit word per level);
//  * Chung-Lu (Chung & Lu, PNAS 2002): expected degrees w_i proportional to
//    (i + i0)^(-1/(gamma-1)), scaled to the requested mean; each of n*mean/2 edge
//    draws picks both endpoints in proportion to w (integer-quantised weights,
//    exact inverse-CDF draws keyed by Philox at counter (e, side, 4, 0)).
// Vertex ids then pass through a seeded bijection so hubs are spread.  The
// symmetrised entries are built in row-range chunks (sort, unique, append), which
// keeps the peak footprint at one chunk of keys plus the final CSR.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>

#include <algorithm>
#include <cmath>
#include <new>

#include "agis_internal.h"
#include "philox.cuh"

namespace agis {
namespace {

constexpr uint64_t kStreamRmat = 3;
constexpr uint64_t kStreamChungLu = 4;

// A bijection of [0, 2^bits): odd multiplies, xor-shifts and adds modulo 2^bits.
struct Scrambler {
    int bits;
    uint64_t mix[3];
    __device__ __forceinline__ uint64_t apply(uint64_t x) const
    {
        const uint64_t mask = (bits >= 64) ? ~0ull : ((1ull << bits) - 1);
        const int sh = (bits + 1) / 2;
        for (int r = 0; r < 3; ++r) {
            x = (x * (mix[r] | 1ull)) & mask;
            x ^= x >> sh;
            x = (x + mix[r]) & mask;
        }
        return x;
    }
    // a bijection of [0, n) for n <= 2^bits, by cycle walking
    __device__ __forceinline__ uint64_t apply_below(uint64_t x, uint64_t n) const
    {
        do {
            x = apply(x);
        } while (x >= n);
        return x;
    }
};

Scrambler make_scrambler(int bits, uint64_t seed)
{
    Scrambler s;
    s.bits = bits;
    s.mix[0] = 0x9E3779B97F4A7C15ull ^ (seed * 0xD1B54A32D192ED03ull);
    s.mix[1] = 0xC2B2AE3D27D4EB4Full ^ (seed * 0x94D049BB133111EBull);
    s.mix[2] = 0x165667B19E3779F9ull ^ (seed * 0xBF58476D1CE4E5B9ull);
    return s;
}

struct RmatSource {
    int scale;
    uint64_t m;              // edge draws
    uint64_t ta, tab, tabc;  // cumulative quadrant thresholds as 64-bit fractions
    uint64_t seed;
    Scrambler perm;
    __device__ __forceinline__ void edge(uint64_t e, uint64_t &u, uint64_t &v) const
    {
        u = 0;
        v = 0;
        uint64_t w0 = 0, w1 = 0;
        for (int level = 0; level < scale; ++level) {
            // level l uses word (l & 1) of the block at counter (e, l >> 1, 3, 0)
            if ((level & 1) == 0) philox4x64_10(e, (uint64_t)(level >> 1), kStreamRmat, 0, seed, 0, w0, w1);
            const uint64_t r = (level & 1) ? w1 : w0;
            const uint64_t bit = 1ull << (scale - 1 - level);
            if (r >= tab) u |= bit;                             // quadrants c, d
            if ((r >= ta && r < tab) || r >= tabc) v |= bit;   // quadrants b, d
        }
        u = perm.apply(u);
        v = perm.apply(v);
    }
};

struct ChungLuSource {
    uint64_t n, m;
    const uint64_t *cum;     // inclusive running sums of the quantised weights
    uint64_t total;
    uint64_t seed;
    Scrambler perm;
    __device__ __forceinline__ uint64_t endpoint(uint64_t e, uint64_t side) const
    {
        const uint64_t r = draw_below(total, e, side, kStreamChungLu, seed);
        uint64_t lo = 0, hi = n - 1;                         // first i with cum[i] > r
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (__ldg(cum + mid) > r) hi = mid; else lo = mid + 1;
        }
        return perm.apply_below(lo, n);
    }
    __device__ __forceinline__ void edge(uint64_t e, uint64_t &u, uint64_t &v) const
    {
        u = endpoint(e, 0);
        v = endpoint(e, 1);
    }
};

// Emits both directions of every non-loop edge whose row falls in [lo, hi).
template <typename Src>
__global__ void k_edge_keys(Src src, uint64_t lo, uint64_t hi, uint64_t *keys, unsigned long long *count,
                            uint64_t cap)
{
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < src.m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t u, v;
        src.edge(e, u, v);
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

template <typename Src>
__global__ void k_edge_count(Src src, uint64_t rows_per_chunk, unsigned long long *per_chunk)
{
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < src.m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t u, v;
        src.edge(e, u, v);
        if (u == v) continue;
        atomicAdd(per_chunk + u / rows_per_chunk, 1ull);
        atomicAdd(per_chunk + v / rows_per_chunk, 1ull);
    }
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

// Chung-Lu weights quantised like the sampler's tables: q_i = floor(w_i / w_0 * 2^K)
// (at least 1) with K chosen so that the sum stays below 2^62 (w_0 is the largest).
__global__ void k_chunglu_weights(uint64_t n, double i0, double alpha, int K, uint64_t *q)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const double rel = pow(((double)i + i0) / i0, -alpha);   // w_i / w_0 in (0, 1]
        const double s = floor(ldexp(rel, K));
        q[i] = s < 1.0 ? 1u : (uint64_t)s;
    }
}

// Builds the symmetrised, deduplicated, loop-free CSR of the edges `src` draws
// over nv vertices.
template <typename Src>
int build_csr(agis_ctx *ctx, const Src &src, uint64_t nv, agis_graph **out)
{
    cudaStream_t st = ctx->stream;
    const int gen_blocks = ctx->sm_count * 8;
    // row chunks small enough that each holds at most 1.5 * 2^30 keys (CUB takes int
    // sizes); every chunk re-draws all edges, so fewer, larger chunks are cheaper
    const uint64_t kChunkKeys = 3ull << 29;
    uint64_t nchunks = 1;
    while ((2 * src.m) / nchunks > kChunkKeys && nchunks < nv) nchunks *= 2;
    std::vector<unsigned long long> per_chunk;
    uint64_t rows_per_chunk = 0;
    for (;;) {
        rows_per_chunk = (nv + nchunks - 1) / nchunks;
        per_chunk.assign(nchunks, 0);
        unsigned long long *d_pc = nullptr;
        AGIS_CUDA_TRY(cudaMalloc(&d_pc, sizeof(unsigned long long) * nchunks));
        cudaMemsetAsync(d_pc, 0, sizeof(unsigned long long) * nchunks, st);
        count_launch();
        k_edge_count<<<gen_blocks, 256, 0, st>>>(src, rows_per_chunk, d_pc);
        cudaMemcpyAsync(per_chunk.data(), d_pc, sizeof(unsigned long long) * nchunks, cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        cudaFree(d_pc);
        if (e != cudaSuccess) return AGIS_ERR_CUDA;
        uint64_t mx = 0;
        for (auto x : per_chunk) mx = std::max<uint64_t>(mx, x);
        if (mx <= kChunkKeys || nchunks >= nv) break;
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
    int key_bits = 1;
    while ((1ull << key_bits) < nv) ++key_bits;
    size_t sort_bytes = 0, uniq_bytes = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, sort_bytes, keys, keys2, (int)std::max<uint64_t>(cap, 1), 0,
                                   32 + key_bits, st);
    cub::DeviceSelect::Unique(nullptr, uniq_bytes, keys2, keys, d_count + 1, (int)std::max<uint64_t>(cap, 1), st);
    if (cudaMalloc(&temp, std::max(sort_bytes, uniq_bytes)) != cudaSuccess) return fail(AGIS_ERR_NOMEM);

    int64_t written = 0;
    for (uint64_t ch = 0; ch < nchunks; ++ch) {
        const uint64_t lo = ch * rows_per_chunk;
        if (lo >= nv) break;
        const uint64_t hi = std::min<uint64_t>(nv, lo + rows_per_chunk);
        cudaMemsetAsync(d_count, 0, 2 * sizeof(unsigned long long), st);
        count_launch();
        k_edge_keys<<<gen_blocks, 256, 0, st>>>(src, lo, hi, keys, d_count, cap);
        unsigned long long n = 0;
        cudaMemcpyAsync(&n, d_count, sizeof(n), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail(AGIS_ERR_CUDA);
        if (n > cap) return fail(AGIS_ERR_CUDA);
        size_t tb = sort_bytes;
        if (cub::DeviceRadixSort::SortKeys(temp, tb, keys, keys2, (int)n, 0, 32 + key_bits, st) != cudaSuccess)
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
    // 16 entries of padding: the sampler's 16-byte row loads may read past the end
    if (cudaMalloc(&g->cols, sizeof(int32_t) * (size_t)(written + 16)) != cudaSuccess) return fail(AGIS_ERR_NOMEM);
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

}  // namespace
}  // namespace agis

using namespace agis;

extern "C" int agis_graph_generate_rmat(agis_ctx *ctx, int scale, int edge_factor, double a, double b, double c,
                                        uint64_t seed, agis_graph **out)
{
    agis::NvtxRange nvtx_range("agis:generate");
    if (!ctx || !out || scale < 1 || scale > 30 || edge_factor < 1 || !(a >= 0 && b >= 0 && c >= 0) ||
        a + b + c > 1.0)
        return AGIS_ERR_ARG;
    *out = nullptr;
    AGIS_CUDA_TRY(cudaSetDevice(ctx->device));
    RmatSource p;
    p.scale = scale;
    p.m = (uint64_t)edge_factor << scale;
    auto frac = [](double x) -> uint64_t { return x >= 1.0 ? ~0ull : (uint64_t)(x * 18446744073709551616.0); };
    p.ta = frac(a);
    p.tab = frac(a + b);
    p.tabc = frac(a + b + c);
    p.seed = seed;
    p.perm = make_scrambler(scale, seed);
    return build_csr(ctx, p, 1ull << scale, out);
}

extern "C" int agis_graph_generate_chunglu(agis_ctx *ctx, int64_t n, double gamma, double mean_degree,
                                           uint64_t seed, agis_graph **out)
{
    agis::NvtxRange nvtx_range("agis:generate");
    if (!ctx || !out || n < 2 || n > INT32_MAX || !(gamma > 1.0) || !(mean_degree > 0.0) ||
        mean_degree >= (double)n)
        return AGIS_ERR_ARG;
    *out = nullptr;
    AGIS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const double alpha = 1.0 / (gamma - 1.0);
    // i0 so that the largest expected degree is at most sqrt(sum of expected degrees);
    // the sum is estimated on a regular sample of the indices
    const int64_t stride = std::max<int64_t>(1, n / 65536);
    double i0 = 1.0;
    for (int it = 0; it < 60; ++it) {
        double sum = 0.0;
        for (int64_t i = 0; i < n; i += stride) sum += std::pow((double)i + i0, -alpha) * (double)stride;
        const double w0 = std::pow(i0, -alpha) * (mean_degree * (double)n / sum);
        if (w0 <= std::sqrt(mean_degree * (double)n)) break;
        i0 *= 2.0;
    }
    int lg = 0;
    while ((1ull << lg) < (uint64_t)(n + 1)) ++lg;
    const int K = 62 - lg;
    uint64_t *q = nullptr, *cum = nullptr;
    AGIS_CUDA_TRY(cudaMalloc(&q, sizeof(uint64_t) * (size_t)n));
    if (cudaMalloc(&cum, sizeof(uint64_t) * (size_t)n) != cudaSuccess) {
        cudaFree(q);
        return AGIS_ERR_NOMEM;
    }
    count_launch();
    k_chunglu_weights<<<ctx->sm_count * 8, 256, 0, st>>>((uint64_t)n, i0, alpha, K, q);
    int rc = inclusive_scan_u64(ctx, q, n, cum);
    uint64_t total = 0;
    if (rc == AGIS_OK && cudaMemcpyAsync(&total, cum + (n - 1), sizeof(uint64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = AGIS_ERR_CUDA;
    if (rc == AGIS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = AGIS_ERR_CUDA;
    cudaFree(q);
    if (rc != AGIS_OK) {
        cudaFree(cum);
        return rc;
    }
    ChungLuSource src;
    src.n = (uint64_t)n;
    src.m = (uint64_t)((double)n * mean_degree / 2.0);
    src.cum = cum;
    src.total = total;
    src.seed = seed;
    int bits = 1;
    while ((1ull << bits) < (uint64_t)n) ++bits;
    src.perm = make_scrambler(bits, seed ^ 0x436875ull);
    rc = build_csr(ctx, src, (uint64_t)n, out);
    cudaFree(cum);
    return rc;
}
