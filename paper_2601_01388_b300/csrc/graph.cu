// Device graph: CSR ingest and validation, Sec. 4.4 preprocessing (neighbour-degree
// sums and sampled clustering coefficients), and the per-step-configuration weight
// tables of Eq. probability_function with their prefix sums.
#include <algorithm>
#include <cmath>
#include <functional>
#include <cstring>
#include <new>

#include "agis_internal.h"
#include "philox.cuh"

namespace agis {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int64_t row_find(const int32_t *row, int64_t d, int32_t x)
{
    // last position with row[pos] <= x; the number of probes depends on d only
    if (d <= 0) return -1;
    int64_t lo = 0, len = d;
    while (len > 1) {
        const int64_t half = len >> 1;
        if (__ldg(row + lo + half) <= x) lo += half;
        len -= half;
    }
    return __ldg(row + lo) == x ? lo : -1;
}

// ---------------------------------------------------------------- validation

__global__ void k_check_offsets(const int64_t *off, int64_t nv, int64_t nnz, int *err)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = off[v];
        bool bad = (v == 0 && o != 0) || (v == nv && o != nnz) || o < 0 || o > nnz;
        if (v < nv && off[v + 1] < o) bad = true;
        if (bad) atomicOr(err, 1);
    }
}

// one warp per row: range, self-loop, strict order, and the reverse entry present
// (undirected graph) or absent (oriented graph)
__global__ void k_check_rows(const int64_t *off, const int32_t *cols, int64_t nv, int oriented, int *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < nv; v += nwarps) {
        const int64_t s = off[v], e = off[v + 1];
        for (int64_t i = s + lane; i < e; i += 32) {
            const int32_t x = cols[i];
            bool bad = x < 0 || x >= nv || x == v || (i > s && cols[i - 1] >= x);
            if (!bad) bad = (row_find(cols + off[x], off[x + 1] - off[x], (int32_t)v) < 0) != (oriented != 0);
            if (bad) atomicOr(err, 2);
        }
    }
}

// ---------------------------------------------------------------- Sec. 4.4

// nsum(v) = sum of d(x) over the neighbours x of v; one warp per vertex
__global__ void k_neighbour_degree_sum(const int64_t *off, const int32_t *cols, int64_t nv,
                                       uint64_t *nsum)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < nv; v += nwarps) {
        const int64_t s = off[v], e = off[v + 1];
        uint64_t acc = 0;
        for (int64_t i = s + lane; i < e; i += 32) {
            const int32_t x = __ldg(cols + i);
            acc += (uint64_t)(__ldg(off + x + 1) - __ldg(off + x));
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) nsum[v] = acc;
    }
}

// hits(v): probe j of v draws r in [0, d(d-1)), names the ordered distinct pair
// a = r / (d-1), b = r mod (d-1) (+1 if >= a) of row positions, and hits when the
// two neighbours are adjacent.  One warp per vertex, lanes over probes.
__global__ void k_cluster_hits(const int64_t *off, const int32_t *cols, int64_t nv, uint64_t seed,
                               uint32_t *hits)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < nv; v += nwarps) {
        const int64_t s = off[v];
        const int64_t d = off[v + 1] - s;
        uint32_t h = 0;
        if (d >= 2) {
            const uint64_t dm1 = (uint64_t)(d - 1);
            for (int64_t j = lane; j < d; j += 32) {
                const uint64_t r = draw_below((uint64_t)d * dm1, (uint64_t)v, (uint64_t)j, kStreamCC, seed);
                const uint64_t a = r / dm1, bp = r - a * dm1;
                const uint64_t b = bp + (bp >= a ? 1u : 0u);
                const int32_t x = __ldg(cols + s + (int64_t)a), y = __ldg(cols + s + (int64_t)b);
                h += row_find(cols + __ldg(off + x), __ldg(off + x + 1) - __ldg(off + x), y) >= 0;
            }
        }
        for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(kFull, h, o);
        if (lane == 0) hits[v] = h;
    }
}

// Neighbour bitmap of hub h (one CTA per hub): bit x set iff x is a neighbour.
__global__ void k_hub_bitmaps(const int64_t *off, const int32_t *cols, const int32_t *hubs,
                              int64_t words, uint32_t *bits)
{
    const int32_t v = hubs[blockIdx.x];
    uint32_t *bm = bits + (int64_t)blockIdx.x * words;
    for (int64_t e = off[v] + threadIdx.x; e < off[v + 1]; e += blockDim.x) {
        const int32_t x = cols[e];
        atomicOr(bm + (x >> 5), 1u << (x & 31));
    }
}

// ---------------------------------------------------------------- Eq. probability_function

// T[F1] * T[I1] * T[F2] in IEEE double, round-to-nearest products and quotients in
// the order written (binom by the multiplicative recurrence, powers by repeated
// products), so that the host-side check reproduces every bit.
__device__ __forceinline__ double step_weight(int64_t d, uint64_t nsum, uint32_t hits, double c_min,
                                              int b, int f1, int ie, int f2)
{
    const int64_t n = d - b;
    if (n < f1) return 0.0;
    double t_f1 = 1.0;
    for (int j = 0; j < f1; ++j) {
        t_f1 = __dmul_rn(t_f1, (double)(n - j));
        t_f1 = __ddiv_rn(t_f1, (double)(j + 1));
    }
    double cv = c_min;
    if (d >= 2) {
        cv = __ddiv_rn((double)hits, (double)d);
        cv = cv < c_min ? c_min : cv;
        cv = cv > 1.0 ? 1.0 : cv;
    }
    double t_i1 = 1.0;
    for (int j = 0; j < ie; ++j) t_i1 = __dmul_rn(t_i1, cv);
    double t_f2 = 1.0;
    if (f2 > 0) {
        const double avg = __ddiv_rn((double)nsum, (double)d);
        for (int j = 0; j < f2; ++j) t_f2 = __dmul_rn(t_f2, avg);
    }
    return __dmul_rn(__dmul_rn(t_f1, t_i1), t_f2);
}

__global__ void k_weight_max(const int64_t *off, const uint64_t *nsum, const uint32_t *hits,
                             int64_t nv, double c_min, int b, int f1, int ie, int f2,
                             unsigned long long *wmax_bits)
{
    double m = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const double w = step_weight(off[v + 1] - off[v], nsum[v], hits[v], c_min, b, f1, ie, f2);
        m = w > m ? w : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_xor_sync(kFull, m, o);
        m = other > m ? other : m;
    }
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(wmax_bits, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_weight_quantise(const int64_t *off, const uint64_t *nsum, const uint32_t *hits,
                                  int64_t nv, double c_min, int b, int f1, int ie, int f2, int shift,
                                  uint64_t *q)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = off[v + 1] - off[v];
        uint64_t out = 0;
        if (d - b >= f1) {
            const double w = step_weight(d, nsum[v], hits[v], c_min, b, f1, ie, f2);
            const double scaled = floor(ldexp(w, shift));
            out = scaled < 1.0 ? 1u : (uint64_t)scaled;
        }
        q[v] = out;
    }
}

// ---------------------------------------------------------------- prefix sums
// Inclusive scan of uint64 over n entries in three passes (tile sums, scan of the
// tile sums, tile-local scans plus carry).  Integer addition makes the result
// independent of the order.

constexpr int kScanThreads = 256, kScanPer = 8, kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ uint64_t block_incl_scan(uint64_t v, uint64_t *warp_tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t n = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += n;
    }
    if (lane == 31) warp_tot[w] = v;
    __syncthreads();
    if (w == 0) {
        uint64_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t n = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += n;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    const uint64_t before = w > 0 ? warp_tot[w - 1] : 0;
    __syncthreads();
    return v + before;
}

__global__ void k_scan_tile_sums(const uint64_t *in, int64_t n, uint64_t *tile_sums)
{
    __shared__ uint64_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    uint64_t s = 0;
    for (int j = 0; j < kScanPer; ++j) if (base + j < n) s += in[base + j];
    const uint64_t incl = block_incl_scan(s, wt);
    if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = incl;
}

__global__ void k_scan_single(uint64_t *x, int64_t n)
{
    __shared__ uint64_t wt[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const uint64_t v = i < n ? x[i] : 0;
        const uint64_t incl = block_incl_scan(v, wt);
        const uint64_t c = carry;
        if (i < n) x[i] = incl + c;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = c + incl;
        __syncthreads();
    }
}

__global__ void k_scan_apply(const uint64_t *in, int64_t n, const uint64_t *tile_incl, uint64_t *out)
{
    __shared__ uint64_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    uint64_t vals[kScanPer];
    uint64_t s = 0;
    for (int j = 0; j < kScanPer; ++j) {
        vals[j] = base + j < n ? in[base + j] : 0;
        s += vals[j];
    }
    const uint64_t incl = block_incl_scan(s, wt);
    uint64_t run = incl - s + (blockIdx.x > 0 ? tile_incl[blockIdx.x - 1] : 0);
    for (int j = 0; j < kScanPer; ++j) {
        run += vals[j];
        if (base + j < n) out[base + j] = run;
    }
}

// Row prefix: for entry e of row v, sum of q(cols[e']) over e' in [off[v], e].
// One warp per row, windows of 32 entries with a running carry.
__global__ void k_row_prefix(const int64_t *off, const int32_t *cols, int64_t nv, const uint64_t *q,
                             uint64_t *rowp)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < nv; v += nwarps) {
        const int64_t s = off[v], e = off[v + 1];
        uint64_t carry = 0;
        for (int64_t i0 = s; i0 < e; i0 += 32) {
            const int64_t i = i0 + lane;
            uint64_t w = i < e ? __ldg(q + __ldg(cols + i)) : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t n = __shfl_up_sync(kFull, w, o);
                if (lane >= o) w += n;
            }
            if (i < e) rowp[i] = carry + w;
            carry += __shfl_sync(kFull, w, 31);
        }
    }
}

// Row prefix of the listed rows only: row of rows[h] goes to out[base[rows[h]] ...].
__global__ void k_row_prefix_partial(const int64_t *off, const int32_t *cols, const int32_t *rows, int64_t nrows,
                                     const int64_t *base, const uint64_t *q, uint64_t *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t h = warp; h < nrows; h += nwarps) {
        const int32_t v = rows[h];
        const int64_t s = off[v], e = off[v + 1];
        uint64_t *dst = out + base[v];
        uint64_t carry = 0;
        for (int64_t i0 = s; i0 < e; i0 += 32) {
            const int64_t i = i0 + lane;
            uint64_t w = i < e ? __ldg(q + __ldg(cols + i)) : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t n = __shfl_up_sync(kFull, w, o);
                if (lane >= o) w += n;
            }
            if (i < e) dst[i - s] = carry + w;
            carry += __shfl_sync(kFull, w, 31);
        }
    }
}

// ---------------------------------------------------------------- degree ordering

// u -> v is kept when (d(u), u) < (d(v), v) lexicographically
__device__ __forceinline__ bool orient_keep(int64_t du, int64_t u, int64_t dv, int64_t v)
{
    return du < dv || (du == dv && u < v);
}

// kept[u] = out-degree of u in the orientation; one warp per row
__global__ void k_orient_count(const int64_t *off, const int32_t *cols, int64_t nv, uint64_t *kept)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < nv; u += nwarps) {
        const int64_t s = off[u], e = off[u + 1], du = e - s;
        uint32_t n = 0;
        for (int64_t i = s + lane; i < e; i += 32) {
            const int32_t v = __ldg(cols + i);
            n += orient_keep(du, u, __ldg(off + v + 1) - __ldg(off + v), v);
        }
        for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(kFull, n, o);
        if (lane == 0) kept[u] = n;
    }
}

// writes the kept entries of each row, in row order, from out_off[u]; one warp per row
__global__ void k_orient_fill(const int64_t *off, const int32_t *cols, int64_t nv, const int64_t *out_off,
                              int32_t *out_cols)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < nv; u += nwarps) {
        const int64_t s = off[u], e = off[u + 1], du = e - s;
        int64_t pos = out_off[u];
        for (int64_t i0 = s; i0 < e; i0 += 32) {
            const int64_t i = i0 + lane;
            int32_t v = 0;
            bool keep = false;
            if (i < e) {
                v = __ldg(cols + i);
                keep = orient_keep(du, u, __ldg(off + v + 1) - __ldg(off + v), v);
            }
            const unsigned b = __ballot_sync(kFull, keep);
            if (keep) out_cols[pos + __popc(b & ((1u << lane) - 1u))] = v;
            pos += __popc(b);
        }
    }
}

int grid_stride_blocks(const agis_graph *g, int64_t work, int threads)
{
    int64_t blocks = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)g->ctx->sm_count * 16;
    if (blocks > cap) blocks = cap;
    return blocks < 1 ? 1 : (int)blocks;
}

int inclusive_scan(agis_graph *g, const uint64_t *in, int64_t n, uint64_t *out)
{
    return inclusive_scan_u64(g->ctx, in, n, out);
}

}  // namespace

int inclusive_scan_u64(agis_ctx *ctx, const uint64_t *in, int64_t n, uint64_t *out)
{
    cudaStream_t st = ctx->stream;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 0) return AGIS_OK;
    uint64_t *tile_sums = nullptr;
    AGIS_CUDA_TRY(cudaMallocAsync(&tile_sums, sizeof(uint64_t) * tiles, st));
    count_launch();
    k_scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tile_sums);
    count_launch();
    k_scan_single<<<1, kScanThreads, 0, st>>>(tile_sums, tiles);
    count_launch();
    k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tile_sums, out);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(tile_sums, st);
    return cuda_status(e);
}


// Bitmaps for every vertex of degree >= max(bitmap_min_degree, t), t the smallest
// degree whose hub set fits the bitmap budget (default a sixteenth of device
// memory; nv bits per hub).  A membership test against such a row is then one
// independent load.
int build_hub_bitmaps(agis_graph *g)
{
    cudaStream_t st = g->ctx->stream;
    cudaFree(g->hub_id);
    cudaFree(g->hub_bits);
    g->hub_id = nullptr;
    g->hub_bits = nullptr;
    g->n_hubs = 0;
    g->hub_words = (g->nv + 31) / 32;
    std::vector<int64_t> off((size_t)g->nv + 1);
    AGIS_CUDA_TRY(cudaMemcpy(off.data(), g->off, sizeof(int64_t) * off.size(), cudaMemcpyDeviceToHost));
    std::vector<int64_t> deg((size_t)g->nv);
    for (int64_t v = 0; v < g->nv; ++v) deg[(size_t)v] = off[(size_t)v + 1] - off[(size_t)v];
    size_t free_b = 0, total_b = 0;
    AGIS_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    const size_t per_hub = sizeof(uint32_t) * (size_t)g->hub_words;
    const size_t budget = g->bitmap_budget ? g->bitmap_budget : total_b / 16;
    const size_t max_hubs = std::min<size_t>(budget / per_hub, 1u << 20);
    std::vector<int64_t> sorted(deg);
    int64_t t = std::max<int64_t>(1, g->bitmap_min_degree);
    if (sorted.size() > max_hubs && max_hubs > 0) {
        std::nth_element(sorted.begin(), sorted.begin() + (max_hubs - 1), sorted.end(), std::greater<int64_t>());
        t = std::max<int64_t>(t, sorted[max_hubs - 1] + 1);
    }
    std::vector<int32_t> hubs;
    for (int64_t v = 0; v < g->nv; ++v)
        if (deg[(size_t)v] >= t && hubs.size() < max_hubs) hubs.push_back((int32_t)v);
    // bitmaps in decreasing degree order (ties by id): the most probed first, so that
    // one address window covers the hottest of them
    std::stable_sort(hubs.begin(), hubs.end(),
                     [&](int32_t a, int32_t b) { return deg[(size_t)a] > deg[(size_t)b]; });
    std::vector<int32_t> hub_id((size_t)g->nv, -1);
    for (size_t h = 0; h < hubs.size(); ++h) hub_id[(size_t)hubs[h]] = (int32_t)h;
    g->hub_min_degree = t;
    AGIS_CUDA_TRY(cudaMalloc(&g->hub_id, sizeof(int32_t) * (size_t)g->nv));
    AGIS_CUDA_TRY(cudaMemcpyAsync(g->hub_id, hub_id.data(), sizeof(int32_t) * (size_t)g->nv, cudaMemcpyHostToDevice, st));
    if (!hubs.empty()) {
        int32_t *d_hubs = nullptr;
        AGIS_CUDA_TRY(cudaMallocAsync(&d_hubs, sizeof(int32_t) * hubs.size(), st));
        AGIS_CUDA_TRY(cudaMemcpyAsync(d_hubs, hubs.data(), sizeof(int32_t) * hubs.size(), cudaMemcpyHostToDevice, st));
        AGIS_CUDA_TRY(cudaMalloc(&g->hub_bits, per_hub * hubs.size()));
        AGIS_CUDA_TRY(cudaMemsetAsync(g->hub_bits, 0, per_hub * hubs.size(), st));
        count_launch();
        k_hub_bitmaps<<<(unsigned)hubs.size(), 256, 0, st>>>(g->off, g->cols, d_hubs, g->hub_words, g->hub_bits);
        AGIS_CUDA_TRY(cudaGetLastError());
        cudaFreeAsync(d_hubs, st);
    }
    AGIS_CUDA_TRY(cudaStreamSynchronize(st));
    g->n_hubs = (int64_t)hubs.size();
    g->lb.generation++;          // a captured epoch graph holds the old bitmap addresses
    return AGIS_OK;
}

bool rowp_full_fits(const agis_graph *g) { return (size_t)g->nnz * sizeof(uint64_t) <= g->rowp_budget; }

// Rows that get a prefix when the full table does not fit: the highest-degree rows
// whose entries fit the row-prefix budget (shared by every configuration).
int build_partial_rowp_layout(agis_graph *g)
{
    if (g->rp_base) return AGIS_OK;
    cudaStream_t st = g->ctx->stream;
    std::vector<int64_t> off((size_t)g->nv + 1);
    AGIS_CUDA_TRY(cudaMemcpy(off.data(), g->off, sizeof(int64_t) * off.size(), cudaMemcpyDeviceToHost));
    // Rows in descending degree, ascending id among equal degrees, are given a
    // prefix while the budget lasts (stopping at the first row that does not fit).
    // A degree histogram replaces the sort: whole degree classes are taken from
    // the top, then the lowest ids of the class that no longer fits entirely.
    auto deg = [&](int64_t v) { return off[(size_t)v + 1] - off[(size_t)v]; };
    const int64_t max_d = g->max_deg;
    std::vector<int64_t> hist((size_t)max_d + 1, 0);
    for (int64_t v = 0; v < g->nv; ++v) hist[(size_t)deg(v)]++;
    const int64_t cap_entries = (int64_t)(g->rowp_budget / sizeof(uint64_t));
    std::vector<int64_t> take((size_t)max_d + 1, 0), start((size_t)max_d + 1, 0), first_row((size_t)max_d + 1, 0);
    int64_t used = 0, nrows = 0, min_deg = 0;
    for (int64_t d = max_d; d >= 1; --d) {
        if (hist[(size_t)d] == 0) continue;
        const int64_t fit = (cap_entries - used) / d;
        const int64_t t = std::min(hist[(size_t)d], std::max<int64_t>(fit, 0));
        take[(size_t)d] = t;
        start[(size_t)d] = used;
        first_row[(size_t)d] = nrows;
        if (t > 0) min_deg = d;
        used += t * d;
        nrows += t;
        if (t < hist[(size_t)d]) break;
    }
    std::vector<int64_t> base((size_t)g->nv, -1);
    std::vector<int32_t> rows((size_t)nrows);
    std::vector<int64_t> seen((size_t)max_d + 1, 0);
    for (int64_t v = 0; v < g->nv; ++v) {
        const int64_t d = deg(v);
        if (d == 0 || seen[(size_t)d] >= take[(size_t)d]) continue;
        const int64_t r = seen[(size_t)d]++;
        base[(size_t)v] = start[(size_t)d] + r * d;
        rows[(size_t)(first_row[(size_t)d] + r)] = (int32_t)v;
    }
    AGIS_CUDA_TRY(cudaMalloc(&g->rp_base, sizeof(int64_t) * (size_t)g->nv));
    AGIS_CUDA_TRY(cudaMemcpyAsync(g->rp_base, base.data(), sizeof(int64_t) * (size_t)g->nv, cudaMemcpyHostToDevice, st));
    if (!rows.empty()) {
        AGIS_CUDA_TRY(cudaMalloc(&g->rp_rows, sizeof(int32_t) * rows.size()));
        AGIS_CUDA_TRY(cudaMemcpyAsync(g->rp_rows, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice, st));
    }
    AGIS_CUDA_TRY(cudaStreamSynchronize(st));
    g->rp_nrows = (int64_t)rows.size();
    g->rp_entries = used;
    g->rp_min_degree = min_deg;
    g->lb.generation++;
    return AGIS_OK;
}

uint64_t cfg_key(const int32_t cfg[4])
{
    return ((uint64_t)(uint8_t)cfg[0] << 24) | ((uint64_t)(uint8_t)cfg[1] << 16) |
           ((uint64_t)(uint8_t)cfg[2] << 8) | (uint64_t)(uint8_t)cfg[3];
}

size_t table_bytes(const agis_graph *g, const int32_t cfg[4], bool need_pref, bool need_rowp)
{
    (void)cfg;
    size_t b = sizeof(uint64_t) * (size_t)g->nv;
    if (need_pref) b += sizeof(uint64_t) * (size_t)g->nv;
    if (need_rowp) b += sizeof(uint64_t) * (size_t)g->nnz;
    return b;
}

void free_table(WeightTable &t)
{
    cudaFree(t.q);
    cudaFree(t.pref);
    cudaFree(t.rowp);
    t.q = t.pref = t.rowp = nullptr;
    t.bytes = 0;
}

// Builds (or extends) the table of one step configuration.  Caller holds g->mu.
int build_weight_table(agis_graph *g, const int32_t cfg[4], bool need_pref, bool need_rowp,
                       WeightTable **out)
{
    agis::NvtxRange nvtx_range("agis:tables");
    if (!g->prepped) return AGIS_ERR_STATE;
    cudaStream_t st = g->ctx->stream;
    const uint64_t key = cfg_key(cfg);
    auto it = g->tables.find(key);
    WeightTable *t;
    if (it == g->tables.end()) {
        WeightTable fresh;
        std::memcpy(fresh.cfg, cfg, sizeof(fresh.cfg));
        t = &g->tables.emplace(key, fresh).first->second;
        const int64_t nv = g->nv;
        AGIS_CUDA_TRY(cudaMalloc(&t->q, sizeof(uint64_t) * (size_t)(nv > 0 ? nv : 1)));
        t->bytes = sizeof(uint64_t) * (size_t)nv;
        unsigned long long *d_max = nullptr;
        AGIS_CUDA_TRY(cudaMallocAsync(&d_max, sizeof(unsigned long long), st));
        AGIS_CUDA_TRY(cudaMemsetAsync(d_max, 0, sizeof(unsigned long long), st));
        const int blocks = grid_stride_blocks(g, nv, 256);
        count_launch();
        k_weight_max<<<blocks, 256, 0, st>>>(g->off, g->nsum, g->hits, nv, g->c_min, cfg[0], cfg[1],
                                             cfg[2], cfg[3], d_max);
        unsigned long long bits = 0;
        AGIS_CUDA_TRY(cudaMemcpyAsync(&bits, d_max, sizeof(bits), cudaMemcpyDeviceToHost, st));
        AGIS_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFreeAsync(d_max, st);
        double wmax;
        std::memcpy(&wmax, &bits, sizeof(wmax));
        // scale so that max weight < 2^K, K = 62 - ceil(log2(nv + 1)): every sum of
        // quantised weights stays below 2^62
        int expo = 0;
        if (wmax > 0.0) std::frexp(wmax, &expo);
        int lg = 0;
        while (lg < 63 && (1ull << lg) < (uint64_t)(nv + 1)) ++lg;
        t->shift = (62 - lg) - expo;
        count_launch();
        k_weight_quantise<<<blocks, 256, 0, st>>>(g->off, g->nsum, g->hits, nv, g->c_min, cfg[0],
                                                  cfg[1], cfg[2], cfg[3], t->shift, t->q);
        AGIS_CUDA_TRY(cudaGetLastError());
    } else {
        t = &it->second;
    }
    if (need_pref && !t->pref) {
        AGIS_CUDA_TRY(cudaMalloc(&t->pref, sizeof(uint64_t) * (size_t)(g->nv > 0 ? g->nv : 1)));
        t->bytes += sizeof(uint64_t) * (size_t)g->nv;
        int rc = inclusive_scan(g, t->q, g->nv, t->pref);
        if (rc != AGIS_OK) return rc;
        if (g->nv > 0)
            AGIS_CUDA_TRY(cudaMemcpyAsync(&t->total, t->pref + (g->nv - 1), sizeof(uint64_t),
                                          cudaMemcpyDeviceToHost, st));
        AGIS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (need_rowp && !t->rowp) {
        if (rowp_full_fits(g)) {
            AGIS_CUDA_TRY(cudaMalloc(&t->rowp, sizeof(uint64_t) * (size_t)(g->nnz > 0 ? g->nnz : 1)));
            t->bytes += sizeof(uint64_t) * (size_t)g->nnz;
            t->rowp_partial = false;
            const int blocks = grid_stride_blocks(g, g->nv * 32, 256);
            count_launch();
            k_row_prefix<<<blocks, 256, 0, st>>>(g->off, g->cols, g->nv, t->q, t->rowp);
            AGIS_CUDA_TRY(cudaGetLastError());
        } else {
            int rc = build_partial_rowp_layout(g);
            if (rc != AGIS_OK) return rc;
            if (g->rp_nrows > 0) {
                AGIS_CUDA_TRY(cudaMalloc(&t->rowp, sizeof(uint64_t) * (size_t)g->rp_entries));
                t->bytes += sizeof(uint64_t) * (size_t)g->rp_entries;
                t->rowp_partial = true;
                const int blocks = grid_stride_blocks(g, g->rp_nrows * 32, 256);
                count_launch();
                k_row_prefix_partial<<<blocks, 256, 0, st>>>(g->off, g->cols, g->rp_rows, g->rp_nrows, g->rp_base,
                                                             t->q, t->rowp);
                AGIS_CUDA_TRY(cudaGetLastError());
            }
        }
    }
    t->last_use = ++g->use_clock;
    *out = t;
    return AGIS_OK;
}

}  // namespace agis

using namespace agis;

extern "C" int agis_graph_load_csr(agis_ctx *ctx, const void *offsets, int offsets_are_64bit,
                                   const int32_t *cols, int64_t nv, int64_t nnz, int on_device,
                                   int validate, agis_graph **out)
{
    agis::NvtxRange nvtx_range("agis:load");
    if (!ctx || !out || !offsets || (nnz > 0 && !cols) || nv < 1 || nnz < 0 || nv > INT32_MAX)
        return AGIS_ERR_ARG;
    *out = nullptr;
    AGIS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    agis_graph *g = new (std::nothrow) agis_graph();
    if (!g) return AGIS_ERR_NOMEM;
    g->ctx = ctx;
    g->nv = nv;
    g->nnz = nnz;
    auto fail = [&](int rc) { cudaFree(g->off); cudaFree(g->cols); delete g; return rc; };
    if (cudaMalloc(&g->off, sizeof(int64_t) * (size_t)(nv + 1)) != cudaSuccess) return fail(AGIS_ERR_NOMEM);
    // 16 entries of padding: the sampler's 16-byte row loads may read past the end
    if (cudaMalloc(&g->cols, sizeof(int32_t) * (size_t)(nnz + 16)) != cudaSuccess)
        return fail(AGIS_ERR_NOMEM);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (offsets_are_64bit) {
        if (cudaMemcpyAsync(g->off, offsets, sizeof(int64_t) * (size_t)(nv + 1), kind, st) != cudaSuccess)
            return fail(AGIS_ERR_CUDA);
    } else {
        // widen int32 offsets on the host side of the copy
        std::vector<int64_t> wide((size_t)nv + 1);
        std::vector<int32_t> narrow;
        const int32_t *src = (const int32_t *)offsets;
        if (on_device) {
            narrow.resize((size_t)nv + 1);
            if (cudaMemcpy(narrow.data(), offsets, sizeof(int32_t) * (size_t)(nv + 1),
                           cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail(AGIS_ERR_CUDA);
            src = narrow.data();
        }
        for (int64_t i = 0; i <= nv; ++i) wide[(size_t)i] = src[i];
        if (cudaMemcpyAsync(g->off, wide.data(), sizeof(int64_t) * (size_t)(nv + 1),
                            cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail(AGIS_ERR_CUDA);
    }
    if (nnz > 0 && cudaMemcpyAsync(g->cols, cols, sizeof(int32_t) * (size_t)nnz, kind, st) != cudaSuccess)
        return fail(AGIS_ERR_CUDA);
    int *d_err = nullptr;
    if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) return fail(AGIS_ERR_NOMEM);
    cudaMemsetAsync(d_err, 0, sizeof(int), st);
    const int blocks = grid_stride_blocks(g, nv + 1, 256);
    count_launch();
    k_check_offsets<<<blocks, 256, 0, st>>>(g->off, nv, nnz, d_err);
    int err = 0;
    cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { cudaFree(d_err); return fail(AGIS_ERR_CUDA); }
    if (err) { cudaFree(d_err); return fail(AGIS_ERR_GRAPH); }
    if (validate) {
        count_launch();
        k_check_rows<<<grid_stride_blocks(g, nv * 32, 256), 256, 0, st>>>(g->off, g->cols, nv, 0, d_err);
        cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) { cudaFree(d_err); return fail(AGIS_ERR_CUDA); }
        if (err) { cudaFree(d_err); return fail(AGIS_ERR_GRAPH); }
    }
    cudaFree(d_err);
    {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) g->rowp_budget = total_b / 4;
    }
    // max degree (host side, from the offsets)
    {
        std::vector<int64_t> h((size_t)nv + 1);
        if (cudaMemcpy(h.data(), g->off, sizeof(int64_t) * (size_t)(nv + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(AGIS_ERR_CUDA);
        int64_t m = 0;
        for (int64_t v = 0; v < nv; ++v) m = std::max(m, h[(size_t)v + 1] - h[(size_t)v]);
        g->max_deg = m;
    }
    ctx_retain(ctx);
    *out = g;
    return AGIS_OK;
}

extern "C" int agis_graph_preprocess(agis_graph *g, uint64_t seed, double c_min)
{
    agis::NvtxRange nvtx_range("agis:preprocess");
    if (!g || !(c_min > 0.0) || c_min > 1.0) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    for (auto &kv : g->tables) free_table(kv.second);
    g->tables.clear();
    if (!g->nsum) AGIS_CUDA_TRY(cudaMalloc(&g->nsum, sizeof(uint64_t) * (size_t)g->nv));
    if (!g->hits) AGIS_CUDA_TRY(cudaMalloc(&g->hits, sizeof(uint32_t) * (size_t)g->nv));
    const int blocks = grid_stride_blocks(g, g->nv * 32, 256);
    count_launch();
    k_neighbour_degree_sum<<<blocks, 256, 0, st>>>(g->off, g->cols, g->nv, g->nsum);
    count_launch();
    k_cluster_hits<<<blocks, 256, 0, st>>>(g->off, g->cols, g->nv, seed, g->hits);
    AGIS_CUDA_TRY(cudaGetLastError());
    AGIS_CUDA_TRY(cudaStreamSynchronize(st));
    int rc = build_hub_bitmaps(g);
    if (rc != AGIS_OK) return rc;
    g->prepped = true;
    g->c_min = c_min;
    g->prep_seed = seed;
    return AGIS_OK;
}

extern "C" int agis_graph_info(const agis_graph *g, int64_t *nv, int64_t *nnz, int64_t *max_degree,
                               uint64_t *device_bytes)
{
    if (!g) return AGIS_ERR_ARG;
    if (nv) *nv = g->nv;
    if (nnz) *nnz = g->nnz;
    if (max_degree) *max_degree = g->max_deg;
    if (device_bytes) {
        uint64_t b = 8ull * (uint64_t)(g->nv + 1) + 4ull * (uint64_t)g->nnz;
        if (g->nsum) b += 12ull * (uint64_t)g->nv;
        for (const auto &kv : g->tables) b += kv.second.bytes;
        *device_bytes = b;
    }
    return AGIS_OK;
}

extern "C" int agis_graph_stats_copy(const agis_graph *g, uint64_t *nsum, uint32_t *hits)
{
    if (!g) return AGIS_ERR_ARG;
    if (!g->prepped) return AGIS_ERR_STATE;
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    AGIS_CUDA_TRY(cudaStreamSynchronize(g->ctx->stream));
    if (nsum) AGIS_CUDA_TRY(cudaMemcpy(nsum, g->nsum, sizeof(uint64_t) * (size_t)g->nv, cudaMemcpyDeviceToHost));
    if (hits) AGIS_CUDA_TRY(cudaMemcpy(hits, g->hits, sizeof(uint32_t) * (size_t)g->nv, cudaMemcpyDeviceToHost));
    return AGIS_OK;
}

extern "C" int agis_graph_weight_table(agis_graph *g, const int32_t cfg[4], uint64_t *q,
                                       uint64_t *prefix, int32_t *shift)
{
    if (!g || !cfg) return AGIS_ERR_ARG;
    for (int i = 0; i < 4; ++i) if (cfg[i] < 0 || cfg[i] > 64) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    WeightTable *t = nullptr;
    int rc = build_weight_table(g, cfg, prefix != nullptr, false, &t);
    if (rc != AGIS_OK) return rc;
    AGIS_CUDA_TRY(cudaStreamSynchronize(g->ctx->stream));
    if (q) AGIS_CUDA_TRY(cudaMemcpy(q, t->q, sizeof(uint64_t) * (size_t)g->nv, cudaMemcpyDeviceToHost));
    if (prefix) AGIS_CUDA_TRY(cudaMemcpy(prefix, t->pref, sizeof(uint64_t) * (size_t)g->nv, cudaMemcpyDeviceToHost));
    if (shift) *shift = t->shift;
    return AGIS_OK;
}

extern "C" int agis_graph_row_prefix(agis_graph *g, const int32_t cfg[4], uint64_t *row_prefix)
{
    if (!g || !cfg || !row_prefix) return AGIS_ERR_ARG;
    for (int i = 0; i < 4; ++i) if (cfg[i] < 0 || cfg[i] > 64) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    WeightTable *t = nullptr;
    int rc = build_weight_table(g, cfg, false, true, &t);
    if (rc != AGIS_OK) return rc;
    AGIS_CUDA_TRY(cudaStreamSynchronize(g->ctx->stream));
    if (!t->rowp || t->rowp_partial) return AGIS_ERR_STATE;
    AGIS_CUDA_TRY(cudaMemcpy(row_prefix, t->rowp, sizeof(uint64_t) * (size_t)g->nnz, cudaMemcpyDeviceToHost));
    return AGIS_OK;
}

extern "C" int agis_graph_drop_tables(agis_graph *g)
{
    if (!g) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    cudaSetDevice(g->ctx->device);
    cudaStreamSynchronize(g->ctx->stream);
    for (auto it = g->tables.begin(); it != g->tables.end();) {
        if (it->second.pins > 0) { ++it; continue; }
        free_table(it->second);
        it = g->tables.erase(it);
    }
    return AGIS_OK;
}

extern "C" int agis_graph_validate(agis_graph *g)
{
    if (!g) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    int *d_err = nullptr;
    AGIS_CUDA_TRY(cudaMalloc(&d_err, sizeof(int)));
    cudaMemsetAsync(d_err, 0, sizeof(int), st);
    count_launch();
    k_check_offsets<<<grid_stride_blocks(g, g->nv + 1, 256), 256, 0, st>>>(g->off, g->nv, g->nnz, d_err);
    int err = 0;
    cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && !err) {
        count_launch();
        k_check_rows<<<grid_stride_blocks(g, g->nv * 32, 256), 256, 0, st>>>(g->off, g->cols, g->nv,
                                                                             g->oriented ? 1 : 0, d_err);
        cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
        e = cudaStreamSynchronize(st);
    }
    cudaFree(d_err);
    if (e != cudaSuccess) return AGIS_ERR_CUDA;
    return err ? AGIS_ERR_GRAPH : AGIS_OK;
}

extern "C" int agis_graph_copy_csr(const agis_graph *g, int64_t *off, int32_t *cols)
{
    if (!g) return AGIS_ERR_ARG;
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    AGIS_CUDA_TRY(cudaStreamSynchronize(g->ctx->stream));
    if (off) AGIS_CUDA_TRY(cudaMemcpy(off, g->off, sizeof(int64_t) * (size_t)(g->nv + 1), cudaMemcpyDeviceToHost));
    if (cols && g->nnz > 0)
        AGIS_CUDA_TRY(cudaMemcpy(cols, g->cols, sizeof(int32_t) * (size_t)g->nnz, cudaMemcpyDeviceToHost));
    return AGIS_OK;
}

extern "C" int agis_graph_orient(agis_graph *g, agis_graph **out)
{
    agis::NvtxRange nvtx_range("agis:orient");
    if (!g || !out) return AGIS_ERR_ARG;
    *out = nullptr;
    if (g->oriented) return AGIS_ERR_STATE;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    AGIS_CUDA_TRY(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    agis_graph *o = new (std::nothrow) agis_graph();
    if (!o) return AGIS_ERR_NOMEM;
    o->ctx = g->ctx;
    o->nv = g->nv;
    o->oriented = true;
    o->rowp_budget = g->rowp_budget;
    o->bitmap_budget = g->bitmap_budget;
    o->bitmap_min_degree = g->bitmap_min_degree;
    o->list_cap = g->list_cap;
    o->l2_window_bytes = g->l2_window_bytes;
    uint64_t *kept = nullptr;
    auto fail = [&](int rc) {
        cudaStreamSynchronize(st);
        cudaFree(kept);
        cudaFree(o->off);
        cudaFree(o->cols);
        delete o;
        return rc;
    };
    if (cudaMalloc(&o->off, sizeof(int64_t) * (size_t)(g->nv + 1)) != cudaSuccess ||
        cudaMalloc(&kept, sizeof(uint64_t) * (size_t)g->nv) != cudaSuccess)
        return fail(AGIS_ERR_NOMEM);
    const int blocks = grid_stride_blocks(g, g->nv * 32, 256);
    count_launch();
    k_orient_count<<<blocks, 256, 0, st>>>(g->off, g->cols, g->nv, kept);
    if (cudaMemsetAsync(o->off, 0, sizeof(int64_t), st) != cudaSuccess) return fail(AGIS_ERR_CUDA);
    // offsets: off[0] = 0 and off[u + 1] = the inclusive running sum of the kept counts
    int rc = inclusive_scan_u64(g->ctx, kept, g->nv, (uint64_t *)(o->off + 1));
    if (rc != AGIS_OK) return fail(rc);
    std::vector<int64_t> h((size_t)g->nv + 1);
    if (cudaMemcpyAsync(h.data(), o->off, sizeof(int64_t) * (size_t)(g->nv + 1), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(AGIS_ERR_CUDA);
    o->nnz = h[(size_t)g->nv];
    for (int64_t v = 0; v < g->nv; ++v) o->max_deg = std::max(o->max_deg, h[(size_t)v + 1] - h[(size_t)v]);
    // 16 entries of padding for the sampler's 16-byte row loads, zeroed
    if (cudaMalloc(&o->cols, sizeof(int32_t) * (size_t)(o->nnz + 16)) != cudaSuccess) return fail(AGIS_ERR_NOMEM);
    if (cudaMemsetAsync(o->cols + o->nnz, 0, sizeof(int32_t) * 16, st) != cudaSuccess) return fail(AGIS_ERR_CUDA);
    count_launch();
    k_orient_fill<<<blocks, 256, 0, st>>>(g->off, g->cols, g->nv, o->off, o->cols);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return fail(AGIS_ERR_CUDA);
    cudaFree(kept);
    ctx_retain(o->ctx);
    *out = o;
    return AGIS_OK;
}

extern "C" int agis_graph_is_oriented(const agis_graph *g)
{
    if (!g) return AGIS_ERR_ARG;
    return g->oriented ? 1 : 0;
}

// ---------------------------------------------------------------- prefix sum without allocation
// Some callers cannot call cudaMalloc: a custom device allocator or memory-pool hook
// that must not re-enter the CUDA allocator, a service whose device memory a pool
// already holds in full (so an allocation would fail), and latency-critical code
// that avoids cudaMalloc because it can block and synchronise the device.  For them
// this variant of the prefix-sum scan keeps its tile-sum scratch in a file-scope
// device array instead of allocating it.  The array exists once on every device that
// loads this library and stays allocated until the process exits.

namespace agis {
namespace {

constexpr int64_t kNoAllocMaxTiles = 65536;   // 512 KiB of tile sums
constexpr int64_t kNoAllocMaxN = kNoAllocMaxTiles * kScanTile;

static __device__ __align__(256) uint64_t g_noalloc_tile_sums[kNoAllocMaxTiles];

std::mutex g_noalloc_mu;
std::unordered_map<unsigned long long, uint64_t *> g_noalloc_ptr;   // context id -> array address

// cuCtxGetCurrent and cuCtxGetId, reached through the runtime's driver entry points
// (the library links only the runtime).
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Unique id of the context current on this thread (0 when none is current); ids are
// never reused within a process, so a reset device or another context gets a new one.
int current_context_id(unsigned long long *id)
{
    *id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return AGIS_ERR_CUDA;
        g_ctx_get_current = (CtxGetCurrentFn)f0;
        g_ctx_get_id = (CtxGetIdFn)f1;
    }
    void *ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0) return AGIS_ERR_CUDA;
    if (ctx && g_ctx_get_id(ctx, id) != 0) return AGIS_ERR_CUDA;
    return AGIS_OK;
}

// Device address of the scratch array in the context current on this thread, looked
// up once per context (host code must not use the array's name as an address).
int noalloc_scratch(uint64_t **out)
{
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    unsigned long long id = 0;
    int rc = current_context_id(&id);
    if (rc != AGIS_OK) return rc;
    if (id != 0) {
        auto it = g_noalloc_ptr.find(id);
        if (it != g_noalloc_ptr.end()) {
            *out = it->second;
            return AGIS_OK;
        }
    }
    // the lookup also makes the device's primary context current when none is
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_tile_sums) != cudaSuccess || !p) return AGIS_ERR_CUDA;
    if (id == 0 && ((rc = current_context_id(&id)) != AGIS_OK || id == 0)) return rc != AGIS_OK ? rc : AGIS_ERR_CUDA;
    g_noalloc_ptr[id] = (uint64_t *)p;
    *out = (uint64_t *)p;
    return AGIS_OK;
}

}  // namespace
}  // namespace agis

extern "C" int agis_prefix_sum_u64_noalloc(const uint64_t *in, int64_t n, uint64_t *out, void *cuda_stream)
{
    using namespace agis;
    if (n < 0 || (n > 0 && (!in || !out))) return AGIS_ERR_ARG;
    if (n > kNoAllocMaxN) return AGIS_ERR_ARG;
    if (n == 0) return AGIS_OK;
    uint64_t *tile_sums = nullptr;
    int rc = noalloc_scratch(&tile_sums);
    if (rc != AGIS_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    // every tile sum read below is written first by k_scan_tile_sums, so the
    // array needs no clearing between calls
    count_launch();
    k_scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tile_sums);
    AGIS_CUDA_TRY(cudaGetLastError());
    count_launch();
    k_scan_single<<<1, kScanThreads, 0, st>>>(tile_sums, tiles);
    AGIS_CUDA_TRY(cudaGetLastError());
    count_launch();
    k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tile_sums, out);
    AGIS_CUDA_TRY(cudaGetLastError());
    return AGIS_OK;
}

extern "C" int agis_graph_set_memory_policy(agis_graph *g, uint64_t row_prefix_bytes, uint64_t bitmap_bytes,
                                            int64_t bitmap_min_degree, uint32_t list_entries)
{
    if (!g || bitmap_min_degree < 0 || (list_entries != 0 && list_entries < 64)) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    cudaSetDevice(g->ctx->device);
    cudaStreamSynchronize(g->ctx->stream);
    if (row_prefix_bytes) g->rowp_budget = (size_t)row_prefix_bytes;
    if (bitmap_bytes) g->bitmap_budget = (size_t)bitmap_bytes;
    if (bitmap_min_degree) g->bitmap_min_degree = bitmap_min_degree;
    if (list_entries) g->list_cap = list_entries;
    // tables and the partial layout follow the new budget when rebuilt
    for (auto it = g->tables.begin(); it != g->tables.end();) {
        if (it->second.pins > 0) { ++it; continue; }
        free_table(it->second);
        it = g->tables.erase(it);
    }
    if (g->tables.empty()) {
        cudaFree(g->rp_base);
        cudaFree(g->rp_rows);
        g->rp_base = nullptr;
        g->rp_rows = nullptr;
        g->rp_nrows = g->rp_entries = g->rp_min_degree = 0;
    }
    g->lb.generation++;
    return AGIS_OK;
}

extern "C" int agis_graph_set_l2_window(agis_graph *g, uint64_t bytes)
{
    if (!g) return AGIS_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    g->l2_window_bytes = bytes;
    g->lb.generation++;          // captured epoch graphs carry the window as a node attribute
    return AGIS_OK;
}
