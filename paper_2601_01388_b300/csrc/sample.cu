// The sampler: Alg. 3 (structure-informed neighbour sampling) with one warp per
// trial, persistent CTAs pulling work items (kTile-trial tiles of any query) from a
// device counter, and a fixed-order FP64 reduction of each tile.
//
// Per step i of a trial (tau = v_1..v_{i-1} so far):
//   step 1        draw over all vertices: f_approx by the inclusive prefix of the
//                 quantised weights, f_uniform by the CSR offsets (edge-uniform);
//   |B[i]| = 1    S = N(a) \ tau for the backward neighbour a: the trajectory
//                 members found in a's row are excluded and the draw is a k-ary
//                 warp search over a's row prefix (f_approx) or over positions;
//   |B[i]| >= 2   S = intersection of the backward rows minus tau: the warp scans
//                 the shortest backward row 32 entries at a time and checks every
//                 entry in the other rows by binary search (closing-edge checks),
//                 then draws from the survivors' weights.
// A draw is r = floor(U * W / 2^128) with U from Philox4x64-10 at counter
// (trial, i, 1, 0), key (seed, 0); the chosen vertex is the first candidate in
// ascending id order whose inclusive running weight exceeds r; X is multiplied by
// W / q(v).  Every integer step is exact, so the device reproduces the CPU
// restatement trial for trial.
#include <cstdio>

#include "agis_internal.h"
#include "philox.cuh"

// Resident CTAs per SM the register allocation is sized for (the build may
// override it; the autotuner then picks up to this many).  Five (40 warps, 48
// registers) ran 2% faster than four and 2% faster than six on the benchmark graph.
#ifndef AGIS_MIN_BLOCKS
#define AGIS_MIN_BLOCKS 5
#endif

namespace agis {

// Optional per-step-kind cycle counters (build with -DAGIS_STEP_TIMERS): kinds are
// 0 step 1, 1 single-backward search, 2 listed intersection, 3 listed reuse,
// 4 list-free scan; entry 2k is cycles, 2k+1 the number of steps.
__device__ unsigned long long g_step_timers[16];

namespace {

constexpr unsigned kFull = 0xffffffffu;

#ifdef AGIS_STEP_TIMERS
#define STEP_T0 long long _t0 = clock64();
#define STEP_T1(kind) if (lane == 0) { atomicAdd(&g_step_timers[2 * (kind)], (unsigned long long)(clock64() - _t0)); atomicAdd(&g_step_timers[2 * (kind) + 1], 1ull); }
#else
#define STEP_T0
#define STEP_T1(kind)
#endif

// ---------------------------------------------------------------- cost model
// Sectors of a search over L entries of w bytes: ceil(log2(ceil(L*w/32))) + 1.
__device__ __forceinline__ uint64_t sec_search(int64_t L, int w)
{
    const uint64_t bytes = (uint64_t)(L > 0 ? L : 1) * (uint64_t)w;
    if (bytes <= 32) return 1;
    const uint64_t n = (bytes + 31) / 32;
    return (uint64_t)(64 - __clzll((long long)(n - 1))) + 1;
}

// Sectors to test d_a entries for membership in a row of m entries: the cheaper of
// reading the row once (a merge, streamed) and one search per entry; `survey` gets
// the search count alone.
__device__ __forceinline__ uint64_t row_check_sectors(int64_t da, int64_t m, uint64_t &streamed,
                                                      uint64_t &survey)
{
    const uint64_t merge = (uint64_t)((4 * (m > 0 ? m : 1) + 31) / 32);
    const uint64_t search = (uint64_t)da * sec_search(m, 4);
    survey += search;
    if (merge < search) {
        streamed += merge;
        return merge;
    }
    return search;
}

// Neighbour bitmap of vertex u, or null when u has none.
__device__ __forceinline__ const uint32_t *bits_of(const GraphView &g, int32_t u)
{
    if (!g.hub_bits) return nullptr;
    const int32_t h = __ldg(g.hub_id + u);
    return h < 0 ? nullptr : g.hub_bits + (int64_t)h * g.hub_words;
}

__device__ __forceinline__ bool bit_test(const uint32_t *bits, int32_t x)
{
    return (__ldg(bits + (x >> 5)) >> (x & 31)) & 1u;
}

// ---------------------------------------------------------------- searches

// Last position with row[pos] <= x, or -1 if x is absent; the probe count depends
// only on d, so lanes searching the same row stay converged.
__device__ __forceinline__ int64_t row_find(const int32_t *row, int64_t d, int32_t x)
{
    if (d <= 0) return -1;
    int64_t lo = 0, len = d;
    while (len > 1) {
        const int64_t half = len >> 1;
        if (__ldg(row + lo + half) <= x) lo += half;
        len -= half;
    }
    return __ldg(row + lo) == x ? lo : -1;
}

// Sum of the excluded weights at positions <= pos.  The excluded positions and
// weights live one per lane (bits of xmask); all lanes must call this together.
__device__ __forceinline__ uint64_t excluded_upto(int64_t pos, uint32_t xmask, int64_t xp, uint64_t xq)
{
    uint64_t s = 0;
    while (xmask) {
        const int src = __ffs(xmask) - 1;
        xmask &= xmask - 1;
        const int64_t p = __shfl_sync(kFull, xp, src);
        const uint64_t q = __shfl_sync(kFull, xq, src);
        if (p <= pos) s += q;
    }
    return s;
}

// A load from the graph or its tables, read-only for the whole launch (__ldg), or,
// with `list`, from a candidate list written earlier in this launch (a coherent load:
// the read-only path is only defined for data no thread writes during the kernel).
template <typename T>
__device__ __forceinline__ T ld_src(const T *p, bool list)
{
    return list ? *p : __ldg(p);
}

// First index j in [0, n) with F(j) > r, where F(j) = P[j] minus the excluded
// weight at or before j (or F(j) = j + 1 minus the excluded count when P is null).
// Excluded entries live one per lane (bits of xmask) as a key and a weight; the key
// is a position, or, when ids (the row's ascending vertex ids) is given, a vertex
// id compared with ids[j].  F is non-decreasing and F(n-1) > r.  Each round splits
// the range into 32 parts and one ballot picks the part, so a row of d entries takes
// ceil(log32 d) rounds of independent loads.
__device__ int64_t warp_find(const uint64_t *P, int64_t n, uint64_t r, uint32_t xmask, int64_t xkey,
                             uint64_t xq, const int32_t *ids, int lane, bool list = false)
{
    int64_t lo = 0, hi = n;
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) >> 5;
        const int64_t pos = lo + (int64_t)(lane + 1) * step - 1;
        const int64_t cpos = pos < hi - 1 ? pos : hi - 1;
        uint64_t ex = 0;
        if (xmask) {
            const int64_t key = ids ? (int64_t)__ldg(ids + cpos) : cpos;
            ex = excluded_upto(key, xmask, xkey, xq);
        }
        bool gt = true;
        if (pos < hi - 1) {
            const uint64_t f = (P ? ld_src(P + pos, list) : (uint64_t)(pos + 1)) - ex;
            gt = f > r;
        }
        const int f = __ffs(__ballot_sync(kFull, gt)) - 1;
        const int64_t nlo = lo + (int64_t)f * step;
        const int64_t nhi = lo + (int64_t)(f + 1) * step;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    const int64_t pos = lo + lane;
    const int64_t cpos = pos < hi ? pos : hi - 1;
    uint64_t ex = 0;
    if (xmask) {
        const int64_t key = ids ? (int64_t)__ldg(ids + cpos) : cpos;
        ex = excluded_upto(key, xmask, xkey, xq);
    }
    bool gt = true;
    if (pos < hi) gt = ((P ? ld_src(P + pos, list) : (uint64_t)(pos + 1)) - ex) > r;
    return lo + (__ffs(__ballot_sync(kFull, gt)) - 1);
}

// The first two rounds of warp_find over the step-1 prefix (n = nv) always read
// the same 32 + 32*32 splitters; they are staged in shared memory per query.
constexpr int kTopSplitters = 32 + 32 * 32;

__device__ __forceinline__ int64_t top_step(int64_t lo, int64_t hi) { return (hi - lo + 31) >> 5; }

// Position of splitter k of the two cached levels (level 1: k < 32; level 2: part
// f = (k-32)/32, lane (k-32)%32), or -1 where the search never reads one.
__device__ __forceinline__ int64_t top_pos(int64_t n, int k)
{
    if (n <= 32) return -1;
    const int64_t s1 = top_step(0, n);
    if (k < 32) {
        const int64_t pos = (int64_t)(k + 1) * s1 - 1;
        return pos < n - 1 ? pos : -1;
    }
    const int f = (k - 32) >> 5, l = (k - 32) & 31;
    const int64_t lo = (int64_t)f * s1, hi = lo + s1 < n ? lo + s1 : n;
    if (lo >= n || hi - lo <= 32) return -1;
    const int64_t pos = lo + (int64_t)(l + 1) * top_step(lo, hi) - 1;
    return pos < hi - 1 ? pos : -1;
}

// warp_find over P[0, n) (no exclusions) whose first two rounds use the staged
// splitters top[k] = P[top_pos(n, k)].
__device__ int64_t warp_find_top(const uint64_t *P, int64_t n, uint64_t r, const uint64_t *top, int lane)
{
    int64_t lo = 0, hi = n;
    for (int level = 0; level < 2 && hi - lo > 32; ++level) {
        const int64_t step = (hi - lo + 31) >> 5;
        const int64_t pos = lo + (int64_t)(lane + 1) * step - 1;
        bool gt = true;
        if (pos < hi - 1) {
            const int k = level == 0 ? lane : 32 + (int)(lo / top_step(0, n)) * 32 + lane;
            gt = top[k] > r;
        }
        const int f = __ffs(__ballot_sync(kFull, gt)) - 1;
        const int64_t nlo = lo + (int64_t)f * step;
        const int64_t nhi = lo + (int64_t)(f + 1) * step;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    return lo + warp_find(P + lo, hi - lo, r, 0u, 0, 0, nullptr, lane);
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, int lane)
{
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t n = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Per-trial output: X, hit flag and the three sector counts (the model, its streamed
// part, and the survey's plain count).
// Paths that few steps take (the per-lane merge, the merge or search filter of rows
// without a bitmap, the list-free scan of an overflowing step) are compiled out of
// line with AGIS_OUTLINE_COLD=1, so that the hot loop of this large kernel takes less
// instruction cache (instruction fetch is its first stall reason).
#ifndef AGIS_OUTLINE_COLD
#define AGIS_OUTLINE_COLD 1
#endif
#if AGIS_OUTLINE_COLD
#define AGIS_COLD __noinline__
#else
#define AGIS_COLD
#endif

struct TrialOut {
    double x;
    uint64_t sectors, streamed, survey;
    int hit;
};

// A backward row of a step: where it starts in cols, its length, its neighbour
// bitmap (null if none).  Kept per warp in shared memory (the values are the same on
// every lane), so they take neither registers nor local memory.
struct RowRef {
    int64_t start, len;
    const uint32_t *bits;
};

// One window of the intersection scan: entry `idx` of the anchor row for this
// lane; returns the lane's candidate weight (0 if not in S) and sets ok / x.
__device__ __forceinline__ uint64_t window_weight(const GraphView &g, const DevStep &S,
                                                  const int32_t *tau_s, int i, int64_t a_start,
                                                  int64_t da, int64_t idx, const RowRef *rows,
                                                  int n_other, bool &ok, int32_t &x)
{
    ok = idx < da;
    x = ok ? __ldg(g.cols + a_start + idx) : -1;
    if (ok) {
        for (int j = 0; j < i; ++j) ok &= (x != tau_s[j]);
    }
    for (int o = 0; o < n_other; ++o) {
        if (ok) ok = rows[o].bits ? bit_test(rows[o].bits, x) : row_find(g.cols + rows[o].start, rows[o].len, x) >= 0;
    }
    if (!ok) return 0;
    return S.approx ? __ldg(S.q + x) : 1u;
}

// Scratch of one warp: two candidate lists (ping-pong), each `cap` vertex ids and
// the inclusive running weights of the ids kept so far.
struct WarpSets {
    int32_t *xs[2];
    uint64_t *pw[2];
    uint32_t cap;
};

// Keeps the entries of the ascending list L[0, n) that are not trajectory members
// (tau_s[0, tau_n)) and that occur in the ascending row R[0, m) (all of them when R
// is null); survivors are appended, in order, to out (room for cap; a return value
// above cap means the list overflowed and out is incomplete).  With kWeigh the survivors'
// weights (q[x] under f_approx, 1 under f_uniform) are accumulated into out_pw as
// inclusive running sums and *W receives the total.
//
// Membership in R is a bit test when R's vertex has a neighbour bitmap (Rbits);
// otherwise it is found either by a warp merge (R read once, 32 entries per
// coalesced load, each loaded entry located among the 32 list entries of the window
// by a shuffle search) or by one binary search per list entry, whichever the sizes
// make cheaper.
// Appends this window's survivors (ok) to out, in lane order, with their running
// weights when kWeigh; cnt and carry advance.
template <bool kWeigh>
__device__ __forceinline__ void emit_window(bool ok, int32_t x, uint64_t w, int32_t *out, uint64_t *out_pw,
                                            uint32_t cap, uint32_t &cnt, uint64_t &carry, int lane)
{
    const uint32_t bal = __ballot_sync(kFull, ok);
    const uint32_t pos = cnt + __popc(bal & ((1u << lane) - 1u));
    const bool store = ok && pos < cap;
    if (store) out[pos] = x;
    if (kWeigh) {
        const uint64_t incl = warp_incl_scan(ok ? w : 0u, lane);
        if (store) out_pw[pos] = carry + incl;
        carry += __shfl_sync(kFull, incl, 31);
    }
    cnt += __popc(bal);
}

// Keeps the entries of the ascending list L[0, n) that are not trajectory members
// (tau_s[0, tau_n)) and that occur in the ascending row R[0, m) (all of them when R
// is null); survivors are appended, in order, to out (room for cap; a return value
// above cap means the list overflowed and out is incomplete).  With kWeigh the survivors'
// weights (q[x] under f_approx, 1 under f_uniform) are accumulated into out_pw as
// inclusive running sums and *W receives the total.
//
// Membership in R is a bit test when R's vertex has a neighbour bitmap (Rbits);
// otherwise it is found either by a warp merge (R read once, 32 entries per
// coalesced load, each loaded entry located among the 32 list entries of the window
// by a shuffle search) or by one binary search per list entry, whichever the sizes
// make cheaper.
#ifndef AGIS_FILTER_GROUPS
#define AGIS_FILTER_GROUPS 2
#endif
constexpr int kGroups = AGIS_FILTER_GROUPS;

// A bitmap probe fetches a 32-byte sector per list entry, a merge reads the other
// row once at 4 bytes per entry; the merge is used while m < AGIS_MERGE_RATIO * n.
#ifndef AGIS_MERGE_RATIO
#define AGIS_MERGE_RATIO 0
#endif

// Running weights of out[0, cnt): gathers q for two windows at a time.
__device__ __forceinline__ uint64_t weigh_list(const int32_t *out, uint32_t cnt, uint64_t *out_pw,
                                               const uint64_t *q, bool approx, int lane)
{
    uint64_t carry = 0;
    for (uint32_t b = 0; b < cnt; b += 64) {
        int32_t x[2];
        uint64_t w[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint32_t idx = b + 32 * u + lane;
            x[u] = idx < cnt ? out[idx] : 0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) w[u] = (b + 32 * u + lane < cnt) ? (approx ? __ldg(q + x[u]) : 1u) : 0u;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint64_t incl = warp_incl_scan(w[u], lane);
            const uint32_t idx = b + 32 * u + lane;
            if (idx < cnt) out_pw[idx] = carry + incl;
            carry += __shfl_sync(kFull, incl, 31);
        }
    }
    return carry;
}

// Per-lane merge: lane l takes the l-th of 32 equal segments of L, finds where the
// segment starts in R by a binary search, and merges its segment against R
// sequentially (each lane walks its own cache lines, so R is read once and the
// loads hit L1); survivors go to the lane's own stretch of tmp (at the segment's
// offset, so at most n entries), then are compacted in order into out.
template <bool kWeigh>
__device__ AGIS_COLD uint32_t filter_lane_merge(const int32_t *L, bool Llist, uint32_t n, const int32_t *R,
                                                int64_t m, const int32_t *tau_s, int tau_n, int32_t *out,
                                                int32_t *tmp, uint64_t *out_pw, uint32_t cap, const uint64_t *q,
                                                bool approx, uint64_t *W, int lane)
{
    const uint32_t seg = (n + 31) >> 5;
    const uint32_t l0 = min(n, (uint32_t)lane * seg), l1 = min(n, l0 + seg);
    uint32_t c = 0;
    if (l0 < l1 && m > 0) {
        const int32_t first = ld_src(L + l0, Llist);
        int64_t lo = 0, len = m;                  // first j with R[j] >= first
        while (len > 0) {
            const int64_t half = len >> 1;
            if (__ldg(R + lo + half) < first) { lo += half + 1; len -= half + 1; } else len = half;
        }
        int64_t j = lo;
        uint32_t i = l0;
        if (j < m) {
            int32_t x = first, y = __ldg(R + j);
            for (;;) {
                if (x < y) {
                    if (++i >= l1) break;
                    x = ld_src(L + i, Llist);
                } else if (x > y) {
                    if (++j >= m) break;
                    y = __ldg(R + j);
                } else {
                    bool ok = true;
                    for (int t = 0; t < tau_n; ++t) ok = ok && (x != tau_s[t]);
                    if (ok) tmp[l0 + c++] = x;
                    if (++i >= l1 || ++j >= m) break;
                    x = ld_src(L + i, Llist);
                    y = __ldg(R + j);
                }
            }
        }
    }
    uint32_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total > cap) return total;
    __syncwarp();
    const uint32_t base = incl - c;
    for (uint32_t k = 0; k < c; ++k) out[base + k] = tmp[l0 + k];
    __syncwarp();
    if (kWeigh) *W = weigh_list(out, total, out_pw, q, approx, lane);
    return total;
}

// The filter of filter_list against a row without a bitmap: a warp merge (the row
// read once in coalesced 32-entry windows, each located among the list window's
// entries by a shuffle search) or one binary search per list entry, whichever the
// sizes make cheaper.
template <bool kWeigh>
__device__ AGIS_COLD uint32_t filter_merge_search(const int32_t *L, uint32_t n, const int32_t *R, int64_t m,
                                                  const int32_t *tau_s, int tau_n, int32_t *out, uint64_t *out_pw,
                                                  uint32_t cap, const uint64_t *q, bool approx, uint64_t *W,
                                                  int lane)
{
    uint32_t cnt = 0;
    uint64_t carry = 0;
    int lg = 1;
    while ((1ll << lg) < m + 1) ++lg;
    const bool merge = ((int64_t)n + m + 31) / 32 <= (((int64_t)n + 31) / 32) * lg;
    int64_t rpos = 0;
    for (uint32_t base = 0; base < n; base += 32) {
        const uint32_t idx = base + lane;
        const bool valid = idx < n;
        const int32_t x = valid ? L[idx] : 0x7fffffff;
        bool ok = valid;
        for (int j = 0; j < tau_n; ++j) ok &= (x != tau_s[j]);
        if (merge) {
            const int last = (n - base) >= 32 ? 31 : (int)(n - base - 1);
            const int32_t x_last = __shfl_sync(kFull, x, last);
            uint32_t found = 0;
            for (;;) {
                const bool rvalid = rpos + lane < m;
                const int32_t rv = rvalid ? __ldg(R + rpos + lane) : 0x7fffffff;
                // position of rv among the window's entries (lanes 0..last, ascending)
                int lo = 0, len = last + 1;
                while (len > 1) {
                    const int half = len >> 1;
                    const int32_t xv = __shfl_sync(kFull, x, lo + half);
                    if (xv <= rv) lo += half;
                    len -= half;
                }
                const int32_t xlo = __shfl_sync(kFull, x, lo);
                uint32_t bit = (rvalid && xlo == rv) ? (1u << lo) : 0u;
                for (int o = 16; o > 0; o >>= 1) bit |= __shfl_xor_sync(kFull, bit, o);
                found |= bit;
                const int c = __popc(__ballot_sync(kFull, rvalid && rv <= x_last));
                rpos += c;
                if (c < 32) break;
            }
            ok = ok && ((found >> lane) & 1u);
        } else if (ok) {
            ok = row_find(R, m, x) >= 0;
        }
        const uint64_t w = (kWeigh && ok) ? (approx ? __ldg(q + x) : 1u) : 0u;
        emit_window<kWeigh>(ok, x, w, out, out_pw, cap, cnt, carry, lane);
        if (cnt > cap) return cnt;
    }
    if (kWeigh) *W = carry;
    return cnt;
}

template <bool kWeigh>
__device__ uint32_t filter_list(const int32_t *L, bool Llist, uint32_t n, const int32_t *R, int64_t m,
                                const uint32_t *Rbits, const int32_t *tau_s, int tau_n, int32_t *out,
                                uint64_t *out_pw, uint32_t cap, const uint64_t *q, bool approx, uint64_t *W,
                                int lane)
{
    uint32_t cnt = 0;
    uint64_t carry = 0;
    // tmp: the id staging of the per-lane merge lives in the (not yet written)
    // running-weight array of out's list, room for 2 * cap ids
    if (R && n >= 256 && m >= 256 && n <= 2 * cap && (!Rbits || m < (int64_t)AGIS_MERGE_RATIO * n))
        return filter_lane_merge<kWeigh>(L, Llist, n, R, m, tau_s, tau_n, out, reinterpret_cast<int32_t *>(out_pw),
                                         out_pw, cap, q, approx, W, lane);
    if (Rbits || !R) {
        // Survivor ids first: 16-byte loads of four consecutive entries per lane,
        // kGroups groups of 128 entries per iteration, so 4 * kGroups bitmap probes
        // per lane are in flight together; the survivors' weights are gathered afterwards in
        // a pass over the (shorter) survivor list.  Loads start at the 16-byte
        // block holding L[0] and may read up to three entries past L[n-1] (the row
        // and list buffers are padded for that); such entries are masked out.
        const uint32_t mis = (uint32_t)(((uintptr_t)L & 15u) >> 2);
        const int32_t *La = L - mis;
        const uint32_t total = n + mis;
        for (uint32_t base = 0; base < total; base += 128 * kGroups) {
            int4 v[kGroups];
#pragma unroll
            for (int gi = 0; gi < kGroups; ++gi) {
                const uint32_t k = base + 128 * gi + 4 * lane;
                v[gi] = k < total ? ld_src(reinterpret_cast<const int4 *>(La + k), Llist) : make_int4(0, 0, 0, 0);
            }
            unsigned okm[kGroups];
#pragma unroll
            for (int gi = 0; gi < kGroups; ++gi) {
                const int64_t i0 = (int64_t)(base + 128 * gi + 4 * lane) - mis;
                const int32_t e4[4] = {v[gi].x, v[gi].y, v[gi].z, v[gi].w};
                unsigned mk = 0;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    bool ok = i0 + e >= 0 && i0 + e < (int64_t)n;
                    for (int j = 0; j < tau_n; ++j) ok = ok && (e4[e] != tau_s[j]);
                    if (Rbits) ok = ok && bit_test(Rbits, e4[e]);
                    mk |= (ok ? 1u : 0u) << e;
                }
                okm[gi] = mk;
            }
#pragma unroll
            for (int gi = 0; gi < kGroups; ++gi) {
                const uint32_t c = __popc(okm[gi]);
                uint32_t incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += t;
                }
                uint32_t pos = cnt + incl - c;
                const int32_t e4[4] = {v[gi].x, v[gi].y, v[gi].z, v[gi].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if ((okm[gi] >> e) & 1u) {
                        if (pos < cap) out[pos] = e4[e];
                        ++pos;
                    }
                }
                cnt += __shfl_sync(kFull, incl, 31);
            }
            if (cnt > cap) return cnt;         // list full: the caller takes the list-free path
        }
        if (kWeigh) {
            __syncwarp();
            for (uint32_t b = 0; b < cnt; b += 64) {
                int32_t x[2];
                uint64_t w[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const uint32_t idx = b + 32 * u + lane;
                    x[u] = idx < cnt ? out[idx] : 0;
                }
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    w[u] = (b + 32 * u + lane < cnt) ? (approx ? __ldg(q + x[u]) : 1u) : 0u;
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const uint64_t incl = warp_incl_scan(w[u], lane);
                    const uint32_t idx = b + 32 * u + lane;
                    if (idx < cnt) out_pw[idx] = carry + incl;
                    carry += __shfl_sync(kFull, incl, 31);
                }
            }
            *W = carry;
        }
        return cnt;
    }
    return filter_merge_search<kWeigh>(L, n, R, m, tau_s, tau_n, out, out_pw, cap, q, approx, W, lane);
}

// The list-free scan of a several-backward step whose survivors overflow the
// warp's list: the anchor row is filtered window by window, the running weight of
// every 32nd part of the windows is kept one per lane, and after the draw only the
// part holding r is filtered again.  Returns W (0: empty S or zero weight) and sets
// the drawn vertex v, its weight qv and the survivor count nsurv.
__device__ AGIS_COLD uint64_t list_free_draw(const GraphView &g, const DevStep &S, const int32_t *tau_s, int i,
                                             int64_t a_start, int64_t da, const RowRef *rows, int n_filter,
                                             uint64_t t, uint64_t seed, int lane, int32_t &v, uint64_t &qv,
                                             uint64_t &nsurv)
{
    const int64_t nwin = (da + 31) >> 5;
    const int64_t bsz = (nwin + 31) >> 5;              // windows per bucket
    uint64_t running = 0, bucket_end = 0;
    nsurv = 0;
    // last window kept in registers (most rows need a single window)
    uint64_t last_before = 0, last_incl = 0, last_w = 0;
    int32_t last_x = -1;
    constexpr int U = 4;       // windows whose loads are in flight together
    for (int64_t w0 = 0; w0 < nwin; w0 += U) {
        bool okv[U];
        int32_t xv[U];
        uint64_t wtv[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            wtv[u] = window_weight(g, S, tau_s, i, a_start, da, (w0 + u) * 32 + lane, rows, n_filter, okv[u], xv[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t w = w0 + u;
            if (w >= nwin) break;
            nsurv += __popc(__ballot_sync(kFull, okv[u]));
            const uint64_t incl = warp_incl_scan(wtv[u], lane);
            const uint64_t wtot = __shfl_sync(kFull, incl, 31);
            last_before = running;
            last_incl = incl;
            last_w = wtv[u];
            last_x = xv[u];
            running += wtot;
            if ((w + 1) % bsz == 0 || w == nwin - 1) {
                if (lane == (int)(w / bsz)) bucket_end = running;
            }
        }
    }
    const uint64_t W = running;
    if (W == 0) return 0;
    const uint64_t r = draw_below(W, t, (uint64_t)(i + 1), kStreamTrial, seed);
    if (r >= last_before) {
        const bool hit = last_w > 0 && last_before + last_incl > r;
        const int src = __ffs(__ballot_sync(kFull, hit)) - 1;
        v = __shfl_sync(kFull, last_x, src);
        qv = __shfl_sync(kFull, last_w, src);
    } else {
        const int64_t nbuck = (nwin + bsz - 1) / bsz;
        const int b = __ffs(__ballot_sync(kFull, lane < nbuck && bucket_end > r)) - 1;
        const uint64_t prev = __shfl_sync(kFull, bucket_end, b > 0 ? b - 1 : 0);
        uint64_t run2 = b > 0 ? prev : 0;
        const int64_t w_end = (b + 1) * bsz < nwin ? (b + 1) * bsz : nwin;
        for (int64_t w = (int64_t)b * bsz; w < w_end; ++w) {
            bool ok;
            int32_t x;
            const uint64_t wt = window_weight(g, S, tau_s, i, a_start, da, w * 32 + lane, rows, n_filter, ok, x);
            const uint64_t incl = warp_incl_scan(wt, lane);
            const uint64_t wtot = __shfl_sync(kFull, incl, 31);
            if (run2 + wtot > r) {
                const bool hit = wt > 0 && run2 + incl > r;
                const int src = __ffs(__ballot_sync(kFull, hit)) - 1;
                v = __shfl_sync(kFull, x, src);
                qv = __shfl_sync(kFull, wt, src);
                break;
            }
            run2 += wtot;
        }
    }
    return W;
}

// Alg. 3 for trial t of query Q; all 32 lanes call it together.  tau_s is the
// warp's shared-memory copy of the trajectory.
// Anchor draw: the drawn v must also be a neighbour of every backward vertex other
// than the anchor (jb); lane b tests backward vertex b.
__device__ __forceinline__ bool closes_all(const GraphView &g, const DevStep &S, const int32_t *tau_s, int jb,
                                           int32_t v, int lane)
{
    bool ok = true;
    if (lane < S.nb && S.back[lane] != jb) {
        const int32_t u = tau_s[S.back[lane]];
        const uint32_t *ub = bits_of(g, u);
        const int64_t s0 = __ldg(g.off + u);
        ok = ub ? bit_test(ub, v) : row_find(g.cols + s0, __ldg(g.off + u + 1) - s0, v) >= 0;
    }
    return __all_sync(kFull, ok);
}

// sector model of the closing checks: per other backward vertex, its offsets and one
// membership search in its row
__device__ __forceinline__ uint64_t closing_sectors(const GraphView &g, const DevStep &S, const int32_t *tau_s,
                                                    int jb)
{
    uint64_t s = 0;
    for (int b = 0; b < S.nb; ++b) {
        if (S.back[b] == jb) continue;
        const int32_t u = tau_s[S.back[b]];
        s += 1 + sec_search(__ldg(g.off + u + 1) - __ldg(g.off + u), 4);
    }
    return s;
}

// The streamed and survey counts are warp-uniform and kept in the warp's shared
// words wsec[0..1] (lane 0 adds to them) to spare registers; sec stays in registers.
#define STORE_SECTORS(o) do { (o).sectors = sec; (o).streamed = wsec[0]; (o).survey = wsec[1]; } while (0)
#define ADD_ST(v) do { if (lane == 0) wsec[0] += (v); } while (0)
#define ADD_SV(v) do { if (lane == 0) wsec[1] += (v); } while (0)

// kStagedTop: the first two levels of the step-1 search come from the CTA's staged
// splitters `top` (the main kernel); without them the search reads the prefix only.
template <bool kAnchor, bool kStagedTop = true>
__device__ TrialOut run_trial(const GraphView &g, const DevQuery &Q, uint64_t t, int32_t *tau_s,
                              const WarpSets &ws, const uint64_t *top, uint64_t *wsec, RowRef *rows, int lane)
{
    TrialOut out{0.0, 0, 0, 0, 0};
    double X = 1.0;
    uint64_t sec = 0;      // model sectors (streamed part and survey count in wsec)
    if (lane == 0) wsec[0] = wsec[1] = 0;
    int cur = -1;          // scratch list holding S of the previous step (-1: none)
    uint32_t n_cur = 0;
    if (lane < kMaxK) tau_s[lane] = -1;
    __syncwarp();
    for (int i = 0; i < Q.k; ++i) {
        const DevStep &S = Q.step[i];
        uint64_t W = 0, qv = 0;
        int32_t v = -1;
        STEP_T0
        // the anchor draw proposes from the shortest backward row (first on ties) and
        // checks the closing edges afterwards, instead of building S
        const bool anch = kAnchor && i > 0 && S.nb >= 2 && (Q.flags & kFlagAnchor);
        int jb = i > 0 ? S.back[0] : 0;
        if (anch) {
            int64_t best = -1;
            for (int b = 0; b < S.nb; ++b) {
                const int32_t u = tau_s[S.back[b]];
                const int64_t len = __ldg(g.off + u + 1) - __ldg(g.off + u);
                if (best < 0 || len < best) { best = len; jb = S.back[b]; }
            }
        }
        // a single-backward (or anchor-draw) step searches its row's prefix when it
        // has one (always under f_uniform, whose prefix is the position)
        bool direct = false;
        const uint64_t *Prow = nullptr;
        if (i > 0 && (S.nb == 1 || anch)) {
            if (!S.approx) {
                direct = true;
            } else if (S.pref) {
                const int32_t a = tau_s[jb];
                if (S.rp_mode == 1) {
                    Prow = S.pref + __ldg(g.off + a);
                    direct = true;
                } else {
                    const int64_t b = __ldg(g.rp_base + a);
                    if (b >= 0) {
                        Prow = S.pref + b;
                        direct = true;
                    }
                }
            }
        }
        if (i == 0) {
            // ---- step 1: the whole vertex set
            W = Q.W1;
            sec += sec_search(g.nv + 1, 8) + (S.approx ? 1 : 0);
            ADD_SV(sec_search(g.nv + 1, 8) + (S.approx ? 1 : 0));
            if (W == 0) { STORE_SECTORS(out); return out; }
            const uint64_t r = draw_below(W, t, 1, kStreamTrial, Q.seed);
            const uint64_t *P = S.approx ? S.pref : (const uint64_t *)(g.off + 1);
            v = kStagedTop ? (int32_t)warp_find_top(P, g.nv, r, top, lane)
                           : (int32_t)warp_find(P, g.nv, r, 0u, 0, 0, nullptr, lane);
            qv = S.approx ? __ldg(S.q + v) : (uint64_t)(__ldg(g.off + v + 1) - __ldg(g.off + v));
            cur = -1;
            STEP_T1(0)
        } else if (direct) {
            // ---- one backward neighbour: S = N(a) \ tau (anchor draw: the proposal set)
            const int32_t a = tau_s[jb];
            const int64_t a_start = __ldg(g.off + a);
            const int64_t d = __ldg(g.off + a + 1) - a_start;
            {
                const uint64_t base = 1 + (uint64_t)(i - 1) * sec_search(d, 4) + 1 +
                                      (anch ? closing_sectors(g, S, tau_s, jb) : 0);
                sec += base + (S.approx ? sec_search(d, 8) + 1 : 0);
                ADD_SV(base + (S.dapprox ? sec_search(d, 8) + 1 : 0));
            }
            // trajectory members inside a's row (lane j checks tau_j): excluded by
            // vertex id, so a hub row needs one bitmap probe and no search
            bool member = false;
            int64_t xkey = -1;
            uint64_t xq = 0;
            const uint32_t *abits = bits_of(g, a);
            if (lane < i && lane != jb) {
                const int32_t m = tau_s[lane];
                member = abits ? bit_test(abits, m) : row_find(g.cols + a_start, d, m) >= 0;
                if (member) {
                    xkey = m;
                    xq = S.approx ? __ldg(S.q + m) : 1u;
                }
            }
            const uint32_t xmask = __ballot_sync(kFull, member);
            const uint64_t excl = warp_sum_u64(xq);
            const uint64_t *P = S.approx ? Prow : nullptr;
            const uint64_t total = d <= 0 ? 0 : (S.approx ? __ldg(P + d - 1) : (uint64_t)d);
            W = total - excl;
            if (W == 0) { STORE_SECTORS(out); return out; }
            const uint64_t r = draw_below(W, t, (uint64_t)(i + 1), kStreamTrial, Q.seed);
            const int64_t pos = warp_find(P, d, r, xmask, xkey, xq, g.cols + a_start, lane);
            v = __ldg(g.cols + a_start + pos);
            qv = S.approx ? __ldg(S.q + v) : 1u;
            cur = -1;
            if (anch && !closes_all(g, S, tau_s, jb, v, lane)) { STORE_SECTORS(out); return out; }
            STEP_T1(1)
        } else {
            // ---- several backward neighbours (or one, with no row-prefix table):
            //      intersect, anchored at the shortest row
            // lane b reads backward row b; the anchor is the shortest row, the first in
            // backward order on ties; the other rows go to the warp's rows[] in order
            int64_t my_start = 0, my_len = INT64_MAX;
            const uint32_t *my_bits = nullptr;
            if (lane < S.nb) {
                const int32_t u = tau_s[S.back[lane]];
                my_start = __ldg(g.off + u);
                my_len = __ldg(g.off + u + 1) - my_start;
                my_bits = bits_of(g, u);
            }
            int64_t da = my_len;
            int ai = lane;
            for (int o = 16; o > 0; o >>= 1) {
                const int64_t ol = __shfl_xor_sync(kFull, da, o);
                const int oa = __shfl_xor_sync(kFull, ai, o);
                if (ol < da || (ol == da && oa < ai)) { da = ol; ai = oa; }
            }
            const int64_t a_start = __shfl_sync(kFull, my_start, ai);
            uint64_t search_sec = 0, merge_st = 0, search_sv = 0;
            if (lane < S.nb && lane != ai) {
                rows[lane - (lane > ai ? 1 : 0)] = RowRef{my_start, my_len, my_bits};
                search_sec = row_check_sectors(da, my_len, merge_st, search_sv);
            }
            search_sec = warp_sum_u64(search_sec);
            merge_st = warp_sum_u64(merge_st);
            search_sv = warp_sum_u64(search_sv);
            const int n_other = S.nb - 1;
            __syncwarp();
            // an anchor draw filters only trajectory members here; the other rows are
            // checked for the drawn vertex alone
            const int n_filter = anch ? 0 : n_other;
            if (S.nb == 1 || anch) {
                // the cost model counts the method's single-backward draw, whichever way it runs
                const uint64_t base = 1 + (uint64_t)(i - 1) * sec_search(da, 4) + 1 +
                                      (anch ? closing_sectors(g, S, tau_s, jb) : 0);
                sec += base + (S.approx ? sec_search(da, 8) + 1 : 0);
                ADD_SV(base + (S.dapprox ? sec_search(da, 8) + 1 : 0));
            } else {
                const uint64_t scan = (uint64_t)((4 * da + 31) / 32);
                sec += (uint64_t)S.nb + scan + search_sec;
                ADD_ST(scan + merge_st);
                ADD_SV((uint64_t)S.nb + scan + search_sv);
            }
            // S of the previous step is reusable when this step's backward set is the
            // previous one plus the previous vertex: S_i = S_{i-1} & N(v_{i-1})
            const bool reuse = S.inc && cur >= 0 && !anch;
            const bool weigh = S.approx || !(Q.flags & kFlagPlainLists);
            const uint32_t n_src = reuse ? n_cur : (uint32_t)da;
            bool listed = false;
            int nxt = reuse ? 1 - cur : 0;
            uint32_t n = n_src;
            uint64_t Wl = 0;
            if (ws.cap > 0 && (reuse || da < 0x7fffffffll)) {
                const int32_t *src = reuse ? ws.xs[cur] : g.cols + a_start;
                const int tau_n = reuse ? 0 : i;
                const int passes = reuse ? 1 : (n_filter > 0 ? n_filter : 1);
                for (int pss = 0; pss < passes; ++pss) {
                    const int32_t *R = nullptr;
                    const uint32_t *Rb = nullptr;
                    int64_t m = 0;
                    if (reuse) {
                        const int32_t u = tau_s[i - 1];
                        R = g.cols + __ldg(g.off + u);
                        m = __ldg(g.off + u + 1) - __ldg(g.off + u);
                        Rb = bits_of(g, u);
                    } else if (n_filter > 0) {
                        R = g.cols + rows[pss].start;
                        m = rows[pss].len;
                        Rb = rows[pss].bits;
                    }
                    // The last pass forms the running weights of an f_approx list.  A
                    // position draw needs survivor ids alone, but only a query none of
                    // whose lists is weighted filters ids only: running both filter
                    // instances in one query cost more instruction fetch in this large
                    // kernel than the running weights save (cliques ran 2-5% slower),
                    // so such a query keeps counts in the weighted instance.
                    const bool last = pss == passes - 1;
                    if (last && weigh) {
                        n = filter_list<true>(src, reuse || pss > 0, n, R, m, Rb, tau_s, pss == 0 ? tau_n : 0, ws.xs[nxt],
                                              ws.pw[nxt], ws.cap, S.q, S.approx != 0, &Wl, lane);
                    } else {
                        n = filter_list<false>(src, reuse || pss > 0, n, R, m, Rb, tau_s, pss == 0 ? tau_n : 0, ws.xs[nxt],
                                               ws.pw[nxt], ws.cap, S.q, S.approx != 0, nullptr, lane);
                        if (!last) {
                            src = ws.xs[nxt];
                            nxt = 1 - nxt;
                        }
                    }
                    if (n > ws.cap) break;
                }
                __syncwarp();
                listed = n <= ws.cap;
                if (listed && !weigh) Wl = n;
            }
            if (listed) {
                if (S.approx && S.nb > 1 && !anch) sec += n;
                if (S.dapprox && S.nb > 1 && !anch) ADD_SV(n);
                W = Wl;
                cur = nxt;
                n_cur = n;
                if (W == 0) { STORE_SECTORS(out); return out; }
                const uint64_t r = draw_below(W, t, (uint64_t)(i + 1), kStreamTrial, Q.seed);
                // equal weights: the r-th survivor (r < W = n)
                const int64_t j = S.approx ? warp_find(ws.pw[cur], n, r, 0u, 0, 0, nullptr, lane, true) : (int64_t)r;
                v = ws.xs[cur][j];
                qv = S.approx ? ws.pw[cur][j] - (j > 0 ? ws.pw[cur][j - 1] : 0) : 1u;
                if (anch) {
                    cur = -1;
                    if (!closes_all(g, S, tau_s, jb, v, lane)) { STORE_SECTORS(out); return out; }
                }
                X = X * ((double)W / (double)qv);
                STEP_T1(reuse ? 3 : 2)
                __syncwarp();
                if (lane == 0) tau_s[i] = v;
                __syncwarp();
                continue;
            }
            cur = -1;
            uint64_t nsurv = 0;
            W = list_free_draw(g, S, tau_s, i, a_start, da, rows, n_filter, t, Q.seed, lane, v, qv, nsurv);
            if (S.approx && S.nb > 1 && !anch) sec += nsurv;
            if (S.dapprox && S.nb > 1 && !anch) ADD_SV(nsurv);
            if (W == 0) { STORE_SECTORS(out); return out; }
        }
        if (i > 0 && !direct) {
            STEP_T1(4)
            if (anch && !closes_all(g, S, tau_s, jb, v, lane)) { STORE_SECTORS(out); return out; }
        }
        X = X * ((double)W / (double)qv);
        __syncwarp();
        if (lane == 0) tau_s[i] = v;
        __syncwarp();
    }
    out.x = X;
    out.hit = 1;
    STORE_SECTORS(out);
    return out;
}
#undef STORE_SECTORS
#undef ADD_ST
#undef ADD_SV

// The fixed-order FP64 reduction of one tile's outputs xs[0, kTile) (zeros past its
// trials): per thread strided partial sums of x and x^2, then a tree over the
// threads; the sums end in red[0] and red2[0].  Both the main kernel and the tile
// reduction of scatter epochs use it, so a tile's sums never depend on the mode.
__device__ __forceinline__ void tile_fp64_sums(const double *xs, double *red, double *red2)
{
    {
        double s = 0.0, s2 = 0.0;
        for (int j = threadIdx.x; j < kTile; j += kBlock) {
            const double x = xs[j];
            s += x;
            s2 += x * x;
        }
        red[threadIdx.x] = s;
        red2[threadIdx.x] = s2;
    }
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[threadIdx.x] += red[threadIdx.x + w];
            red2[threadIdx.x] += red2[threadIdx.x + w];
        }
        __syncthreads();
    }
}

// Work items come from `items`, or, when it is null, are implicit: item j covers
// implicit_span tiles, trials [implicit_first + kTile implicit_span j, ...) of query 0
// up to implicit_count trials, and writes slots implicit_span j, ...  n_items_ptr[0]
// holds the number of items.
// kAnchor: the instance that can run anchor-draw queries (the other one compiles
// that code away; both give the same results for queries without the flag)
template <bool kDump, bool kAnchor>
__global__ void __launch_bounds__(kBlock, AGIS_MIN_BLOCKS) sample_kernel(GraphView g, const DevQuery *__restrict__ queries,
                                                        const WorkItem *__restrict__ items,
                                                        const uint32_t *__restrict__ n_items_ptr,
                                                        uint32_t *counter, uint64_t *tile_out,
                                                        DumpView dump, uint64_t implicit_first,
                                                        uint64_t implicit_count, uint32_t implicit_span,
                                                        char *scratch,
                                                        uint32_t scratch_cap)
{
    __shared__ DevQuery sq;
    __shared__ double xs[kMaxSpan * kTile];
    __shared__ double red[kBlock];
    __shared__ double red2[kBlock];
    __shared__ int32_t tau_s[kWarps][kMaxK];
    __shared__ uint64_t s_wsec[kWarps][2];
    __shared__ RowRef s_rows[kWarps][kMaxK - 1];
    __shared__ uint64_t s_top[kTopSplitters];
    __shared__ uint32_t s_item, s_next, s_hits[kMaxSpan];
    __shared__ unsigned long long s_sec[kMaxSpan][3];
    __shared__ int s_query, s_reload;
    __shared__ WorkItem s_it;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n_items = *n_items_ptr;
    // the warp's candidate lists (pointers kept in shared memory: warp-uniform values)
    __shared__ WarpSets s_ws[kWarps];
    if (lane == 0) {
        const size_t per = (size_t)scratch_cap * 2 * (sizeof(int32_t) + sizeof(uint64_t));
        const size_t stride = (per + 255) / 256 * 256;
        char *base = scratch + stride * ((size_t)blockIdx.x * kWarps + warp);
        WarpSets &w = s_ws[warp];
        w.cap = scratch ? scratch_cap : 0;
        w.xs[0] = (int32_t *)base;
        w.xs[1] = w.xs[0] + scratch_cap;
        w.pw[0] = (uint64_t *)(base + (size_t)scratch_cap * 2 * sizeof(int32_t));
        w.pw[1] = w.pw[0] + scratch_cap;
    }
    __syncwarp();
    const WarpSets &ws = s_ws[warp];
    if (threadIdx.x == 0) s_query = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t id = atomicAdd(counter, 1u);
            s_item = id;
            if (id < n_items) {
                WorkItem w;
                if (items) {
                    w = items[id];
                } else {
                    const uint64_t per = (uint64_t)kTile * implicit_span;
                    const uint64_t done = (uint64_t)id * per;
                    const uint64_t left = implicit_count - done;
                    w.query = 0;
                    w.count = (uint32_t)(left < per ? left : per);
                    w.first = implicit_first + done;
                    w.slot = (uint64_t)id * implicit_span;
                }
                s_it = w;
                s_reload = (int)w.query != s_query;
                s_query = (int)w.query;
            }
            s_next = 0;
            for (int t = 0; t < kMaxSpan; ++t) {
                s_hits[t] = 0;
                s_sec[t][0] = s_sec[t][1] = s_sec[t][2] = 0;
            }
        }
        __syncthreads();
        if (s_item >= n_items) break;
        const WorkItem it = s_it;
        if (s_reload) {
            // stage the query description in shared memory
            const int words = (int)(sizeof(DevQuery) / sizeof(uint32_t));
            const uint32_t *src = (const uint32_t *)(queries + it.query);
            uint32_t *dst = (uint32_t *)&sq;
            for (int j = threadIdx.x; j < words; j += kBlock) dst[j] = src[j];
            __syncthreads();
            const uint64_t *P = sq.step[0].approx ? sq.step[0].pref : (const uint64_t *)(g.off + 1);
            for (int k = threadIdx.x; k < kTopSplitters; k += kBlock) {
                const int64_t pos = top_pos(g.nv, k);
                s_top[k] = pos >= 0 ? __ldg(P + pos) : 0;
            }
        }
        const int ntile = (int)((it.count + kTile - 1) / kTile);
        for (int j = threadIdx.x; j < ntile * kTile; j += kBlock) xs[j] = 0.0;
        __syncthreads();
        for (;;) {
            uint32_t tt = 0;
            if (lane == 0) tt = atomicAdd(&s_next, 1u);
            tt = __shfl_sync(kFull, tt, 0);
            if (tt >= it.count) break;
            const uint64_t t = it.first + tt;
            const TrialOut r = run_trial<kAnchor>(g, sq, t, tau_s[warp], ws, s_top, s_wsec[warp], s_rows[warp], lane);
            if (lane == 0) {
                xs[tt] = r.x;
                if (r.hit) atomicAdd(&s_hits[tt / kTile], 1u);
                atomicAdd(&s_sec[tt / kTile][0], (unsigned long long)r.sectors);
                atomicAdd(&s_sec[tt / kTile][1], (unsigned long long)r.streamed);
                atomicAdd(&s_sec[tt / kTile][2], (unsigned long long)r.survey);
                if (kDump) {
                    const uint64_t d = t - dump.first;
                    if (dump.hit) dump.hit[d] = (uint8_t)r.hit;
                    if (dump.x) dump.x[d] = r.x;
                    if (dump.sectors) {
                        dump.sectors[3 * d] = r.sectors;
                        dump.sectors[3 * d + 1] = r.streamed;
                        dump.sectors[3 * d + 2] = r.survey;
                    }
                }
            }
            if (kDump && dump.emb && lane < kMaxK) dump.emb[(t - dump.first) * kMaxK + lane] = tau_s[warp][lane];
            __syncwarp();
        }
        __syncthreads();
        // fixed-order reduction of each tile: strided partial sums, then a tree
        for (int tl = 0; tl < ntile; ++tl) {
            tile_fp64_sums(xs + tl * kTile, red, red2);
            if (threadIdx.x == 0) {
                uint64_t *o = tile_out + kTileWords * ((uint64_t)it.slot + tl);
                o[0] = s_hits[tl];
                o[1] = s_sec[tl][0];
                o[2] = (uint64_t)__double_as_longlong(red[0]);
                o[3] = (uint64_t)__double_as_longlong(red2[0]);
                o[4] = s_sec[tl][1];
                o[5] = s_sec[tl][2];
            }
            __syncthreads();
        }
    }
}

// Scatter epochs (epochs of few tiles, e.g. a query's first Alg. 1 checkpoints, and
// the last grid-full of tiles of larger ones): in the main kernel one CTA runs a
// whole tile, 32 trials per warp in sequence, so such tiles take as long as 32 trials
// back to back on an almost idle GPU.  Here every warp of a full grid pulls single
// trials from the device counter (trial c is trial c mod kTile of item c / kTile;
// items are single tiles) and writes its output to per-trial buffers at index c;
// tile_reduce_kernel then forms each tile's sums with the main kernel's fixed-order
// reduction, so the results are the same bits.
template <bool kAnchor>
__global__ void __launch_bounds__(kBlock, AGIS_MIN_BLOCKS) scatter_kernel(GraphView g, const DevQuery *__restrict__ queries,
                                                         const WorkItem *__restrict__ items,
                                                         const uint32_t *__restrict__ n_items_ptr,
                                                         uint32_t *counter, ScatterView sv, char *scratch,
                                                         uint32_t scratch_cap)
{
    __shared__ DevQuery wq[kWarps];          // the warp's current query
    __shared__ int s_wq[kWarps];
    __shared__ int32_t tau_s[kWarps][kMaxK];
    __shared__ uint64_t s_wsec[kWarps][2];
    __shared__ RowRef s_rows[kWarps][kMaxK - 1];
    __shared__ WarpSets s_ws[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        const size_t per = (size_t)scratch_cap * 2 * (sizeof(int32_t) + sizeof(uint64_t));
        const size_t stride = (per + 255) / 256 * 256;
        char *base = scratch + stride * ((size_t)blockIdx.x * kWarps + warp);
        WarpSets &w = s_ws[warp];
        w.cap = scratch ? scratch_cap : 0;
        w.xs[0] = (int32_t *)base;
        w.xs[1] = w.xs[0] + scratch_cap;
        w.pw[0] = (uint64_t *)(base + (size_t)scratch_cap * 2 * sizeof(int32_t));
        w.pw[1] = w.pw[0] + scratch_cap;
        s_wq[warp] = -1;
    }
    __syncwarp();
    const WarpSets &ws = s_ws[warp];
    const uint32_t total = *n_items_ptr * (uint32_t)kTile;
    for (;;) {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(counter, 1u);
        c = __shfl_sync(kFull, c, 0);
        if (c >= total) break;
        const WorkItem it = items[c / kTile];
        const uint32_t local = c % kTile;
        if (local >= it.count) continue;
        if ((int)it.query != s_wq[warp]) {
            const int words = (int)(sizeof(DevQuery) / sizeof(uint32_t));
            const uint32_t *qsrc = (const uint32_t *)(queries + it.query);
            uint32_t *dst = (uint32_t *)&wq[warp];
            for (int j = lane; j < words; j += 32) dst[j] = qsrc[j];
            if (lane == 0) s_wq[warp] = (int)it.query;
            __syncwarp();
        }
        const TrialOut r = run_trial<kAnchor, false>(g, wq[warp], it.first + local, tau_s[warp], ws, nullptr,
                                                     s_wsec[warp], s_rows[warp], lane);
        if (lane == 0) {
            const uint64_t k = c;          // = item * kTile + trial within the tile
            sv.x[k] = r.x;
            sv.hit[k] = (uint8_t)r.hit;
            sv.sec[3 * k] = r.sectors;
            sv.sec[3 * k + 1] = r.streamed;
            sv.sec[3 * k + 2] = r.survey;
        }
        __syncwarp();
    }
}

// One CTA per item (tile) of a scatter epoch: the tile's hit and sector totals and its
// fixed-order FP64 sums, written to its output slot as the main kernel writes them.
__global__ void __launch_bounds__(kBlock) tile_reduce_kernel(const WorkItem *__restrict__ items,
                                                             const uint32_t *__restrict__ n_items_ptr, ScatterView sv,
                                                             uint64_t *tile_out)
{
    __shared__ double xs[kTile];
    __shared__ double red[kBlock];
    __shared__ double red2[kBlock];
    __shared__ unsigned long long s_cnt[4];
    if (blockIdx.x >= *n_items_ptr) return;
    const WorkItem it = items[blockIdx.x];
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
    unsigned long long h = 0, s0 = 0, s1 = 0, s2 = 0;
    for (int j = threadIdx.x; j < kTile; j += kBlock) {
        const bool in = (uint32_t)j < it.count;
        xs[j] = in ? sv.x[base + j] : 0.0;
        if (in) {
            h += sv.hit[base + j];
            s0 += sv.sec[3 * (base + j)];
            s1 += sv.sec[3 * (base + j) + 1];
            s2 += sv.sec[3 * (base + j) + 2];
        }
    }
    atomicAdd(&s_cnt[0], h);
    atomicAdd(&s_cnt[1], s0);
    atomicAdd(&s_cnt[2], s1);
    atomicAdd(&s_cnt[3], s2);
    __syncthreads();
    tile_fp64_sums(xs, red, red2);
    if (threadIdx.x == 0) {
        uint64_t *o = tile_out + kTileWords * it.slot;
        o[0] = s_cnt[0];
        o[1] = s_cnt[1];
        o[2] = (uint64_t)__double_as_longlong(red[0]);
        o[3] = (uint64_t)__double_as_longlong(red2[0]);
        o[4] = s_cnt[2];
        o[5] = s_cnt[3];
    }
}

}  // namespace

const void *scatter_function(bool anchor)
{
    return anchor ? (const void *)scatter_kernel<true> : (const void *)scatter_kernel<false>;
}

const void *tile_reduce_function() { return (const void *)tile_reduce_kernel; }

int sampler_occupancy(int *blocks_per_sm)
{
    return cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sample_kernel<false, false>,
                                                                    kBlock, 0));
}

// The kernel instances, for the launch code in launch.cu: the dump instance, the
// anchor-capable one, and the plain one.
const void *sampler_function(bool dump, bool anchor)
{
    if (dump) return (const void *)sample_kernel<true, true>;
    return anchor ? (const void *)sample_kernel<false, true> : (const void *)sample_kernel<false, false>;
}

}  // namespace agis

extern "C" int agis_step_timers(uint64_t *out16, int reset)
{
    if (!out16) return AGIS_ERR_ARG;
    AGIS_CUDA_TRY(cudaMemcpyFromSymbol(out16, agis::g_step_timers, 16 * sizeof(uint64_t)));
    if (reset) {
        static const uint64_t zero[16] = {0};
        AGIS_CUDA_TRY(cudaMemcpyToSymbol(agis::g_step_timers, zero, sizeof(zero)));
    }
    return AGIS_OK;
}
