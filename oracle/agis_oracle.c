/*
 * agis_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of AGIS's structure-informed
 * neighbour sampling for approximate pattern counting (Lee & Lee, "AGIS: Fast
 * Approximate Graph Pattern Mining with Structure-Informed Sampling", PVLDB 19(2),
 * arXiv 2601.01388).  It exists so that the CUDA library can be checked against
 * something obviously correct.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never does.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Every function cites the passage it follows.  Readings of points the paper leaves
 * open are marked READING and are the same ones the design notes list:
 *   R1  counted quantity = embeddings C(G,P) (Sec. 2.1), automorphisms included;
 *   R2  E^{>=2hop} in the decision function uses edges of E_P (Def. decision function);
 *   R3  Alg. 2 ties go to the smallest pattern-vertex id;
 *   R4  C_v is sampled from d(v) uniform ordered distinct neighbour pairs, floored
 *       at c_min; d(v) < 2 gives c_min (Sec. 4.4);
 *   R5  f_approx weights are quantised to integers per (graph, step config) so that
 *       draws are exact; intended zeros (d(v)-|B| < |F1|) stay zero (Thm. 2 keeps the
 *       estimator unbiased for any positive weights on the reachable set);
 *   R6  draws: 128 random bits U from Philox4x64-10, r = floor(U*W / 2^128), the
 *       chosen vertex is the first candidate (ascending id) whose inclusive running
 *       weight exceeds r;
 *   R7  Alg. 1 is evaluated at whole-chunk checkpoints (Sec. 5.4 "every fixed number
 *       of iterations"), population variance, clamped at 0.
 *
 * Compile: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_MAXK 8
#define ORC_STREAM_TRIAL 1u
#define ORC_STREAM_CC 2u

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Philox4x64-10, from its definition in Salmon, Moraes, Dror & Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 64x64->128
 * multiplies with the round-key bumped by the Weyl constants between rounds.    */
/* ------------------------------------------------------------------------ */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        u128 p0 = (u128)M0 * x0;
        u128 p1 = (u128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* READING R6: r = floor(U * W / 2^128), U = out[1]*2^64 + out[0] of the block
 * keyed (seed, 0) at counter (a, b, stream, 0). */
uint64_t orc_draw_below(uint64_t W, uint64_t a, uint64_t b, uint64_t stream, uint64_t seed)
{
    uint64_t ctr[4] = {a, b, stream, 0}, key[2] = {seed, 0}, o[4];
    orc_philox4x64_10(ctr, key, o);
    u128 lo = (u128)o[0] * W;
    u128 hi = (u128)o[1] * W;
    u128 s = hi + (lo >> 64);
    return (uint64_t)(s >> 64);
}

/* ------------------------------------------------------------------------ */
/* Pattern analysis: matching order (Alg. 2), hop groups, auxiliary arrays
 * A^pi = {B, F1, F2, I_eff} (Def. auxiliary arrays), Certainty and D^pi
 * (Def. decision function), |Aut(P)| by brute force.                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t k;
    int32_t order[ORC_MAXK];        /* pi: order[i] is the pattern vertex u_{i+1}   */
    int32_t nback[ORC_MAXK];        /* |B[i]|                                        */
    int32_t back[ORC_MAXK][ORC_MAXK];/* step indices j < i of the backward neighbours */
    int32_t f1[ORC_MAXK], i1[ORC_MAXK], ieff[ORC_MAXK], f2[ORC_MAXK];
    double certainty[ORC_MAXK];
    int64_t aut;
} orc_plan;

static int popc(unsigned x) { int c = 0; while (x) { c += x & 1u; x >>= 1; } return c; }

/* Terms of the unsampled sub-pattern P_i (Eq. Pi) seen from vertex u: BFS over the
 * vertex set U (bitmask, contains u) gives hop levels; F1 = edges hop0-hop1,
 * I1 = edges inside hop 1, I_eff = spanning-forest size of the graph formed by I1
 * (|V_ind| - #components), F2 = edges hop1-hop2, V2/E2 = the ">= 2 hop" vertex and
 * edge counts of the decision function (E2 counts edges of E_P, READING R2). */
static void hop_terms(int k, const unsigned adj[], unsigned U, int u,
                      int *f1, int *i1, int *ieff, int *f2, int *v2, int *e2)
{
    int dist[ORC_MAXK];
    for (int x = 0; x < k; ++x) dist[x] = -1;
    dist[u] = 0;
    int queue[ORC_MAXK], qh = 0, qt = 0;
    queue[qt++] = u;
    while (qh < qt) {
        int x = queue[qh++];
        for (int y = 0; y < k; ++y)
            if ((adj[x] >> y & 1u) && (U >> y & 1u) && dist[y] < 0) {
                dist[y] = dist[x] + 1;
                queue[qt++] = y;
            }
    }
    int cf1 = 0, ci1 = 0, cf2 = 0;
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b) {
            if (!(adj[a] >> b & 1u) || !(U >> a & 1u) || !(U >> b & 1u)) continue;
            int da = dist[a], db = dist[b];
            if (da < 0 || db < 0) continue;
            int lo = da < db ? da : db, hi = da < db ? db : da;
            if (lo == 0 && hi == 1) cf1++;
            else if (lo == 1 && hi == 1) ci1++;
            else if (lo == 1 && hi == 2) cf2++;
        }
    /* spanning forest of (V_ind, I1): union-find */
    int parent[ORC_MAXK];
    for (int x = 0; x < k; ++x) parent[x] = x;
    unsigned vind = 0;
    int forest = 0;
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b) {
            if (!(adj[a] >> b & 1u) || dist[a] != 1 || dist[b] != 1) continue;
            if (!(U >> a & 1u) || !(U >> b & 1u)) continue;
            vind |= (1u << a) | (1u << b);
            int ra = a, rb = b;
            while (parent[ra] != ra) ra = parent[ra];
            while (parent[rb] != rb) rb = parent[rb];
            if (ra != rb) { parent[ra] = rb; forest++; }
        }
    (void)vind;
    int cv2 = 0, ce2 = 0;
    unsigned V2 = 0;
    for (int x = 0; x < k; ++x)
        if ((U >> x & 1u) && dist[x] >= 2) { cv2++; V2 |= 1u << x; }
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b)
            if ((adj[a] >> b & 1u) && ((V2 >> a & 1u) || (V2 >> b & 1u))) ce2++;
    *f1 = cf1; *i1 = ci1; *ieff = forest; *f2 = cf2; *v2 = cv2; *e2 = ce2;
}

static int64_t count_automorphisms(int k, const unsigned adj[])
{
    int perm[ORC_MAXK], used[ORC_MAXK] = {0};
    int64_t count = 0;
    /* iterative DFS over all k! permutations, checking edge preservation */
    int depth = 0;
    int next[ORC_MAXK + 1];
    next[0] = 0;
    while (depth >= 0) {
        if (depth == k) {
            int ok = 1;
            for (int a = 0; a < k && ok; ++a)
                for (int b = 0; b < k; ++b)
                    if ((adj[a] >> b & 1u) && !(adj[perm[a]] >> perm[b] & 1u)) { ok = 0; break; }
            count += ok;
            depth--;
            if (depth >= 0) used[perm[depth]] = 0;
            continue;
        }
        int c = next[depth];
        while (c < k && used[c]) c++;
        if (c >= k) {
            depth--;
            if (depth >= 0) used[perm[depth]] = 0;
            continue;
        }
        perm[depth] = c;
        used[c] = 1;
        next[depth] = c + 1;
        depth++;
        next[depth] = 0;
    }
    return count;
}

/* Returns 0 on success, -1 on an invalid pattern (k outside 2..8, bad or repeated
 * edge, self-loop, disconnected). */
int orc_plan_compile(int32_t k, int32_t ne, const int32_t *edges, orc_plan *out)
{
    if (k < 2 || k > ORC_MAXK || ne < 1 || ne > k * (k - 1) / 2) return -1;
    unsigned adj[ORC_MAXK] = {0};
    for (int e = 0; e < ne; ++e) {
        int a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b) return -1;
        if (adj[a] >> b & 1u) return -1;
        adj[a] |= 1u << b;
        adj[b] |= 1u << a;
    }
    /* connectivity */
    unsigned seen = 1u, frontier = 1u;
    while (frontier) {
        unsigned nf = 0;
        for (int x = 0; x < k; ++x) if (frontier >> x & 1u) nf |= adj[x];
        nf &= ~seen;
        seen |= nf;
        frontier = nf;
    }
    if (seen != (1u << k) - 1u) return -1;

    memset(out, 0, sizeof(*out));
    out->k = k;
    const unsigned all = (1u << k) - 1u;
    unsigned in_pi = 0;
    /* Alg. 2: greedy order maximising s(u) = |F1| + |I1| of P_i seen from u. */
    for (int i = 0; i < k; ++i) {
        unsigned cand;
        if (i == 0) cand = all;
        else {
            cand = 0;
            for (int x = 0; x < k; ++x) if (in_pi >> x & 1u) cand |= adj[x];
            cand &= ~in_pi;
        }
        int best = -1, best_s = -1;
        for (int u = 0; u < k; ++u) {           /* ascending id: ties keep the smallest (R3) */
            if (!(cand >> u & 1u)) continue;
            int f1, i1, ie, f2, v2, e2;
            hop_terms(k, adj, all & ~in_pi, u, &f1, &i1, &ie, &f2, &v2, &e2);
            int s = f1 + i1;
            if (s > best_s) { best_s = s; best = u; }
        }
        out->order[i] = best;
        in_pi |= 1u << best;
    }
    /* Auxiliary arrays and Certainty per step. */
    unsigned sampled = 0;
    for (int i = 0; i < k; ++i) {
        int u = out->order[i];
        int nb = 0;
        for (int j = 0; j < i; ++j)
            if (adj[u] >> out->order[j] & 1u) out->back[i][nb++] = j;
        out->nback[i] = nb;
        unsigned Vi = all & ~sampled;          /* V_i: u_i and later vertices (Eq. Pi) */
        int f1, i1, ie, f2, v2, e2;
        hop_terms(k, adj, Vi, u, &f1, &i1, &ie, &f2, &v2, &e2);
        out->f1[i] = f1; out->i1[i] = i1; out->ieff[i] = ie; out->f2[i] = f2;
        out->certainty[i] = 1.0 - (double)(e2 - v2) / (double)popc(Vi);
        sampled |= 1u << u;
    }
    out->aut = count_automorphisms(k, adj);
    return 0;
}

/* D^pi(i) = [Certainty(i) >= beta]; mode 1 forces f_approx, mode 2 forces f_uniform
 * (the beta = -inf / +inf extremes of the beta sweep, Sec. 6). */
void orc_plan_decide(const orc_plan *p, int32_t mode, double beta, int32_t use_approx[ORC_MAXK])
{
    for (int i = 0; i < ORC_MAXK; ++i) {
        if (i >= p->k) { use_approx[i] = 0; continue; }
        if (mode == 1) use_approx[i] = 1;
        else if (mode == 2) use_approx[i] = 0;
        else use_approx[i] = p->certainty[i] >= beta;
    }
}

/* ------------------------------------------------------------------------ */
/* Graph preprocessing (Sec. 4.4).                                           */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int is_neighbour(const int64_t *off, const int32_t *cols, int32_t x, int32_t y)
{
    int64_t n = off[x + 1] - off[x];
    if (n <= 0) return 0;
    return bsearch(&y, cols + off[x], (size_t)n, sizeof(int32_t), cmp_i32) != NULL;
}

/* The ordered distinct pair (a, b) of row positions that the number
 * r in [0, d(d-1)) names: a = r / (d-1), b' = r mod (d-1), b = b' + [b' >= a]
 * (READING R4).  Exposed so that a test can enumerate it. */
void orc_cc_pair(uint64_t d, uint64_t r, uint64_t *a, uint64_t *b)
{
    uint64_t aa = r / (d - 1), bb = r % (d - 1);
    *a = aa;
    *b = bb + (bb >= aa ? 1u : 0u);
}

/* nsum[v] = sum of d(x) over x in N(v)  (numerator of the average neighbour degree);
 * hits[v] = number of the d(v) sampled neighbour pairs that are joined by an edge
 * (the sampled clustering coefficient, Sec. 4.4). */
void orc_graph_stats_range(int64_t nv, const int64_t *off, const int32_t *cols, uint64_t seed,
                           int64_t v0, int64_t v1, uint64_t *nsum, uint32_t *hits)
{
    (void)nv;
    for (int64_t v = v0; v < v1; ++v) {
        int64_t d = off[v + 1] - off[v];
        uint64_t s = 0;
        for (int64_t e = off[v]; e < off[v + 1]; ++e) {
            int32_t x = cols[e];
            s += (uint64_t)(off[x + 1] - off[x]);
        }
        nsum[v] = s;
        uint32_t h = 0;
        if (d >= 2) {
            for (int64_t j = 0; j < d; ++j) {
                uint64_t r = orc_draw_below((uint64_t)d * (uint64_t)(d - 1), (uint64_t)v,
                                            (uint64_t)j, ORC_STREAM_CC, seed);
                uint64_t a, b;
                orc_cc_pair((uint64_t)d, r, &a, &b);
                h += (uint32_t)is_neighbour(off, cols, cols[off[v] + (int64_t)a], cols[off[v] + (int64_t)b]);
            }
        }
        hits[v] = h;
    }
}

void orc_graph_stats(int64_t nv, const int64_t *off, const int32_t *cols, uint64_t seed,
                     uint64_t *nsum, uint32_t *hits)
{
    orc_graph_stats_range(nv, off, cols, seed, 0, nv, nsum, hits);
}

/* Eq. probability_function: T[F1] * T[I1] * T[F2] with
 *   T[F1] = binom(d - |B|, |F1|), T[I1] = C_v^{|I_eff|}, T[F2] = (nsum/d)^{|F2|}.
 * binom by the multiplicative recurrence, powers by repeated products, all in
 * IEEE double with the product order written here. */
double orc_weight(int64_t d, uint64_t nsum, uint32_t hits, double c_min,
                  int32_t b, int32_t f1, int32_t ie, int32_t f2)
{
    int64_t n = d - b;
    if (n < f1) return 0.0;
    double tf1 = 1.0;
    for (int j = 0; j < f1; ++j) {
        tf1 = tf1 * (double)(n - j);
        tf1 = tf1 / (double)(j + 1);
    }
    double cv = c_min;
    if (d >= 2) {
        cv = (double)hits / (double)d;
        if (cv < c_min) cv = c_min;
        if (cv > 1.0) cv = 1.0;
    }
    double ti = 1.0;
    for (int j = 0; j < ie; ++j) ti = ti * cv;
    double tf2 = 1.0;
    if (f2 > 0) {
        double base = (double)nsum / (double)d;
        for (int j = 0; j < f2; ++j) tf2 = tf2 * base;
    }
    return (tf1 * ti) * tf2;
}

/* READING R5: scale = K - E with E the binary exponent of max_v w(v) (frexp) and
 * K = 62 - ceil(log2(nv + 1)), so that any sum of quantised weights is < 2^62. */
int32_t orc_quant_shift(int64_t nv, const int64_t *off, const uint64_t *nsum,
                        const uint32_t *hits, double c_min, int32_t b, int32_t f1,
                        int32_t ie, int32_t f2)
{
    double wmax = 0.0;
    for (int64_t v = 0; v < nv; ++v) {
        double w = orc_weight(off[v + 1] - off[v], nsum[v], hits[v], c_min, b, f1, ie, f2);
        if (w > wmax) wmax = w;
    }
    int E = 0;
    if (wmax > 0.0) frexp(wmax, &E);
    int L = 0;
    while (L < 63 && ((uint64_t)1 << L) < (uint64_t)(nv + 1)) L++;
    return (62 - L) - E;
}

uint64_t orc_quantise(double w, int64_t d, int32_t b, int32_t f1, int32_t shift)
{
    if (d - b < f1) return 0;                 /* intended zero: no extension exists */
    double s = ldexp(w, shift);
    uint64_t q = (uint64_t)floor(s);
    return q < 1 ? 1 : q;
}

/* Whole quantised table of one configuration: q[v] for every vertex and the shift
 * used (a plain loop over orc_weight / orc_quantise). */
int32_t orc_weight_table(int64_t nv, const int64_t *off, const uint64_t *nsum, const uint32_t *hits,
                         double c_min, int32_t b, int32_t f1, int32_t ie, int32_t f2, uint64_t *q)
{
    int32_t shift = orc_quant_shift(nv, off, nsum, hits, c_min, b, f1, ie, f2);
    for (int64_t v = 0; v < nv; ++v) {
        int64_t d = off[v + 1] - off[v];
        q[v] = orc_quantise(orc_weight(d, nsum[v], hits[v], c_min, b, f1, ie, f2), d, b, f1, shift);
    }
    return shift;
}

/* ------------------------------------------------------------------------ */
/* One query: a plan, the distribution choice per step and the per-step
 * quantisation shifts.                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t nv, nnz;
    const int64_t *off;
    const int32_t *cols;
    const uint64_t *nsum;
    const uint32_t *hits;
    double c_min;
    uint64_t seed;
    orc_plan plan;
    int32_t use_approx[ORC_MAXK];
    int32_t wb[ORC_MAXK];  /* |B| in the weight's T[F1]: nback, or 0 on an orientation */
    int32_t anchor;        /* steps with several backward vertices use the anchor draw */
    int32_t shift[ORC_MAXK];
    uint64_t *cum1;       /* step-1 f_approx: inclusive running weight over v = 0..nv-1 */
    uint64_t W1;
    int32_t *cand;        /* candidate-set scratch, max degree entries */
    uint64_t *candq;
} orc_query;

static uint64_t step_weight(const orc_query *Q, int i, int32_t v)
{
    int64_t d = Q->off[v + 1] - Q->off[v];
    if (!Q->use_approx[i]) return i == 0 ? (uint64_t)d : 1u;   /* f_uniform (Sec. 5.3) */
    const orc_plan *p = &Q->plan;
    double w = orc_weight(d, Q->nsum[v], Q->hits[v], Q->c_min, Q->wb[i], p->f1[i],
                          p->ieff[i], p->f2[i]);
    return orc_quantise(w, d, Q->wb[i], p->f1[i], Q->shift[i]);
}

/* terms: which factors of Eq. probability_function are kept (bit 0 T[F1], bit 1
 * T[I1], bit 2 T[F2]; 0 = all three), the incremental versions of the Sec. 6.2
 * ablation.  A dropped factor is 1, i.e. its exponent in the step configuration is
 * zero (for T[F1]: binom(d-|B|, 0), which keeps d >= |B|). */
/* oriented: the CSR is a degree-ordered orientation (orc_orient) and the pattern a
 * clique.  Each clique is then one trajectory, every step intersects the out-rows
 * of all earlier vertices, and the weight takes |B| = 0 since no earlier vertex
 * lies in a later vertex's out-row (Sec. 5.4 orientation for cliques). */
orc_query *orc_query_create_ex(int64_t nv, const int64_t *off, const int32_t *cols,
                               const uint64_t *nsum, const uint32_t *hits, double c_min,
                               int32_t k, int32_t ne, const int32_t *edges,
                               int32_t mode, double beta, uint64_t seed, int32_t terms,
                               int32_t oriented, int32_t anchor)
{
    orc_query *Q = (orc_query *)calloc(1, sizeof(orc_query));
    if (!Q) return NULL;
    Q->anchor = anchor != 0;
    if (orc_plan_compile(k, ne, edges, &Q->plan) != 0) { free(Q); return NULL; }
    if (oriented && ne != k * (k - 1) / 2) { free(Q); return NULL; }
    /* T[F1] stays in every incremental version: without it a vertex of degree 0
     * would reach the nsum/d factor of T[F2] */
    if (terms < 0 || terms > 7 || (terms != 0 && !(terms & 1))) { free(Q); return NULL; }
    for (int i = 0; i < Q->plan.k; ++i) Q->wb[i] = oriented ? 0 : Q->plan.nback[i];
    if (terms != 0) {
        for (int i = 0; i < Q->plan.k; ++i) {
            if (!(terms & 1)) Q->plan.f1[i] = 0;
            if (!(terms & 2)) Q->plan.ieff[i] = 0;
            if (!(terms & 4)) Q->plan.f2[i] = 0;
        }
    }
    Q->nv = nv; Q->nnz = off[nv]; Q->off = off; Q->cols = cols; Q->nsum = nsum; Q->hits = hits;
    Q->c_min = c_min; Q->seed = seed;
    orc_plan_decide(&Q->plan, mode, beta, Q->use_approx);
    const orc_plan *p = &Q->plan;
    for (int i = 0; i < p->k; ++i)
        Q->shift[i] = Q->use_approx[i]
            ? orc_quant_shift(nv, off, nsum, hits, c_min, Q->wb[i], p->f1[i], p->ieff[i], p->f2[i])
            : 0;
    int64_t maxd = 1;
    for (int64_t v = 0; v < nv; ++v) if (off[v + 1] - off[v] > maxd) maxd = off[v + 1] - off[v];
    Q->cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)maxd);
    Q->candq = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)maxd);
    Q->cum1 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nv > 0 ? nv : 1));
    if (!Q->cand || !Q->candq || !Q->cum1) {
        free(Q->cand); free(Q->candq); free(Q->cum1); free(Q);
        return NULL;
    }
    uint64_t run = 0;
    for (int64_t v = 0; v < nv; ++v) {
        if (Q->use_approx[0]) run += step_weight(Q, 0, (int32_t)v);
        else run = (uint64_t)off[v + 1];
        Q->cum1[v] = run;
    }
    Q->W1 = run;
    return Q;
}

orc_query *orc_query_create_terms(int64_t nv, const int64_t *off, const int32_t *cols,
                                  const uint64_t *nsum, const uint32_t *hits, double c_min,
                                  int32_t k, int32_t ne, const int32_t *edges,
                                  int32_t mode, double beta, uint64_t seed, int32_t terms)
{
    return orc_query_create_ex(nv, off, cols, nsum, hits, c_min, k, ne, edges, mode, beta, seed, terms, 0, 0);
}

orc_query *orc_query_create(int64_t nv, const int64_t *off, const int32_t *cols,
                            const uint64_t *nsum, const uint32_t *hits, double c_min,
                            int32_t k, int32_t ne, const int32_t *edges,
                            int32_t mode, double beta, uint64_t seed)
{
    return orc_query_create_ex(nv, off, cols, nsum, hits, c_min, k, ne, edges, mode, beta, seed, 0, 0, 0);
}

/* The degree-ordered orientation of Sec. 5.4: u -> v is kept when d(u) < d(v), or
 * d(u) = d(v) and u < v.  off_out has nv + 1 entries and cols_out room for off[nv]
 * entries; rows keep their ascending order.  Returns the number of kept entries. */
int64_t orc_orient(int64_t nv, const int64_t *off, const int32_t *cols, int64_t *off_out, int32_t *cols_out)
{
    int64_t n = 0;
    off_out[0] = 0;
    for (int64_t u = 0; u < nv; ++u) {
        const int64_t du = off[u + 1] - off[u];
        for (int64_t j = off[u]; j < off[u + 1]; ++j) {
            const int32_t v = cols[j];
            const int64_t dv = off[v + 1] - off[v];
            if (du < dv || (du == dv && u < v)) cols_out[n++] = v;
        }
        off_out[u + 1] = n;
    }
    return n;
}

void orc_query_free(orc_query *Q)
{
    if (!Q) return;
    free(Q->cand); free(Q->candq); free(Q->cum1); free(Q);
}

void orc_query_info(const orc_query *Q, orc_plan *plan, int32_t use_approx[ORC_MAXK],
                    int32_t shift[ORC_MAXK], uint64_t *W1)
{
    *plan = Q->plan;
    memcpy(use_approx, Q->use_approx, sizeof(Q->use_approx));
    memcpy(shift, Q->shift, sizeof(Q->shift));
    *W1 = Q->W1;
}

/* Sectors of a search over L entries of w bytes: ceil(log2(ceil(L*w/32))) + 1,
 * one sector when the whole range fits in one. */
static uint64_t sec_search(int64_t L, int w)
{
    uint64_t bytes = (uint64_t)(L > 0 ? L : 1) * (uint64_t)w;
    if (bytes <= 32) return 1;
    uint64_t n = (bytes + 31) / 32;
    uint64_t lg = 0;
    while (((uint64_t)1 << lg) < n) lg++;
    return lg + 1;
}

/* Builds S_tau for step i (Alg. 3, candidate set) in ascending id order together
 * with the step weights; returns |S|. */
static int64_t build_candidates(const orc_query *Q, int i, const int32_t *tau, uint64_t *W)
{
    const orc_plan *p = &Q->plan;
    int32_t first = tau[p->back[i][0]];
    int64_t n = 0;
    uint64_t sum = 0;
    for (int64_t e = Q->off[first]; e < Q->off[first + 1]; ++e) {
        int32_t x = Q->cols[e];
        int in_tau = 0;
        for (int j = 0; j < i; ++j) if (tau[j] == x) { in_tau = 1; break; }
        if (in_tau) continue;
        int ok = 1;
        for (int b = 1; b < p->nback[i] && ok; ++b)
            ok = is_neighbour(Q->off, Q->cols, tau[p->back[i][b]], x);
        if (!ok) continue;
        uint64_t q = step_weight(Q, i, x);
        Q->cand[n] = x;
        Q->candq[n] = q;
        sum += q;
        n++;
    }
    *W = sum;
    return n;
}

/* Anchor draw, the alternative to building S_tau for a step with several backward
 * vertices: the proposal set is the row of one backward vertex, the anchor (the
 * shortest backward row, the first in backward order on ties), minus tau, with the
 * step's weights (q under f_approx, 1 under f_uniform).  The drawn vertex must then
 * be a neighbour of every other backward vertex (the closing edges), else the trial
 * returns 0.  Every extension in S_tau keeps a positive probability q / W, so Thm. 2
 * still gives an unbiased estimate; S_tau is never built.  Returns the anchor's
 * index in the backward list and fills cand/candq; *W is the proposal total. */
static int anchor_candidates(const orc_query *Q, int i, const int32_t *tau, uint64_t *W, int64_t *n_out)
{
    const orc_plan *p = &Q->plan;
    int a = 0;
    int64_t da = -1;
    for (int b = 0; b < p->nback[i]; ++b) {
        int32_t u = tau[p->back[i][b]];
        int64_t d = Q->off[u + 1] - Q->off[u];
        if (da < 0 || d < da) { da = d; a = b; }
    }
    int32_t anchor = tau[p->back[i][a]];
    int64_t n = 0;
    uint64_t sum = 0;
    for (int64_t e = Q->off[anchor]; e < Q->off[anchor + 1]; ++e) {
        int32_t x = Q->cols[e];
        int in_tau = 0;
        for (int j = 0; j < i; ++j) if (tau[j] == x) { in_tau = 1; break; }
        if (in_tau) continue;
        uint64_t q = step_weight(Q, i, x);
        Q->cand[n] = x;
        Q->candq[n] = q;
        sum += q;
        n++;
    }
    *W = sum;
    *n_out = n;
    return a;
}

static int closes_all(const orc_query *Q, int i, const int32_t *tau, int a, int32_t v)
{
    const orc_plan *p = &Q->plan;
    for (int b = 0; b < p->nback[i]; ++b)
        if (b != a && !is_neighbour(Q->off, Q->cols, tau[p->back[i][b]], v)) return 0;
    return 1;
}

/* Sector model of an anchor-draw step: the single-backward draw on the anchor row
 * plus, per other backward vertex, one offsets sector and one membership search.
 * Every sector of it is a random access, and the survey's count is the same (an
 * anchor step always reads its weights under f_approx). */
static void anchor_sectors(const orc_query *Q, int i, const int32_t *tau, int a, uint64_t sec[3])
{
    const orc_plan *p = &Q->plan;
    int32_t anchor = tau[p->back[i][a]];
    int64_t d = Q->off[anchor + 1] - Q->off[anchor];
    uint64_t s = 1 + (uint64_t)(i - 1) * sec_search(d, 4);
    if (Q->use_approx[i]) s += sec_search(d, 8) + 1;
    s += 1;
    for (int b = 0; b < p->nback[i]; ++b) {
        if (b == a) continue;
        int32_t u = tau[p->back[i][b]];
        s += 1 + sec_search(Q->off[u + 1] - Q->off[u], 4);
    }
    sec[0] += s;
    sec[2] += s;
}

/* Whether the cost model counts weight reads for step i.  A later step whose
 * configuration has |F1| = |I_eff| = |F2| = 0 gives every candidate of S_tau the
 * same quantised weight: each candidate is adjacent to the |B| backward vertices,
 * so binom(d - |B|, 0) = 1 for all of them (|B| is 0 on an orientation).  A draw
 * over equal weights is a draw of a position and needs no weight reads.  The
 * arithmetic below still weighs such steps with q; only the sector count differs. */
static int weights_read(const orc_query *Q, int i)
{
    const orc_plan *p = &Q->plan;
    if (!Q->use_approx[i]) return 0;
    if (i == 0) return 1;
    return p->f1[i] != 0 || p->ieff[i] != 0 || p->f2[i] != 0;
}

/* Algorithmic-sector model of one step (a count of 32-byte sectors the step must
 * touch with no reuse; see the design notes), added into sec[0]:
 *   step 1: search over the (nv+1)-entry running-weight array (+1 for q(v_1));
 *   later : one sector per backward vertex's offsets; one backward edge: i-1
 *           trajectory-membership searches in the row, a running-weight search in
 *           the row under f_approx (+1 for q(v)), one sector for the chosen entry;
 *           several: a scan of the shortest backward row; for each other backward
 *           row the cheaper of reading it once (a merge) and one membership search
 *           per scanned entry; one q gather per candidate under f_approx
 *           (weights_read: none where the weights are equal on S_tau).
 * sec[1] receives the streamed part of sec[0]: the scan of the shortest row and the
 * other rows read once; every other sector is a random access (searches, offsets,
 * gathers).  sec[2] receives the plain count of the method's reads with neither
 * saving: one membership search per scanned entry in every other backward row, and
 * the weight reads of every step that D(i) puts under f_approx, equal weights or
 * not. */
static void step_sectors(const orc_query *Q, int i, const int32_t *tau, int64_t nS, uint64_t sec[3])
{
    const orc_plan *p = &Q->plan;
    if (i == 0) {
        uint64_t s = sec_search(Q->nv + 1, 8) + (Q->use_approx[0] ? 1u : 0u);
        sec[0] += s;
        sec[2] += s;
        return;
    }
    int nb = p->nback[i];
    if (nb == 1) {
        int64_t d = Q->off[tau[p->back[i][0]] + 1] - Q->off[tau[p->back[i][0]]];
        uint64_t s = 1 + (uint64_t)(i - 1) * sec_search(d, 4) + 1;
        uint64_t w = sec_search(d, 8) + 1;
        sec[0] += s + (weights_read(Q, i) ? w : 0);
        sec[2] += s + (Q->use_approx[i] ? w : 0);
        return;
    }
    int a = 0;
    int64_t da = -1;
    for (int b = 0; b < nb; ++b) {
        int32_t v = tau[p->back[i][b]];
        int64_t d = Q->off[v + 1] - Q->off[v];
        if (da < 0 || d < da) { da = d; a = b; }
    }
    uint64_t scan = (uint64_t)((4 * da + 31) / 32);
    uint64_t s = (uint64_t)nb + scan, streamed = scan, survey = (uint64_t)nb + scan;
    for (int b = 0; b < nb; ++b) {
        if (b == a) continue;
        int32_t v = tau[p->back[i][b]];
        int64_t m = Q->off[v + 1] - Q->off[v];
        uint64_t read_once = (uint64_t)((4 * (m > 0 ? m : 1) + 31) / 32);
        uint64_t search_each = (uint64_t)da * sec_search(m, 4);
        if (read_once < search_each) {
            s += read_once;
            streamed += read_once;
        } else {
            s += search_each;
        }
        survey += search_each;
    }
    if (weights_read(Q, i)) s += (uint64_t)nS;
    if (Q->use_approx[i]) survey += (uint64_t)nS;
    sec[0] += s;
    sec[1] += streamed;
    sec[2] += survey;
}

/* Alg. 3 for trial t: returns X = prod_i W_i / q_i (the inverse of the trajectory's
 * probability) on success and 0 when a candidate set is empty or has zero weight.
 * tau receives the sampled vertices (-1 past a failure). */
double orc_trial(const orc_query *Q, uint64_t t, int32_t tau[ORC_MAXK], uint8_t *hit,
                 uint64_t sectors[3])
{
    const orc_plan *p = &Q->plan;
    for (int i = 0; i < ORC_MAXK; ++i) tau[i] = -1;
    double X = 1.0;
    uint64_t sec[3] = {0, 0, 0};
    *hit = 0;
    for (int i = 0; i < p->k; ++i) {
        uint64_t W, q;
        int32_t v;
        if (i == 0) {
            W = Q->W1;
            if (W == 0) { X = 0.0; step_sectors(Q, i, tau, 0, sec); goto done; }
            uint64_t r = orc_draw_below(W, t, 1, ORC_STREAM_TRIAL, Q->seed);
            int64_t lo = 0, hi = Q->nv - 1;          /* first v with cum1[v] > r */
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (Q->cum1[mid] > r) hi = mid; else lo = mid + 1;
            }
            v = (int32_t)lo;
            q = step_weight(Q, 0, v);
            step_sectors(Q, i, tau, 0, sec);
        } else if (Q->anchor && p->nback[i] >= 2) {
            int64_t n;
            int a = anchor_candidates(Q, i, tau, &W, &n);
            anchor_sectors(Q, i, tau, a, sec);
            if (n == 0 || W == 0) { X = 0.0; goto done; }
            uint64_t r = orc_draw_below(W, t, (uint64_t)(i + 1), ORC_STREAM_TRIAL, Q->seed);
            uint64_t run = 0;
            int64_t c = 0;
            for (c = 0; c < n; ++c) {
                run += Q->candq[c];
                if (run > r) break;
            }
            v = Q->cand[c];
            q = Q->candq[c];
            if (!closes_all(Q, i, tau, a, v)) { X = 0.0; goto done; }
        } else {
            int64_t n = build_candidates(Q, i, tau, &W);
            step_sectors(Q, i, tau, n, sec);
            if (n == 0 || W == 0) { X = 0.0; goto done; }
            uint64_t r = orc_draw_below(W, t, (uint64_t)(i + 1), ORC_STREAM_TRIAL, Q->seed);
            uint64_t run = 0;
            int64_t c = 0;
            for (c = 0; c < n; ++c) {
                run += Q->candq[c];
                if (run > r) break;
            }
            v = Q->cand[c];
            q = Q->candq[c];
        }
        X = X * ((double)W / (double)q);
        tau[i] = v;
    }
    *hit = 1;
done:
    for (int j = 0; j < 3; ++j) sectors[j] = sec[j];
    return X;
}

/* Per-trial dump over trials [first, first+count); sectors: 3 words per trial. */
void orc_trials(const orc_query *Q, uint64_t first, uint64_t count, int32_t *emb,
                uint8_t *hit, double *x, uint64_t *sectors)
{
    for (uint64_t c = 0; c < count; ++c) {
        int32_t tau[ORC_MAXK];
        uint8_t h;
        uint64_t s[3];
        double X = orc_trial(Q, first + c, tau, &h, s);
        if (emb) memcpy(emb + 8 * c, tau, sizeof(tau));
        if (hit) hit[c] = h;
        if (x) x[c] = X;
        if (sectors) for (int j = 0; j < 3; ++j) sectors[3 * c + j] = s[j];
    }
}

/* Sums over trials [first, first+count): n, hits, sum X, sum X^2, and the three
 * sector counts. */
void orc_sums(const orc_query *Q, uint64_t first, uint64_t count, uint64_t *hits,
              double *sx, double *sx2, uint64_t sectors[3])
{
    uint64_t h = 0, sec[3] = {0, 0, 0};
    double a = 0.0, b = 0.0;
    for (uint64_t c = 0; c < count; ++c) {
        int32_t tau[ORC_MAXK];
        uint8_t hh;
        uint64_t s[3];
        double X = orc_trial(Q, first + c, tau, &hh, s);
        h += hh;
        for (int j = 0; j < 3; ++j) sec[j] += s[j];
        a += X;
        b += X * X;
    }
    *hits = h; *sx = a; *sx2 = b;
    for (int j = 0; j < 3; ++j) sectors[j] = sec[j];
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 (online convergence) at chunk checkpoints (READING R7).           */
/* ------------------------------------------------------------------------ */
/* Phi^{-1}(1 - delta/2), found by bisection on the upper tail 0.5*erfc(z/sqrt 2) =
 * delta/2 (the tail form avoids cancellation in 1 - delta/2). */
double orc_z_of_delta(double delta)
{
    double lo = 0.0, hi = 40.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (0.5 * erfc(mid / sqrt(2.0)) > delta / 2.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

typedef struct {
    uint64_t trials, hits, sectors;
    double sum_x, sum_x2, mean, var, eps_hat;
    int32_t converged;
    uint64_t sectors_streamed, sectors_survey;
} orc_estimate_result;

static void alg1(double n, double sx, double sx2, double z, double *mu, double *var, double *eps_hat)
{
    double m = sx / n;
    double s2 = sx2 / n - m * m;
    if (s2 < 0.0) s2 = 0.0;
    *mu = m;
    *var = s2;
    *eps_hat = (m > 0.0) ? z * sqrt(s2) / sqrt(n) / m : INFINITY;
}

void orc_estimate(const orc_query *Q, double eps, double delta, uint64_t chunk,
                  uint64_t min_trials, uint64_t max_trials, orc_estimate_result *res)
{
    double z = orc_z_of_delta(delta);
    uint64_t n = 0, h = 0, sec[3] = {0, 0, 0};
    double sx = 0.0, sx2 = 0.0, mu = 0.0, var = 0.0, eh = INFINITY;
    int conv = 0;
    while (n < max_trials) {
        uint64_t c = chunk;
        if (n + c > max_trials) c = max_trials - n;
        for (uint64_t j = 0; j < c; ++j) {
            int32_t tau[ORC_MAXK];
            uint8_t hh;
            uint64_t s[3];
            double X = orc_trial(Q, n + j, tau, &hh, s);
            h += hh;
            for (int w = 0; w < 3; ++w) sec[w] += s[w];
            sx += X;
            sx2 += X * X;
        }
        n += c;
        alg1((double)n, sx, sx2, z, &mu, &var, &eh);
        if (n >= min_trials && mu > 0.0 && eh <= eps) { conv = 1; break; }
    }
    res->trials = n; res->hits = h; res->sectors = sec[0];
    res->sectors_streamed = sec[1]; res->sectors_survey = sec[2];
    res->sum_x = sx; res->sum_x2 = sx2;
    res->mean = mu; res->var = var; res->eps_hat = eh; res->converged = conv;
}

/* ------------------------------------------------------------------------ */
/* Exact references for tiny graphs.                                         */
/* ------------------------------------------------------------------------ */

/* C(G,P) by exhaustive backtracking (Sec. 2.1 definition: injective maps that keep
 * every pattern edge).  Pattern vertices are matched in index order; no pruning
 * beyond the definition. */
static uint64_t bf_rec(int64_t nv, const int64_t *off, const int32_t *cols, int k,
                       const unsigned adj[], int32_t *map, int depth)
{
    if (depth == k) return 1;
    uint64_t total = 0;
    /* A pattern vertex with an already-matched neighbour can only go to a neighbour of
     * that image; otherwise every graph vertex is tried. */
    int anchor = -1;
    for (int j = 0; j < depth; ++j) if (adj[depth] >> j & 1u) { anchor = j; break; }
    int64_t lo = 0, hi = nv;
    if (anchor >= 0) { lo = off[map[anchor]]; hi = off[map[anchor] + 1]; }
    for (int64_t it = lo; it < hi; ++it) {
        int64_t v = anchor >= 0 ? cols[it] : it;
        int ok = 1;
        for (int j = 0; j < depth && ok; ++j) {
            if (map[j] == v) ok = 0;
            else if ((adj[depth] >> j & 1u) && !is_neighbour(off, cols, map[j], (int32_t)v)) ok = 0;
        }
        if (!ok) continue;
        map[depth] = (int32_t)v;
        total += bf_rec(nv, off, cols, k, adj, map, depth + 1);
    }
    return total;
}

/* n_(v) of Sec. 4.1 for every v: embeddings whose first pattern vertex in the
 * matching order pi maps to v (so that f_ideal(v | ()) = n_(v) / C(G,P), Thm. 1). */
int orc_bruteforce_by_first(int64_t nv, const int64_t *off, const int32_t *cols,
                            int32_t k, int32_t ne, const int32_t *edges, int64_t *counts)
{
    orc_plan plan;
    if (orc_plan_compile(k, ne, edges, &plan) != 0) return -1;
    /* relabel the pattern so that pattern vertex 0 is u_1 = pi(1) */
    int inv[ORC_MAXK];
    for (int i = 0; i < k; ++i) inv[plan.order[i]] = i;
    unsigned adj[ORC_MAXK] = {0};
    for (int e = 0; e < ne; ++e) {
        int a = inv[edges[2 * e]], b = inv[edges[2 * e + 1]];
        adj[a] |= 1u << b;
        adj[b] |= 1u << a;
    }
    int32_t map[ORC_MAXK];
    for (int64_t v = 0; v < nv; ++v) {
        map[0] = (int32_t)v;
        counts[v] = (int64_t)bf_rec(nv, off, cols, k, adj, map, 1);
    }
    return 0;
}

int64_t orc_bruteforce_count(int64_t nv, const int64_t *off, const int32_t *cols,
                             int32_t k, int32_t ne, const int32_t *edges)
{
    if (k < 1 || k > ORC_MAXK) return -1;
    unsigned adj[ORC_MAXK] = {0};
    for (int e = 0; e < ne; ++e) {
        adj[edges[2 * e]] |= 1u << edges[2 * e + 1];
        adj[edges[2 * e + 1]] |= 1u << edges[2 * e];
    }
    int32_t map[ORC_MAXK];
    return (int64_t)bf_rec(nv, off, cols, k, adj, map, 0);
}

/* Exact embedding counts for three small patterns on graphs too large for the
 * backtracking counter, by the classical identities (each pinned to brute force on
 * tiny graphs by the tests):
 *   triangle: C = sum over ordered adjacent (u, v) of |N(u) & N(v)|;
 *   4-cycle:  C = sum over ordered a != c of w(a,c) (w(a,c) - 1), w = |N(a) & N(c)|
 *             (u0 = a, u2 = c, then an ordered pair of distinct common neighbours);
 *   4-clique: C = 24 * #K4, #K4 counted over id-increasing vertex quadruples. */
static int64_t common_count(const int64_t *off, const int32_t *cols, int32_t a, int32_t b)
{
    int64_t i = off[a], j = off[b], c = 0;
    while (i < off[a + 1] && j < off[b + 1]) {
        if (cols[i] < cols[j]) i++;
        else if (cols[i] > cols[j]) j++;
        else { c++; i++; j++; }
    }
    return c;
}

int64_t orc_exact_triangle(int64_t nv, const int64_t *off, const int32_t *cols)
{
    int64_t total = 0;
    for (int64_t u = 0; u < nv; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e)
            total += common_count(off, cols, (int32_t)u, cols[e]);
    return total;
}

int64_t orc_exact_4cycle(int64_t nv, const int64_t *off, const int32_t *cols)
{
    int64_t *w = (int64_t *)calloc((size_t)nv, sizeof(int64_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    if (!w || !touched) { free(w); free(touched); return -1; }
    int64_t total = 0;
    for (int64_t a = 0; a < nv; ++a) {
        int64_t nt = 0;
        for (int64_t e = off[a]; e < off[a + 1]; ++e) {
            int32_t b = cols[e];
            for (int64_t f = off[b]; f < off[b + 1]; ++f) {
                int32_t c = cols[f];
                if (c == a) continue;
                if (w[c] == 0) touched[nt++] = c;
                w[c]++;
            }
        }
        for (int64_t t = 0; t < nt; ++t) {
            int64_t x = w[touched[t]];
            total += x * (x - 1);
            w[touched[t]] = 0;
        }
    }
    free(w);
    free(touched);
    return total;
}

int64_t orc_exact_4clique(int64_t nv, const int64_t *off, const int32_t *cols)
{
    int64_t k4 = 0;
    int32_t *t = NULL;
    int64_t cap = 0;
    for (int64_t u = 0; u < nv; ++u) {
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int32_t v = cols[e];
            if (v <= u) continue;
            /* T = common neighbours of u and v above v */
            int64_t need = off[u + 1] - off[u];
            if (need > cap) { free(t); cap = need; t = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap); if (!t) return -1; }
            int64_t n = 0, i = off[u], j = off[v];
            while (i < off[u + 1] && j < off[v + 1]) {
                if (cols[i] < cols[j]) i++;
                else if (cols[i] > cols[j]) j++;
                else { if (cols[i] > v) t[n++] = cols[i]; i++; j++; }
            }
            for (int64_t x = 0; x < n; ++x)
                for (int64_t y = x + 1; y < n; ++y)
                    k4 += is_neighbour(off, cols, t[x], t[y]);
        }
    }
    free(t);
    return 24 * k4;
}

/* Exact first and second moments of the sampler output by walking every branch of
 * Alg. 3 with its probability q(v)/W (Thm. 2 says E[X] = C(G,P)).  Also counts the
 * successful trajectories. */
static void enum_rec(const orc_query *Q, int i, int32_t *tau, long double p, double X,
                     long double *m1, long double *m2, uint64_t *nsucc)
{
    const orc_plan *pl = &Q->plan;
    if (i == pl->k) {
        *m1 += p * (long double)X;
        *m2 += p * (long double)X * (long double)X;
        (*nsucc)++;
        return;
    }
    if (i == 0) {
        uint64_t W = Q->W1;
        if (W == 0) return;
        for (int64_t v = 0; v < Q->nv; ++v) {
            uint64_t q = step_weight(Q, 0, (int32_t)v);
            if (q == 0) continue;
            tau[0] = (int32_t)v;
            enum_rec(Q, 1, tau, p * (long double)q / (long double)W, X * ((double)W / (double)q),
                     m1, m2, nsucc);
        }
        return;
    }
    uint64_t W;
    int64_t n;
    int a = -1;
    if (Q->anchor && pl->nback[i] >= 2) a = anchor_candidates(Q, i, tau, &W, &n);
    else n = build_candidates(Q, i, tau, &W);
    if (n == 0 || W == 0) return;
    int32_t *c = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint64_t *cq = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    memcpy(c, Q->cand, sizeof(int32_t) * (size_t)n);
    memcpy(cq, Q->candq, sizeof(uint64_t) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) {
        if (cq[j] == 0) continue;
        if (a >= 0 && !closes_all(Q, i, tau, a, c[j])) continue;   /* a failed trial: X = 0 */
        tau[i] = c[j];
        enum_rec(Q, i + 1, tau, p * (long double)cq[j] / (long double)W,
                 X * ((double)W / (double)cq[j]), m1, m2, nsucc);
    }
    tau[i] = -1;
    free(c);
    free(cq);
}

void orc_enumerate(const orc_query *Q, double *mean, double *second, uint64_t *n_success)
{
    int32_t tau[ORC_MAXK];
    for (int i = 0; i < ORC_MAXK; ++i) tau[i] = -1;
    long double m1 = 0.0L, m2 = 0.0L;
    uint64_t ns = 0;
    enum_rec(Q, 0, tau, 1.0L, 1.0, &m1, &m2, &ns);
    *mean = (double)m1;
    *second = (double)m2;
    *n_success = ns;
}

/* Exact probability of one full trajectory under the query's distributions
 * (product of q(v_i)/W_i), 0 if any step is impossible. */
double orc_trajectory_prob(const orc_query *Q, const int32_t *tau_in)
{
    int32_t tau[ORC_MAXK];
    for (int i = 0; i < ORC_MAXK; ++i) tau[i] = -1;
    long double p = 1.0L;
    for (int i = 0; i < Q->plan.k; ++i) {
        uint64_t W, q = 0;
        if (i == 0) {
            W = Q->W1;
            q = step_weight(Q, 0, tau_in[0]);
        } else {
            int64_t n = build_candidates(Q, i, tau, &W);
            int found = 0;
            for (int64_t j = 0; j < n; ++j) if (Q->cand[j] == tau_in[i]) { q = Q->candq[j]; found = 1; break; }
            if (!found) return 0.0;
        }
        if (W == 0 || q == 0) return 0.0;
        p *= (long double)q / (long double)W;
        tau[i] = tau_in[i];
    }
    return (double)p;
}
