// Host-side pattern analysis: matching order (Alg. 2), auxiliary arrays
// A^pi = {B, F1, F2, I_eff} per step (Def. auxiliary arrays, Sec. 4.2.3), Certainty
// and the decision function D^pi (Def. decision function), and |Aut(P)|.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>

#include "agis_internal.h"

namespace {

struct PatternGraph {
    int k = 0;
    bool e[agis::kMaxK][agis::kMaxK] = {{false}};
};

// Hop structure of P_i (Eq. Pi): the sub-pattern induced by the not-yet-matched
// vertices `alive`, seen from its vertex `root`.
struct HopView {
    int hop[agis::kMaxK];       // distance from root inside P_i, -1 if unreachable/absent
    int forward1 = 0;           // |F1|: edges between hop 0 and hop 1
    int internal1 = 0;          // |I1|: edges with both ends at hop 1
    int internal_eff = 0;       // |I_eff|: edges of a spanning forest of (V_ind, I1)
    int forward2 = 0;           // |F2|: edges between hop 1 and hop 2
    int far_vertices = 0;       // |V_i^{>=2hop}|
    int far_edges = 0;          // |E_i^{>=2hop}|, counted over all of E_P
};

HopView look_from(const PatternGraph &P, const bool alive[], int root)
{
    HopView h;
    for (int v = 0; v < P.k; ++v) h.hop[v] = -1;
    h.hop[root] = 0;
    // breadth-first levels restricted to alive vertices
    for (int level = 0; level < P.k; ++level) {
        bool grew = false;
        for (int v = 0; v < P.k; ++v) {
            if (h.hop[v] != level) continue;
            for (int w = 0; w < P.k; ++w)
                if (P.e[v][w] && alive[w] && h.hop[w] < 0) { h.hop[w] = level + 1; grew = true; }
        }
        if (!grew) break;
    }
    // label of the component of each hop-1 vertex under I1 edges
    int comp[agis::kMaxK];
    for (int v = 0; v < P.k; ++v) comp[v] = v;
    auto find = [&](int v) { while (comp[v] != v) v = comp[v] = comp[comp[v]]; return v; };
    for (int a = 0; a < P.k; ++a) {
        for (int b = a + 1; b < P.k; ++b) {
            if (!P.e[a][b]) continue;
            const int ha = h.hop[a], hb = h.hop[b];
            if (ha >= 0 && hb >= 0) {
                if (std::min(ha, hb) == 0 && std::max(ha, hb) == 1) h.forward1++;
                if (ha == 1 && hb == 1) {
                    h.internal1++;
                    int ra = find(a), rb = find(b);
                    if (ra != rb) { comp[ra] = rb; h.internal_eff++; }
                }
                if (std::min(ha, hb) == 1 && std::max(ha, hb) == 2) h.forward2++;
            }
            // E^{>=2hop}: any pattern edge touching a vertex at finite distance >= 2
            if (ha >= 2 || hb >= 2) h.far_edges++;
        }
    }
    for (int v = 0; v < P.k; ++v) if (h.hop[v] >= 2) h.far_vertices++;
    return h;
}

uint64_t automorphism_count(const PatternGraph &P)
{
    int perm[agis::kMaxK];
    std::iota(perm, perm + P.k, 0);
    uint64_t n = 0;
    do {
        bool keeps = true;
        for (int a = 0; a < P.k && keeps; ++a)
            for (int b = a + 1; b < P.k; ++b)
                if (P.e[a][b] && !P.e[perm[a]][perm[b]]) { keeps = false; break; }
        n += keeps;
    } while (std::next_permutation(perm, perm + P.k));
    return n;
}

}  // namespace

extern "C" int agis_pattern_create(int k, int ne, const int32_t *edge_pairs, agis_pattern **out)
{
    if (!out) return AGIS_ERR_ARG;
    *out = nullptr;
    if (!edge_pairs && ne > 0) return AGIS_ERR_ARG;
    if (k < 2 || k > agis::kMaxK || ne < k - 1 || ne > k * (k - 1) / 2) return AGIS_ERR_PATTERN;
    PatternGraph P;
    P.k = k;
    for (int i = 0; i < ne; ++i) {
        const int a = edge_pairs[2 * i], b = edge_pairs[2 * i + 1];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b || P.e[a][b]) return AGIS_ERR_PATTERN;
        P.e[a][b] = P.e[b][a] = true;
    }
    // connected?
    bool all_alive[agis::kMaxK];
    for (int v = 0; v < agis::kMaxK; ++v) all_alive[v] = v < k;
    HopView whole = look_from(P, all_alive, 0);
    for (int v = 0; v < k; ++v) if (whole.hop[v] < 0) return AGIS_ERR_PATTERN;

    agis_pattern *p = new (std::nothrow) agis_pattern();
    if (!p) return AGIS_ERR_NOMEM;
    p->k = k;
    bool alive[agis::kMaxK];
    bool matched[agis::kMaxK];
    for (int v = 0; v < agis::kMaxK; ++v) { alive[v] = v < k; matched[v] = false; }

    // Alg. 2: grow pi greedily; candidates are all vertices at step 1 and the
    // unmatched neighbours of pi afterwards; score |F1| + |I1| of P_i seen from the
    // candidate; the smallest id wins a tie.
    for (int i = 0; i < k; ++i) {
        int pick = -1, best = -1;
        for (int u = 0; u < k; ++u) {
            if (matched[u]) continue;
            bool touches = (i == 0);
            for (int w = 0; w < k && !touches; ++w) touches = matched[w] && P.e[u][w];
            if (!touches) continue;
            HopView h = look_from(P, alive, u);
            const int score = h.forward1 + h.internal1;
            if (score > best) { best = score; pick = u; }
        }
        p->order[i] = pick;
        // auxiliary arrays and Certainty of step i (P_i still contains u_i)
        HopView h = look_from(P, alive, pick);
        int nb = 0;
        for (int j = 0; j < i; ++j)
            if (P.e[pick][p->order[j]]) p->back[i][nb++] = j;
        p->nback[i] = nb;
        p->cfg[i][0] = nb;
        p->cfg[i][1] = h.forward1;
        p->cfg[i][2] = h.internal_eff;
        p->cfg[i][3] = h.forward2;
        int n_alive = 0;
        for (int v = 0; v < k; ++v) n_alive += alive[v];
        p->certainty[i] = 1.0 - double(h.far_edges - h.far_vertices) / double(n_alive);
        matched[pick] = true;
        alive[pick] = false;
    }
    p->aut = automorphism_count(P);
    *out = p;
    return AGIS_OK;
}

extern "C" int agis_pattern_info(const agis_pattern *p, int32_t *k, int32_t order[8],
                                 int32_t cfg[8][4], double certainty[8], uint8_t back[8],
                                 uint64_t *automorphisms)
{
    if (!p) return AGIS_ERR_ARG;
    if (k) *k = p->k;
    for (int i = 0; i < agis::kMaxK; ++i) {
        const bool in = i < p->k;
        if (order) order[i] = in ? p->order[i] : 0;
        if (cfg) for (int c = 0; c < 4; ++c) cfg[i][c] = in ? p->cfg[i][c] : 0;
        if (certainty) certainty[i] = in ? p->certainty[i] : 0.0;
        if (back) {
            uint8_t m = 0;
            if (in) for (int j = 0; j < p->nback[i]; ++j) m |= uint8_t(1u << p->back[i][j]);
            back[i] = m;
        }
    }
    if (automorphisms) *automorphisms = p->aut;
    return AGIS_OK;
}

extern "C" int agis_pattern_decide(const agis_pattern *p, int32_t mode, double beta,
                                   uint8_t use_approx[8])
{
    if (!p || !use_approx || mode < 0 || mode > 2) return AGIS_ERR_ARG;
    for (int i = 0; i < agis::kMaxK; ++i) {
        uint8_t d = 0;
        if (i < p->k) {
            if (mode == AGIS_MODE_APPROX) d = 1;
            else if (mode == AGIS_MODE_AUTO) d = p->certainty[i] >= beta ? 1 : 0;
        }
        use_approx[i] = d;
    }
    return AGIS_OK;
}

extern "C" int agis_pattern_free(agis_pattern *p)
{
    delete p;
    return AGIS_OK;
}
