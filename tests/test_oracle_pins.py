"""Pins of the CPU oracle to things other than itself: independent libraries
(numpy's Philox, scipy's normal quantile, networkx's matcher), closed forms,
values the paper prints (tests/golden/paper_facts.json), invariants and brute
force on tiny inputs.  CPU only."""
import itertools
import json
import math
import os

import networkx as nx
import numpy as np
import pytest
import scipy.stats

from paper_2601_01388_b300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))
CMIN = 2.0 ** -10
MODES = (0, 1, 2)


def nx_graph(off, cols):
    g = nx.Graph()
    g.add_nodes_from(range(len(off) - 1))
    s, d = I.edges_of(off, cols)
    g.add_edges_from(zip(s.tolist(), d.tolist()))
    return g


def nx_pattern(k, edges):
    p = nx.Graph()
    p.add_nodes_from(range(k))
    p.add_edges_from(edges)
    return p


def nx_embeddings(off, cols, k, edges):
    """C(G,P) (Sec. 2.1): non-induced embeddings = subgraph monomorphisms."""
    gm = nx.algorithms.isomorphism.GraphMatcher(nx_graph(off, cols), nx_pattern(k, edges))
    return sum(1 for _ in gm.subgraph_monomorphisms_iter())


def falling(n, k):
    r = 1
    for j in range(k):
        r *= n - j
    return r


TINY_GRAPHS = {
    "gnp10": lambda: I.gnp_graph(10, 0.5, 3),
    "gnp12": lambda: I.gnp_graph(12, 0.45, 7),
    "k6": lambda: I.complete_graph(6),
    "c7": lambda: I.cycle_graph(7),
    "tree9": lambda: I.random_tree(9, 2),
    "star6": lambda: I.star_graph(6),
    "mixed": lambda: I.disjoint_union(I.complete_graph(5), I.cycle_graph(6), I.gnp_graph(7, 0.6, 11)),
}

SMALL_PATTERNS = ["edge", "triangle", "4-cycle", "4-clique", "5-cycle", "house", "tailed-triangle",
                  "diamond", "3-path", "4-path", "3-star", "chordal-5-cycle"]


# ---------------------------------------------------------------- RNG and draw

@pytest.mark.parametrize("ctr,key", [([1, 0, 0, 0], [0, 0]), ([5, 7, 1, 0], [123, 456]),
                                     ([2 ** 63, 2 ** 64 - 1, 3, 9], [2 ** 64 - 1, 17]),
                                     ([99, 2, 1, 0], [1, 0])])
def test_philox_matches_numpy(oracle_mod, ctr, key):
    # numpy's Philox4x64-10 bumps its counter before producing a block
    g = np.random.Philox(key=np.array(key, dtype=np.uint64),
                         counter=np.array([ctr[0] - 1] + ctr[1:], dtype=np.uint64))
    assert [int(x) for x in g.random_raw(4)] == oracle_mod.philox(ctr, key)


def test_draw_below_is_floor_of_128bit_product(oracle_mod):
    # large W: the carry out of the low 64-bit half changes the result about W/2^64 of the time
    for W, n in [(1, 5), (2, 5), (3, 5), (1000, 5), (2 ** 40 + 7, 5), (2 ** 62 - 1, 300), (3 * 2 ** 60, 300)]:
        for t in range(1, n + 1):
            g = np.random.Philox(key=np.array([42, 0], dtype=np.uint64),
                                 counter=np.array([t - 1, 3, 1, 0], dtype=np.uint64))
            o = [int(x) for x in g.random_raw(4)]
            U = o[0] + (o[1] << 64)
            assert oracle_mod.draw_below(W, t, 3, 1, 42) == (U * W) >> 128


def test_draw_below_uniform_chi2(oracle_mod):
    W, n = 7, 14000
    counts = np.bincount([oracle_mod.draw_below(W, t, 1, 1, 5) for t in range(n)], minlength=W)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4


def test_draw_over_equal_weights_is_a_position_draw(oracle_mod):
    # n candidates of equal weight c: the weighted draw picks position floor(r / c)
    # with r = floor(U n c / 2^128), which is floor(U n / 2^128), the draw over n
    # (nested floors); and W / q = n c / c is exactly n in double.  A step whose
    # weights are equal on every candidate can therefore draw by position.
    rng = np.random.default_rng(3)
    for n in [1, 2, 3, 7, 1000, 65537, 2 ** 31 - 1]:
        for c in [1, 2, 3, 2 ** 20, 2 ** 30 + 5, (2 ** 62 - 1) // n]:
            if c < 1 or n * c >= 2 ** 62:
                continue
            for t in rng.integers(0, 2 ** 40, size=6):
                t = int(t)
                assert oracle_mod.draw_below(n * c, t, 4, 1, 9) // c == oracle_mod.draw_below(n, t, 4, 1, 9)
            assert float(n * c) / float(c) == float(n)


@pytest.mark.parametrize("cfg", [(1, 0, 0, 0), (2, 0, 0, 0), (3, 0, 0, 0), (4, 0, 0, 0)])
def test_configs_without_exponents_weigh_candidates_equally(oracle_mod, cfg):
    # binom(d - |B|, 0) = 1 from d = |B| on, 0 below: one constant on every vertex
    # of degree >= |B|, which every candidate of a step with |B| backward edges has
    off, cols = I.rmat_graph(9, 8, seed=5)
    nsum, hits = oracle_mod.graph_stats(off, cols, 1)
    q, shift = oracle_mod.weight_table(off, nsum, hits, 2.0 ** -10, cfg)
    deg = np.diff(off)
    assert (q[deg < cfg[0]] == 0).all()
    vals = np.unique(q[deg >= cfg[0]])
    assert len(vals) == 1 and vals[0] > 0


@pytest.mark.parametrize("d", [2, 3, 4, 7])
def test_cc_pair_is_bijection_on_ordered_distinct_pairs(oracle_mod, d):
    pairs = [oracle_mod.cc_pair(d, r) for r in range(d * (d - 1))]
    assert sorted(pairs) == sorted((a, b) for a in range(d) for b in range(d) if a != b)


@pytest.mark.parametrize("delta", [0.5, 0.1, 0.05, 0.01, 1e-3, 1e-6])
def test_z_matches_scipy(oracle_mod, delta):
    assert oracle_mod.z_of_delta(delta) == pytest.approx(scipy.stats.norm.isf(delta / 2), rel=1e-12)


# ---------------------------------------------------------------- pattern analysis

@pytest.mark.parametrize("name", sorted(I.PATTERNS))
def test_automorphisms_match_networkx(oracle_mod, name):
    k, edges = I.PATTERNS[name]
    p = nx_pattern(k, edges)
    want = sum(1 for _ in nx.algorithms.isomorphism.GraphMatcher(p, p).isomorphisms_iter())
    assert oracle_mod.compile_pattern(k, edges)["aut"] == want


def test_automorphisms_random_patterns(oracle_mod):
    rng = np.random.Generator(np.random.Philox(key=[9, 0]))
    for _ in range(25):
        k, edges = I.random_connected_pattern(rng, 3, 7)
        p = nx_pattern(k, edges)
        want = sum(1 for _ in nx.algorithms.isomorphism.GraphMatcher(p, p).isomorphisms_iter())
        assert oracle_mod.compile_pattern(k, edges)["aut"] == want


def test_house_has_one_uniform_step(oracle_mod):
    g = GOLDEN["house_uniform_steps_sec_6_1"]
    k, edges = I.PATTERNS["house"]
    use = oracle_mod.decide(k, edges, 0, g["beta"])
    assert len(use) == g["pattern_vertices"]
    assert use.count(0) == g["uniform_steps"]


@pytest.mark.parametrize("name", GOLDEN["certainty_one_patterns_sec_6_1"]["patterns"])
def test_table2_patterns_have_certainty_one(oracle_mod, name):
    k, edges = I.PATTERNS[name]
    assert all(c == 1.0 for c in oracle_mod.compile_pattern(k, edges)["certainty"])


def test_hand_derived_plans(oracle_mod):
    # Worked by hand from Alg. 2, Eq. Pi and Def. auxiliary arrays.
    tri = oracle_mod.compile_pattern(*I.PATTERNS["triangle"])
    assert tri["order"] == [0, 1, 2]
    assert tri["cfg"] == [(0, 2, 1, 0), (1, 1, 0, 0), (2, 0, 0, 0)]
    c4 = oracle_mod.compile_pattern(*I.PATTERNS["4-cycle"])
    assert c4["order"] == [0, 1, 2, 3]
    assert c4["cfg"] == [(0, 2, 0, 2), (1, 1, 0, 1), (1, 1, 0, 0), (2, 0, 0, 0)]
    assert c4["certainty"][:2] == [pytest.approx(0.75), pytest.approx(2 / 3)]
    house = oracle_mod.compile_pattern(*I.PATTERNS["house"])
    assert house["order"] == [0, 1, 2, 3, 4]
    assert house["cfg"] == [(0, 3, 1, 2), (1, 2, 0, 1), (1, 1, 0, 0), (2, 0, 0, 0), (2, 0, 0, 0)]
    assert house["certainty"][1] == pytest.approx(0.75)
    star = oracle_mod.compile_pattern(*I.PATTERNS["4-star"])
    assert star["order"][0] == 0
    assert star["cfg"][0] == (0, 4, 0, 0)
    assert all(c == (1, 0, 0, 0) for c in star["cfg"][1:])
    # Alg. 2 scores s(u) = |F1| + |I1|: vertices 0 and 1 both have three pattern
    # neighbours, only 1 has an edge among them (5-6), so 1 comes first.
    two_hubs = oracle_mod.compile_pattern(7, [(0, 1), (0, 3), (0, 4), (1, 5), (1, 6), (5, 6), (2, 3)])
    assert two_hubs["order"][0] == 1
    assert two_hubs["cfg"][0] == (0, 3, 1, 2)
    k5 = oracle_mod.compile_pattern(*I.PATTERNS["5-clique"])
    assert k5["cfg"] == [(0, 4, 3, 0), (1, 3, 2, 0), (2, 2, 1, 0), (3, 1, 0, 0), (4, 0, 0, 0)]


def test_matching_order_is_connected_and_backward_sets_cover_edges(oracle_mod):
    rng = np.random.Generator(np.random.Philox(key=[10, 0]))
    for _ in range(40):
        k, edges = I.random_connected_pattern(rng, 2, 8)
        plan = oracle_mod.compile_pattern(k, edges)
        order = plan["order"]
        assert sorted(order) == list(range(k))
        es = {frozenset(e) for e in edges}
        for i in range(1, k):
            assert plan["back"][i], "every later step has a backward edge (connected order)"
        n_back = sum(len(b) for b in plan["back"])
        assert n_back == len(edges)
        for i in range(k):
            for j in plan["back"][i]:
                assert frozenset((order[i], order[j])) in es


@pytest.mark.parametrize("bad", [(1, [(0, 0)]), (3, [(0, 1)]), (3, [(0, 1), (0, 1)]),
                                 (9, [(i, i + 1) for i in range(8)]), (3, [(0, 3)]),
                                 (4, [(0, 1), (2, 3)])])
def test_invalid_patterns_rejected(oracle_mod, bad):
    with pytest.raises(ValueError):
        oracle_mod.compile_pattern(*bad)


# ---------------------------------------------------------------- weights (Eq. probability_function)

def worked_example_graph():
    """A graph realising the Sec. 4.2.3 example: vertex 0 has degree 6, neighbours
    1..6 of degrees 4,4,3,3,3,3 and 5 edges among them."""
    e = [(0, v) for v in range(1, 7)] + [(1, 2), (1, 3), (2, 4), (3, 5), (4, 6)]
    e += [(1, 7), (2, 8), (5, 9), (6, 10)]
    s, d = zip(*e)
    return I.csr_from_edges(11, np.array(s), np.array(d))


def test_worked_example_terms(oracle_mod):
    g = GOLDEN["worked_example_sec_4_2_3"]
    off, cols = worked_example_graph()
    deg = np.diff(off)
    assert deg[0] == g["degree"]
    assert sorted(deg[cols[off[0]:off[1]]].tolist(), reverse=True) == g["neighbour_degrees"]
    nb = set(cols[off[0]:off[1]].tolist())
    inner = sum(1 for a, b in itertools.combinations(sorted(nb), 2)
                if b in set(cols[off[a]:off[a + 1]].tolist()))
    assert inner == g["edges_among_neighbours"]
    nsum, _ = oracle_mod.graph_stats(off, cols)
    assert nsum[0] == sum(g["neighbour_degrees"])
    # C_a = 5/15 as a sampled ratio hits/d: 2 of 6 probes
    hits = 2
    d = g["degree"]
    ca = g["C_a_num"] / g["C_a_den"]
    tf1 = math.comb(g["T_F1_binom_n"], g["T_F1_binom_k"])
    assert oracle_mod.weight(d, int(nsum[0]), hits, CMIN, (2, 3, 0, 0)) == tf1
    assert oracle_mod.weight(d, int(nsum[0]), hits, CMIN, (0, 0, g["I_eff"], 0)) == pytest.approx(ca ** 2, rel=1e-15)
    tf2 = (sum(g["neighbour_degrees"]) / d) ** g["F2"]
    assert oracle_mod.weight(d, int(nsum[0]), hits, CMIN, (0, 0, 0, g["F2"])) == pytest.approx(tf2, rel=1e-15)
    full = oracle_mod.weight(d, int(nsum[0]), hits, CMIN, (2, 3, g["I_eff"], g["F2"]))
    assert full == pytest.approx(tf1 * ca ** 2 * tf2, rel=1e-14)


def test_weight_edge_cases(oracle_mod):
    # binom(n, k) = 0 when n < k: an intended zero (no extension exists)
    assert oracle_mod.weight(3, 9, 3, CMIN, (2, 2, 0, 0)) == 0.0
    assert oracle_mod.quantise(0.0, 3, (2, 2, 0, 0), 40) == 0
    # floor at c_min keeps every other weight positive (Sec. 4.4)
    w = oracle_mod.weight(5, 10, 0, CMIN, (0, 2, 3, 0))
    assert w == pytest.approx(10 * CMIN ** 3)
    assert oracle_mod.quantise(w, 5, (0, 2, 3, 0), -200) == 1
    # degree < 2 gives c_min
    assert oracle_mod.weight(1, 4, 0, CMIN, (0, 1, 1, 0)) == pytest.approx(CMIN)
    # binom recurrence equals math.comb while exact
    for n in range(0, 60):
        for k in range(0, 8):
            assert oracle_mod.weight(n + 1, n + 1, 0, CMIN, (1, k, 0, 0)) == (math.comb(n, k) if n >= k else 0)


def test_quantised_sums_fit_62_bits(oracle_mod):
    off, cols = I.rmat_graph(10, 16)
    nsum, hits = oracle_mod.graph_stats(off, cols)
    for cfg in [(0, 4, 3, 0), (0, 3, 1, 2), (1, 2, 0, 1), (0, 6, 0, 0)]:
        sh = oracle_mod.quant_shift(off, nsum, hits, CMIN, cfg)
        deg = np.diff(off)
        total = 0
        wmax = 0
        for v in range(len(deg)):
            w = oracle_mod.weight(int(deg[v]), int(nsum[v]), int(hits[v]), CMIN, cfg)
            q = oracle_mod.quantise(w, int(deg[v]), cfg, sh)
            total += q
            wmax = max(wmax, q)
        assert total < 2 ** 62
        assert wmax >= 2 ** (62 - math.ceil(math.log2(len(deg) + 1)) - 1)


# ---------------------------------------------------------------- preprocessing (Sec. 4.4)

def test_cc_hits_on_closed_form_graphs(oracle_mod):
    off, cols = I.complete_graph(7)           # every neighbour pair joined: C_v = 1
    _, hits = oracle_mod.graph_stats(off, cols)
    assert (hits == 6).all()
    off, cols = I.star_graph(9)               # no pair of leaves joined: C_v = 0
    nsum, hits = oracle_mod.graph_stats(off, cols)
    assert (hits == 0).all()
    assert nsum[0] == 9 and (nsum[1:] == 9).all()
    off, cols = I.random_tree(30, 4)
    _, hits = oracle_mod.graph_stats(off, cols)
    assert (hits == 0).all()


def test_cc_hits_track_exact_clustering(oracle_mod):
    off, cols = I.gnp_graph(200, 0.3, 5)
    _, hits = oracle_mod.graph_stats(off, cols)
    deg = np.diff(off)
    g = nx_graph(off, cols)
    exact = nx.clustering(g)
    est = hits.sum() / deg.sum()
    want = sum(exact[v] * deg[v] for v in range(200)) / deg.sum()
    assert est == pytest.approx(want, abs=0.02)


# ---------------------------------------------------------------- exact counts

@pytest.mark.parametrize("gname", sorted(TINY_GRAPHS))
@pytest.mark.parametrize("pname", ["triangle", "4-cycle", "4-clique", "house", "tailed-triangle", "3-star", "5-cycle"])
def test_bruteforce_matches_networkx(oracle_mod, gname, pname):
    off, cols = TINY_GRAPHS[gname]()
    k, edges = I.PATTERNS[pname]
    assert oracle_mod.bruteforce_count(off, cols, k, edges) == nx_embeddings(off, cols, k, edges)


def test_bruteforce_closed_forms(oracle_mod):
    for n in (5, 6, 7):
        off, cols = I.complete_graph(n)
        for name in ("triangle", "4-cycle", "4-clique", "house", "4-star", "5-clique"):
            k, edges = I.PATTERNS[name]
            assert oracle_mod.bruteforce_count(off, cols, k, edges) == falling(n, k)
    for n in (5, 6, 8):
        off, cols = I.cycle_graph(n)
        assert oracle_mod.bruteforce_count(off, cols, *I.cycle(n)) == 2 * n
        for k in range(2, n):
            assert oracle_mod.bruteforce_count(off, cols, *I.path(k)) == 2 * n
    off, cols = I.star_graph(6)
    for leaves in (2, 3, 4):
        assert oracle_mod.bruteforce_count(off, cols, *I.star(leaves)) == falling(6, leaves) + (2 * 6 if leaves == 1 else 0)


@pytest.mark.parametrize("gname", ["gnp10", "mixed", "k6"])
def test_counts_divided_by_aut_are_integers(oracle_mod, gname):
    off, cols = TINY_GRAPHS[gname]()
    for name in SMALL_PATTERNS:
        k, edges = I.PATTERNS[name]
        c = oracle_mod.bruteforce_count(off, cols, k, edges)
        assert c % oracle_mod.compile_pattern(k, edges)["aut"] == 0


@pytest.mark.parametrize("name", ["triangle", "4-cycle", "house"])
def test_gnp_mean_count_matches_expectation(oracle_mod, name):
    # over G(n, p) instances every injective map is an embedding with probability
    # p^|E_P|, so E[C(G,P)] = n^(k) p^|E_P|: the brute-force counts and the oracle's
    # estimates (unbiased per instance, Thm. 2) must both average to it
    n, p, reps = 10, 0.5, 240
    k, edges = I.PATTERNS[name]
    expect = falling(n, k) * p ** len(edges)
    exact, est = [], []
    for seed in range(reps):
        off, cols = I.gnp_graph(n, p, 1000 + seed)
        exact.append(oracle_mod.bruteforce_count(off, cols, k, edges))
        q = oracle_mod.Query(off, cols, k, edges, mode=oracle_mod.MODE_APPROX, seed=seed + 1)
        est.append(q.sums(0, 512)["sum_x"] / 512)
    for vals in (np.array(exact, dtype=float), np.array(est)):
        se = vals.std(ddof=1) / np.sqrt(reps)
        assert abs(vals.mean() - expect) <= 4.5 * se, (vals.mean(), expect, se)


def _sec_search(L, w):
    nbytes = max(L, 1) * w
    if nbytes <= 32:
        return 1
    return math.ceil(math.log2(-(-nbytes // 32))) + 1


@pytest.mark.parametrize("name", ["triangle", "4-cycle", "house", "4-clique", "3-path", "5-cycle",
                                  "diamond", "chordal-5-cycle"])
@pytest.mark.parametrize("mode", MODES)
def test_sector_model_restated(oracle_mod, name, mode):
    # The algorithmic-sector model (this build's cost model; the kernel counts the
    # same one, checked on the GPU) restated from its definition, trial by trial
    # from the oracle's trajectories: step 1 a search over the nv+1 running weights
    # (+1 for q); one backward edge: offsets, i-1 membership searches in the row, a
    # row-prefix search and q where weights are read, the chosen entry; several: one
    # offsets sector each, a scan of the shortest row, per other row the cheaper of a
    # merge and one search per scanned entry, one q per candidate where weights are
    # read.  Weights are read under f_approx except on a later step whose
    # configuration has no F1, I1 or F2 term (equal weights on S_tau).
    # Column 1 is the streamed part (the scan and the rows read once by a merge);
    # column 2 the plain count: a search per scanned entry in every other row and
    # the weights of every step D(i) puts under f_approx.
    off, cols = I.rmat_graph(8, 8, seed=9)
    k, edges = I.PATTERNS[name]
    q = oracle_mod.Query(off, cols, k, edges, mode=mode, seed=5)
    info = q.info()
    back = oracle_mod.compile_pattern(k, edges)["back"]
    nv = len(off) - 1
    deg = np.diff(off)
    adj = [set(cols[off[v]:off[v + 1]].tolist()) for v in range(nv)]
    emb, hit, x, sec = q.trials(0, 400)
    for t in range(len(emb)):
        tau = emb[t]
        want = _sec_search(nv + 1, 8) + (1 if info["use_approx"][0] else 0)
        streamed, plain = 0, want
        for i in range(1, k):
            reads = info["use_approx"][i] and any(info["cfg"][i][1:])
            rows = [int(tau[j]) for j in back[i]]
            if len(rows) == 1:
                d = int(deg[rows[0]])
                base = 1 + (i - 1) * _sec_search(d, 4) + 1
                want += base + ((_sec_search(d, 8) + 1) if reads else 0)
                plain += base + ((_sec_search(d, 8) + 1) if info["use_approx"][i] else 0)
            else:
                ds = [int(deg[u]) for u in rows]
                a = ds.index(min(ds))
                scan = -(-4 * ds[a] // 32)
                want += len(rows) + scan
                plain += len(rows) + scan
                streamed += scan
                for b, m in enumerate(ds):
                    if b != a:
                        merge, search = -(-4 * max(m, 1) // 32), ds[a] * _sec_search(m, 4)
                        want += min(merge, search)
                        streamed += merge if merge < search else 0
                        plain += search
                S = set.intersection(*[adj[u] for u in rows]) - set(int(v) for v in tau[:i])
                if reads:
                    want += len(S)
                if info["use_approx"][i]:
                    plain += len(S)
            if tau[i] < 0:
                break
        assert list(sec[t]) == [want, streamed, plain], (t, list(tau))


# ---------------------------------------------------------------- sampler (Alg. 3, Thm. 2)

@pytest.mark.parametrize("gname", sorted(TINY_GRAPHS))
@pytest.mark.parametrize("mode", MODES)
def test_unbiased_exact_expectation(oracle_mod, gname, mode):
    """Thm. 2: summing p_tau * X_tau over every branch of Alg. 3 gives C(G,P)."""
    off, cols = TINY_GRAPHS[gname]()
    for name in SMALL_PATTERNS:
        k, edges = I.PATTERNS[name]
        truth = oracle_mod.bruteforce_count(off, cols, k, edges)
        q = oracle_mod.Query(off, cols, k, edges, mode=mode)
        mean, second, nsucc = q.enumerate()
        assert nsucc == truth, (name, "each embedding is exactly one successful trajectory")
        assert mean == pytest.approx(truth, rel=1e-12, abs=1e-12), name
        assert second >= mean * mean * (1 - 1e-12)


def test_kstar_zero_variance(oracle_mod):
    """Sec. 3.2: f_approx on the k-star returns k! * sum binom(d, k) on every trial."""
    off, cols = I.gnp_graph(40, 0.2, 21)
    deg = np.diff(off)
    for leaves in (2, 3, 4):
        k, edges = I.star(leaves)
        want = math.factorial(leaves) * sum(math.comb(int(d), leaves) for d in deg)
        q = oracle_mod.Query(off, cols, k, edges, mode=1)
        _, hit, x, _ = q.trials(0, 2000)
        assert hit.all()
        assert np.allclose(x, want, rtol=1e-12, atol=0)
        assert oracle_mod.bruteforce_count(off, cols, k, edges) == want


@pytest.mark.parametrize("name", ["triangle", "4-cycle", "house", "4-clique", "5-cycle", "chordal-5-cycle"])
def test_complete_graph_constant_output(oracle_mod, name):
    """On K_n every candidate has the same weight, so X = n!/(n-k)! always."""
    off, cols = I.complete_graph(9)
    k, edges = I.PATTERNS[name]
    for mode in MODES:
        q = oracle_mod.Query(off, cols, k, edges, mode=mode)
        _, hit, x, _ = q.trials(0, 500)
        assert hit.all()
        assert np.allclose(x, falling(9, k), rtol=1e-13, atol=0)


def circulant_sq(n):
    a = np.arange(n)
    return I.csr_from_edges(n, np.concatenate([a, a]), np.concatenate([(a + 1) % n, (a + 2) % n]))


def test_triangle_eta_closed_form(oracle_mod):
    """Eq. alpha-def: with the exact clustering coefficient, a successful triangle
    trajectory (v1, v2, v3) returns C(G,P) * (1 + eta) with
    1 + eta = sum_{v in N(v1)} (d(v)-1) * |N(v1) & N(v2)| / (d(v2)-1) / (d(v1)(d(v1)-1)C_v1)."""
    off, cols = I.disjoint_union(circulant_sq(9), I.complete_graph(5), I.complete_graph(4), circulant_sq(11))
    n = len(off) - 1
    deg = np.diff(off)
    nbr = [set(cols[off[v]:off[v + 1]].tolist()) for v in range(n)]
    tri_at = [sum(1 for a, b in itertools.combinations(sorted(nbr[v]), 2) if b in nbr[a]) for v in range(n)]
    # exact C_v = T(v) / binom(d, 2) written as hits / d (integer on these graphs)
    hits = np.array([2 * tri_at[v] // (deg[v] - 1) for v in range(n)], dtype=np.uint32)
    assert all(2 * tri_at[v] % (deg[v] - 1) == 0 for v in range(n))
    nsum, _ = oracle_mod.graph_stats(off, cols)
    k, edges = I.PATTERNS["triangle"]
    C = oracle_mod.bruteforce_count(off, cols, k, edges)
    q = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, mode=1)
    emb, hit, x, _ = q.trials(0, 3000)
    assert hit.all()
    for t in range(len(x)):
        v1, v2 = int(emb[t, 0]), int(emb[t, 1])
        cv1 = tri_at[v1] / math.comb(int(deg[v1]), 2)
        one_eta = (sum(int(deg[v]) - 1 for v in nbr[v1]) * len(nbr[v1] & nbr[v2]) / (int(deg[v2]) - 1)
                   / (int(deg[v1]) * (int(deg[v1]) - 1) * cv1))
        assert x[t] == pytest.approx(C * one_eta, rel=1e-12)


@pytest.mark.parametrize("pair", [("triangle", lambda: I.random_tree(25, 3)),
                                  ("4-cycle", lambda: I.star_graph(12)),
                                  ("4-clique", lambda: I.disjoint_union(I.cycle_graph(8), I.random_tree(10, 1))),
                                  ("5-cycle", lambda: I.complete_graph(4))])
def test_zero_when_closing_edge_absent(oracle_mod, pair):
    name, gfun = pair
    off, cols = gfun()
    k, edges = I.PATTERNS[name]
    assert oracle_mod.bruteforce_count(off, cols, k, edges) == 0
    for mode in MODES:
        q = oracle_mod.Query(off, cols, k, edges, mode=mode)
        _, hit, x, _ = q.trials(0, 400)
        assert not hit.any() and (x == 0).all()


def test_empirical_trajectory_frequencies(oracle_mod):
    """The inverse-CDF draw reproduces the exact trajectory probabilities (chi-square)."""
    off, cols = I.gnp_graph(8, 0.55, 13)
    k, edges = I.PATTERNS["tailed-triangle"]
    for mode in MODES:
        q = oracle_mod.Query(off, cols, k, edges, mode=mode, seed=77)
        emb, hit, _, _ = q.trials(0, 30000)
        succ = emb[hit.astype(bool), :k]
        keys, counts = np.unique(succ, axis=0, return_counts=True)
        probs = np.array([q.trajectory_prob(list(t)) for t in keys])
        assert (probs > 0).all()
        # every successful trajectory seen has positive probability; the seen mass is
        # compared bin by bin against the exact probabilities
        n = 30000
        expected = probs * n
        big = expected >= 5
        stat = ((counts[big] - expected[big]) ** 2 / expected[big]).sum()
        dof = max(1, int(big.sum()) - 1)
        assert scipy.stats.chi2.sf(stat, dof) > 1e-4


def test_sample_mean_matches_exact_moments(oracle_mod):
    off, cols = I.gnp_graph(12, 0.45, 7)
    for name in ("house", "4-clique", "5-cycle"):
        k, edges = I.PATTERNS[name]
        for mode in MODES:
            q = oracle_mod.Query(off, cols, k, edges, mode=mode, seed=3)
            mean, second, _ = q.enumerate()
            n = 20000
            s = q.sums(0, n)
            sd = math.sqrt(max(second - mean * mean, 0.0) / n)
            assert abs(s["sum_x"] / n - mean) <= 5 * sd + 1e-9 * mean


def test_confidence_interval_coverage(oracle_mod):
    """Alg. 1's 95% interval covers the brute-force count in at least 90% of 200 seeded runs."""
    off, cols = I.gnp_graph(14, 0.4, 17)
    k, edges = I.PATTERNS["4-cycle"]
    truth = oracle_mod.bruteforce_count(off, cols, k, edges)
    z = oracle_mod.z_of_delta(0.05)
    cover = 0
    for seed in range(200):
        q = oracle_mod.Query(off, cols, k, edges, mode=0, seed=1000 + seed)
        r = q.estimate(eps=0.05, delta=0.05, chunk=256, min_trials=256, max_trials=1 << 16)
        half = z * math.sqrt(r["var"] / r["trials"])
        cover += abs(r["mean"] - truth) <= half
    assert cover >= 180


def test_estimate_stops_at_first_converged_checkpoint(oracle_mod):
    off, cols = I.gnp_graph(30, 0.3, 1)
    k, edges = I.PATTERNS["triangle"]
    q = oracle_mod.Query(off, cols, k, edges, mode=0, seed=9)
    r = q.estimate(eps=0.02, delta=0.05, chunk=128, min_trials=128, max_trials=1 << 20)
    assert r["converged"] == 1 and r["trials"] % 128 == 0
    z = oracle_mod.z_of_delta(0.05)
    # the previous checkpoint had not converged
    prev = q.sums(0, r["trials"] - 128)
    n = prev["trials"]
    mu = prev["sum_x"] / n
    var = max(prev["sum_x2"] / n - mu * mu, 0.0)
    assert n < 128 or z * math.sqrt(var) / math.sqrt(n) / mu > 0.02
    s = q.sums(0, r["trials"])
    assert s["sum_x"] == pytest.approx(r["sum_x"], rel=1e-12)


def test_trials_are_reproducible_and_independent_of_range_split(oracle_mod):
    off, cols = I.gnp_graph(20, 0.35, 2)
    k, edges = I.PATTERNS["house"]
    q = oracle_mod.Query(off, cols, k, edges, seed=4)
    e1, h1, x1, s1 = q.trials(0, 300)
    e2, h2, x2, s2 = q.trials(100, 200)
    assert (e1[100:] == e2).all() and (x1[100:] == x2).all() and (s1[100:] == s2).all()
    q2 = oracle_mod.Query(off, cols, k, edges, seed=5)
    _, _, x3, _ = q2.trials(0, 300)
    assert not (x3 == x1).all()


def test_min_trials_gate(oracle_mod):
    """Alg. 1 is only consulted once min_trials trials are in (zero-variance case)."""
    off, cols = I.complete_graph(9)
    k, edges = I.PATTERNS["triangle"]
    q = oracle_mod.Query(off, cols, k, edges, mode=0, seed=2)
    r = q.estimate(eps=0.01, delta=0.05, chunk=64, min_trials=256, max_trials=4096)
    assert r["converged"] == 1 and r["trials"] == 256
    r = q.estimate(eps=0.01, delta=0.05, chunk=64, min_trials=64, max_trials=4096)
    assert r["trials"] == 64


@pytest.mark.parametrize("gname", sorted(TINY_GRAPHS))
def test_exact_counters_match_bruteforce(oracle_mod, gname):
    off, cols = TINY_GRAPHS[gname]()
    for name in ("triangle", "4-cycle", "4-clique"):
        k, edges = I.PATTERNS[name]
        assert oracle_mod.exact_count(off, cols, name) == oracle_mod.bruteforce_count(off, cols, k, edges)


def test_exact_counters_on_rmat_match_bruteforce(oracle_mod):
    off, cols = I.rmat_graph(7, 8, seed=2)
    for name in ("triangle", "4-cycle", "4-clique"):
        k, edges = I.PATTERNS[name]
        assert oracle_mod.exact_count(off, cols, name) == oracle_mod.bruteforce_count(off, cols, k, edges)
