"""Pattern concentration (Sec. 6.3): the connected-pattern catalogue, the
non-induced -> induced conversion, and GPU concentrations against brute force."""
import itertools

import networkx as nx
import numpy as np
import pytest

from paper_2601_01388_b300 import concentration as K
from paper_2601_01388_b300 import inputs as I
from tests.test_oracle_pins import nx_graph, nx_pattern


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_catalogue_matches_graph_atlas(k):
    """Connected graphs up to isomorphism: 1, 1, 2, 6, 21, 112 (networkx's atlas of all
    graphs on at most 7 vertices)."""
    pats = K.connected_patterns(k)
    atlas = [g for g in nx.graph_atlas_g() if g.number_of_nodes() == k and nx.is_connected(g)]
    assert len(pats) == len(atlas) == [1, 1, 2, 6, 21, 112][k - 1]
    gs = [nx_pattern(*p) for p in pats]
    assert all(nx.is_connected(g) for g in gs)
    for a, b in itertools.combinations(range(len(gs)), 2):
        if gs[a].number_of_edges() == gs[b].number_of_edges():
            assert not nx.is_isomorphic(gs[a], gs[b])
    # every atlas graph has exactly one match in the catalogue
    for g in atlas:
        assert sum(nx.is_isomorphic(g, h) for h in gs) == 1


def test_spanning_matrix_small_cases():
    pats = K.connected_patterns(4)
    names = {frozenset(map(frozenset, I.PATTERNS[n][1])): n for n in ("4-cycle", "4-clique", "3-star", "4-path")}
    S = K.spanning_matrix(4)
    idx = {}
    for i, p in enumerate(pats):
        for n in ("4-cycle", "4-clique", "3-star", "4-path"):
            if nx.is_isomorphic(nx_pattern(*p), nx_pattern(*I.PATTERNS[n])):
                idx[n] = i
    assert len(idx) == 4 and names
    # a 4-clique holds 3 spanning 4-cycles, 12 Hamiltonian paths and 4 spanning stars
    assert S[idx["4-cycle"], idx["4-clique"]] == 3
    assert S[idx["4-path"], idx["4-clique"]] == 12
    assert S[idx["3-star"], idx["4-clique"]] == 4
    assert S[idx["4-path"], idx["4-cycle"]] == 4
    assert S[idx["3-star"], idx["4-cycle"]] == 0


def induced_by_bruteforce(off, cols, k):
    g = nx_graph(off, cols)
    pats = [nx_pattern(*p) for p in K.connected_patterns(k)]
    out = np.zeros(len(pats), dtype=np.int64)
    for s in itertools.combinations(range(len(off) - 1), k):
        h = g.subgraph(s)
        if h.number_of_edges() < k - 1 or not nx.is_connected(h):
            continue
        for i, p in enumerate(pats):
            if p.number_of_edges() == h.number_of_edges() and nx.is_isomorphic(h, p):
                out[i] += 1
                break
    return out


@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("gfun", [lambda: I.gnp_graph(11, 0.45, 2), lambda: I.rmat_graph(4, 4, seed=9),
                                  lambda: I.disjoint_union(I.complete_graph(5), I.cycle_graph(6))])
def test_noninduced_equals_spanning_times_induced(oracle_mod, k, gfun):
    off, cols = gfun()
    ind = induced_by_bruteforce(off, cols, k)
    emb = [oracle_mod.bruteforce_count(off, cols, *p) for p in K.connected_patterns(k)]
    sub = K.subgraph_counts(emb, k)
    assert np.array_equal(sub, np.round(sub))
    assert np.array_equal(K.spanning_matrix(k) @ ind, sub.astype(np.int64))
    assert np.allclose(K.induced_counts(sub, k), ind, rtol=0, atol=1e-9)


def test_concentration_and_distance():
    c = K.concentration([1.0, 3.0, 0.0, 4.0])
    assert np.allclose(c, [0.125, 0.375, 0.0, 0.5])
    assert K.variation_distance(c, c) == 0.0
    assert K.variation_distance([1, 0], [0, 1]) == 1.0


# ---------------------------------------------------------------- GPU

@pytest.fixture(scope="module")
def agis():
    from tests.conftest import has_gpu
    if not has_gpu():
        pytest.skip("needs a CUDA device")
    from paper_2601_01388_b300 import build
    build.build()
    from paper_2601_01388_b300 import agis as A
    return A


@pytest.mark.gpu
@pytest.mark.parametrize("k", [4, 5])
def test_gpu_concentration_matches_bruteforce(agis, oracle_mod, k):
    """All connected k-vertex patterns as one batch at +-1% (95%): each estimate equals
    the oracle's Alg. 1 run with the same seed, the concentration vector is within 0.01
    variation distance of the brute-force one, and the induced conversion (which
    amplifies relative errors: a rare induced pattern is a small difference of large
    non-induced counts) within 0.1."""
    off, cols = I.rmat_graph(7, 8, seed=4)
    ctx = agis.Context(0)
    g = agis.Graph(ctx, off, cols, validate=True)
    g.preprocess(1, 2.0 ** -10)
    pats = K.connected_patterns(k)
    ps = [agis.Pattern(*p) for p in pats]
    opts = [agis.default_opts(eps=0.01, delta=0.05, seed=50 + i, chunk_trials=1 << 14, min_trials=1 << 14,
                              max_trials=1 << 30) for i in range(len(ps))]
    rs = agis.estimate_batch(g, ps, opts)
    assert all(r["converged"] for r in rs)
    for i, (p, r) in enumerate(zip(pats, rs)):
        o = oracle_mod.Query(off, cols, *p, seed=50 + i).estimate(
            eps=0.01, delta=0.05, chunk=1 << 14, min_trials=1 << 14, max_trials=1 << 30)
        assert r["trials"] == o["trials"] and r["hits"] == o["hits"]
        assert r["estimate"] == pytest.approx(o["mean"], rel=1e-9)
    est = K.subgraph_counts([r["estimate"] for r in rs], k)
    truth = K.subgraph_counts([oracle_mod.bruteforce_count(off, cols, *p) for p in pats], k)
    assert K.variation_distance(K.concentration(est), K.concentration(truth)) < 0.01
    ind_t = K.induced_counts(truth, k)
    ind_e = np.maximum(K.induced_counts(est, k), 0.0)
    assert K.variation_distance(K.concentration(ind_e), K.concentration(ind_t)) < 0.1
