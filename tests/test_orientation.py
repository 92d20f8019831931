"""Degree-ordered orientation for clique patterns (Sec. 5.4): on the DAG that keeps
u -> v when (d(u), u) < (d(v), v), every k-clique is one trajectory, so Alg. 3 on
the out-rows estimates the number of cliques.  CPU: the oracle's orientation and
its unbiasedness (Thm. 2) against brute force.  GPU: the device orientation, its
statistics and trials bit-identical to the oracle, and the reported counts."""
import math
import time

import numpy as np
import pytest

from paper_2601_01388_b300 import inputs as I
from tests.test_oracle_pins import TINY_GRAPHS

CMIN = 2.0 ** -10
CLIQUES = ["triangle", "4-clique", "5-clique"]


def undirected_edges(off, cols):
    s, d = I.edges_of(off, cols)
    return {(min(a, b), max(a, b)) for a, b in zip(s.tolist(), d.tolist())}


@pytest.mark.parametrize("gname", sorted(TINY_GRAPHS))
def test_orientation_keeps_each_edge_once_upward(oracle_mod, gname):
    off, cols = TINY_GRAPHS[gname]()
    oo, oc = oracle_mod.orient(off, cols)
    deg = np.diff(off)
    assert len(oc) * 2 == len(cols)
    arcs = [(u, int(v)) for u in range(len(deg)) for v in oc[oo[u]:oo[u + 1]]]
    assert {(min(a, b), max(a, b)) for a, b in arcs} == undirected_edges(off, cols)
    for u, v in arcs:
        assert (deg[u], u) < (deg[v], v)
    for u in range(len(deg)):
        row = oc[oo[u]:oo[u + 1]]
        assert (np.diff(row) > 0).all()
        # out-neighbours have degree >= d+(u) each, so d+(u)^2 <= 2|E|
        assert (oo[u + 1] - oo[u]) ** 2 <= len(cols)


@pytest.mark.parametrize("gname", sorted(TINY_GRAPHS))
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_oriented_sampler_counts_cliques(oracle_mod, gname, mode):
    """Thm. 2 on the orientation: the exact expectation is the number of cliques,
    C(G, K_k) / k!, and each clique is exactly one successful trajectory."""
    off, cols = TINY_GRAPHS[gname]()
    oo, oc = oracle_mod.orient(off, cols)
    for name in CLIQUES:
        k, edges = I.PATTERNS[name]
        cliques = oracle_mod.bruteforce_count(off, cols, k, edges) // math.factorial(k)
        q = oracle_mod.Query(oo, oc, k, edges, mode=mode, oriented=True)
        mean, _, nsucc = q.enumerate()
        assert nsucc == cliques
        assert mean == pytest.approx(cliques, rel=1e-12, abs=1e-12), (name, gname)


@pytest.mark.parametrize("gname", ["gnp10", "gnp12", "k6", "mixed"])
def test_oriented_anchor_draw_counts_cliques(oracle_mod, gname):
    """The anchor draw on the orientation: still one trajectory per clique."""
    off, cols = TINY_GRAPHS[gname]()
    oo, oc = oracle_mod.orient(off, cols)
    for name in CLIQUES:
        k, edges = I.PATTERNS[name]
        cliques = oracle_mod.bruteforce_count(off, cols, k, edges) // math.factorial(k)
        for mode in (1, 2):
            q = oracle_mod.Query(oo, oc, k, edges, mode=mode, oriented=True, anchor=True)
            mean, _, nsucc = q.enumerate()
            assert nsucc == cliques
            assert mean == pytest.approx(cliques, rel=1e-12, abs=1e-12)


def test_oriented_weight_takes_no_backward_vertices(oracle_mod):
    """On an orientation a k-clique's first vertex needs k - 1 out-neighbours, so the
    step-1 weight is binom(d+, k - 1) times the other factors; a vertex with fewer
    out-neighbours is never drawn."""
    off, cols = I.gnp_graph(40, 0.3, 12)
    oo, oc = oracle_mod.orient(off, cols)
    k, edges = I.PATTERNS["4-clique"]
    q = oracle_mod.Query(oo, oc, k, edges, mode=1, oriented=True, seed=3)
    emb, hit, x, _ = q.trials(0, 3000)
    dplus = np.diff(oo)
    assert (dplus[emb[:, 0]] >= 3).all()
    assert hit.any()


def test_non_clique_on_orientation_rejected(oracle_mod):
    off, cols = I.gnp_graph(12, 0.4, 1)
    oo, oc = oracle_mod.orient(off, cols)
    with pytest.raises(ValueError):
        oracle_mod.Query(oo, oc, *I.PATTERNS["4-cycle"], oriented=True)


# ---------------------------------------------------------------- GPU

GRAPHS = {
    "rmat12": lambda: I.rmat_graph(12, 16, seed=3),
    "gnp60": lambda: I.gnp_graph(60, 0.15, 4),
    "k9": lambda: I.complete_graph(9),
    "isolated": lambda: I.disjoint_union(I.cycle_graph(9), I.csr_from_edges(5, np.array([0]), np.array([0]))),
}


@pytest.fixture(scope="module")
def agis():
    from tests.conftest import has_gpu
    if not has_gpu():
        pytest.skip("needs a CUDA device")
    from paper_2601_01388_b300 import build
    build.build()
    from paper_2601_01388_b300 import agis as A
    return A


@pytest.fixture(scope="module")
def oriented(agis, oracle_mod):
    ctx = agis.Context(0)
    out = {}
    for name, fn in GRAPHS.items():
        off, cols = fn()
        g = agis.Graph(ctx, off, cols, validate=True)
        o = g.orient()
        o.preprocess(1, CMIN)
        oo, oc = oracle_mod.orient(off, cols)
        nsum, hits = oracle_mod.graph_stats(oo, oc, 1)
        out[name] = (off, cols, g, o, oo, oc, nsum, hits)
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("gname", sorted(GRAPHS))
def test_device_orientation_bit_exact(agis, oriented, gname):
    off, cols, g, o, oo, oc, nsum, hits = oriented[gname]
    assert o.oriented and not g.oriented
    doff, dcols = o.csr()
    assert np.array_equal(doff, oo) and np.array_equal(dcols, oc)
    assert o.info()["nnz"] * 2 == g.info()["nnz"]
    o.validate()
    gn, gh = o.stats()
    assert np.array_equal(gn, nsum) and np.array_equal(gh, hits)
    with pytest.raises(agis.AgisError) as e:
        o.orient()
    assert e.value.status == agis.ERR_STATE


@pytest.mark.gpu
@pytest.mark.parametrize("gname", sorted(GRAPHS))
@pytest.mark.parametrize("name", ["triangle", "4-clique", "5-clique", "6-clique"])
def test_oriented_trials_bit_exact(agis, oracle_mod, oriented, gname, name):
    off, cols, g, o, oo, oc, nsum, hits = oriented[gname]
    k, edges = I.PATTERNS[name]
    p = agis.Pattern(k, edges)
    for mode in (0, 1, 2):
        for anchor in (0, 1):
            emb, hit, x, sec = agis.dump_trials(o, p, agis.default_opts(mode=mode, seed=9, anchor=anchor), 1000, 2100)
            q = oracle_mod.Query(oo, oc, k, edges, nsum=nsum, hits=hits, c_min=CMIN, mode=mode, seed=9,
                                 oriented=True, anchor=bool(anchor))
            oemb, ohit, ox, osec = q.trials(1000, 2100)
            bad = np.nonzero((emb != oemb).any(axis=1) | (hit != ohit) | (x != ox) | (sec != osec).any(axis=1))[0]
            assert len(bad) == 0, (name, mode, anchor, int(bad[0]))


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["triangle", "4-clique"])
@pytest.mark.parametrize("mode", [1, 2])
def test_oriented_estimates_cover_exact_counts(agis, oracle_mod, name, mode):
    """R-MAT scale 14, 2^20 trials on the orientation: estimate = cliques * k! lies
    within 4 standard errors of the exact embedding count; subgraphs = cliques."""
    ctx = agis.Context(0)
    off, cols = I.rmat_graph(14, 16, 0.57, 0.19, 0.19, seed=1)
    o = agis.Graph(ctx, off, cols).orient()
    o.preprocess(1, CMIN)
    k, edges = I.PATTERNS[name]
    n = 1 << 20
    r = agis.estimate(o, agis.Pattern(k, edges), agis.default_opts(mode=mode, seed=1, eps=0.0, max_trials=n))
    truth = oracle_mod.exact_count(off, cols, name)
    f = math.factorial(k)
    assert r["estimate"] == pytest.approx(r["mean"] * f, rel=1e-15)
    assert r["subgraphs"] == pytest.approx(r["mean"], rel=1e-15)
    se = (r["var"] / n) ** 0.5 * f
    assert abs(r["estimate"] - truth) <= 4 * se + 1e-9 * truth, (r["estimate"], truth, se)


@pytest.mark.gpu
def test_oriented_batch_server_and_rejection(agis, oriented):
    off, cols, g, o, *_ = oriented["rmat12"]
    names = ["triangle", "4-clique", "5-clique"]
    pats = [agis.Pattern(*I.PATTERNS[n]) for n in names]
    opts = [agis.default_opts(seed=20 + i, eps=0.02, chunk_trials=1 << 14, min_trials=1 << 14,
                              max_trials=1 << 24) for i in range(3)]
    single = [agis.estimate(o, p, op) for p, op in zip(pats, opts)]
    batch = agis.estimate_batch(o, pats, opts)
    for a, b in zip(single, batch):
        assert a["trials"] == b["trials"] and a["estimate"] == b["estimate"]
    srv = agis.Server(o, 1 << 30, 8)
    try:
        tk = [srv.submit(p, op) for p, op in zip(pats, opts)]
        for t, a in zip(tk, single):
            t0 = time.time()
            r = srv.poll(t)
            while r is None and time.time() - t0 < 120:
                time.sleep(0.001)
                r = srv.poll(t)
            assert r is not None
            assert r["trials"] == a["trials"] and r["estimate"] == a["estimate"]
    finally:
        srv.close()
    with pytest.raises(agis.AgisError) as e:
        agis.estimate(o, agis.Pattern(*I.PATTERNS["4-cycle"]), agis.default_opts())
    assert e.value.status == agis.ERR_PATTERN
