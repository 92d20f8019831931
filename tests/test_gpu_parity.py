"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work (trajectories, hit flags, tables, prefix sums, sector counts) must
be bit-identical; FP64 sampler outputs are bit-identical too because each one is
the same sequence of IEEE products and quotients; FP64 sums over many trials are
compared at 1e-9 relative (summation order differs).
"""
import numpy as np
import pytest

from paper_2601_01388_b300 import inputs as I

pytestmark = pytest.mark.gpu

CMIN = 2.0 ** -10
REL = 1e-9
MODES = (0, 1, 2)


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
def ctx(agis):
    return agis.Context(0)


def make_graph(agis, ctx, off, cols, seed=1):
    g = agis.Graph(ctx, off, cols, validate=True)
    g.preprocess(seed, CMIN)
    return g


GRAPHS = {
    "rmat12": lambda: I.rmat_graph(12, 16, seed=3),
    "rmat10_unpermuted": lambda: I.rmat_graph(10, 8, seed=5, permute=False),
    "gnp60": lambda: I.gnp_graph(60, 0.15, 4),
    "k7": lambda: I.complete_graph(7),
    "star20_tree": lambda: I.disjoint_union(I.star_graph(20), I.random_tree(15, 8)),
    "isolated": lambda: I.disjoint_union(I.cycle_graph(9), I.csr_from_edges(5, np.array([0]), np.array([0]))),
}


@pytest.fixture(scope="module")
def graphs(agis, ctx, oracle_mod):
    out = {}
    for name, fn in GRAPHS.items():
        off, cols = fn()
        g = make_graph(agis, ctx, off, cols)
        nsum, hits = oracle_mod.graph_stats(off, cols, 1)
        out[name] = (off, cols, g, nsum, hits)
    return out


# ------------------------------------------------------------------ preprocessing

@pytest.mark.parametrize("gname", sorted(GRAPHS))
def test_preprocess_bit_exact(graphs, gname):
    off, cols, g, nsum, hits = graphs[gname]
    gn, gh = g.stats()
    assert (gn == nsum).all()
    assert (gh == hits).all()


@pytest.mark.parametrize("gname", ["rmat12", "gnp60", "star20_tree", "isolated"])
@pytest.mark.parametrize("cfg", [(0, 4, 3, 0), (0, 3, 1, 2), (0, 2, 0, 2), (1, 2, 0, 1), (1, 1, 0, 0),
                                 (2, 2, 1, 0), (3, 1, 0, 0), (0, 7, 6, 0), (1, 0, 0, 0)])
def test_weight_tables_bit_exact(graphs, oracle_mod, gname, cfg):
    off, cols, g, nsum, hits = graphs[gname]
    q, pref, shift = g.weight_table(cfg)
    oq, oshift = oracle_mod.weight_table(off, nsum, hits, CMIN, cfg)
    assert shift == oshift
    assert (q == oq).all()
    assert (pref == np.cumsum(oq, dtype=np.uint64)).all()
    rp = g.row_prefix(cfg)
    deg = np.diff(off)
    want = np.zeros(len(cols), dtype=np.uint64)
    for v in np.nonzero(deg)[0]:
        s, e = off[v], off[v + 1]
        want[s:e] = np.cumsum(oq[cols[s:e]], dtype=np.uint64)
    assert (rp == want).all()


# ------------------------------------------------------------------ trials

def compare_dumps(agis, oracle_mod, off, cols, g, nsum, hits, name, mode, first, count, seed=7):
    k, edges = I.PATTERNS[name]
    p = agis.Pattern(k, edges)
    opts = agis.default_opts(mode=mode, seed=seed)
    emb, hit, x, sec = agis.dump_trials(g, p, opts, first, count)
    q = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, c_min=CMIN, mode=mode, seed=seed)
    oemb, ohit, ox, osec = q.trials(first, count)
    bad = np.nonzero((emb != oemb).any(axis=1) | (hit != ohit) | (x != ox) | (sec != osec).any(axis=1))[0]
    assert len(bad) == 0, (name, mode, int(bad[0]), emb[bad[0]], oemb[bad[0]], x[bad[0]], ox[bad[0]],
                           sec[bad[0]], osec[bad[0]])
    return hit


@pytest.mark.parametrize("name", sorted(I.PATTERNS))
@pytest.mark.parametrize("mode", MODES)
def test_trials_bit_exact_rmat(agis, oracle_mod, graphs, name, mode):
    off, cols, g, nsum, hits = graphs["rmat12"]
    # three tiles with a ragged tail, at an offset into the trial sequence
    hit = compare_dumps(agis, oracle_mod, off, cols, g, nsum, hits, name, mode, 5000, 2500)
    if name in ("triangle", "edge", "3-path", "3-star"):
        assert hit.sum() > 0


@pytest.mark.parametrize("gname", ["rmat10_unpermuted", "gnp60", "k7", "star20_tree", "isolated"])
@pytest.mark.parametrize("name", ["triangle", "4-cycle", "4-clique", "house", "5-cycle", "4-star",
                                  "chordal-5-cycle", "edge"])
def test_trials_bit_exact_small_graphs(agis, oracle_mod, graphs, gname, name):
    off, cols, g, nsum, hits = graphs[gname]
    for mode in MODES:
        compare_dumps(agis, oracle_mod, off, cols, g, nsum, hits, name, mode, 0, 1100)


def test_eight_vertex_pattern(agis, oracle_mod, graphs):
    off, cols, g, nsum, hits = graphs["gnp60"]
    rng = np.random.Generator(np.random.Philox(key=[77, 0]))
    for _ in range(6):
        k, edges = I.random_connected_pattern(rng, 8, 8, 0.4)
        p = agis.Pattern(k, edges)
        for mode in MODES:
            opts = agis.default_opts(mode=mode, seed=11)
            emb, hit, x, sec = agis.dump_trials(g, p, opts, 0, 1024)
            q = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, c_min=CMIN, mode=mode, seed=11)
            oemb, ohit, ox, osec = q.trials(0, 1024)
            assert (emb == oemb).all() and (hit == ohit).all() and (x == ox).all() and (sec == osec).all()


# ------------------------------------------------------------------ estimates

@pytest.mark.parametrize("name", ["triangle", "4-clique", "house", "5-cycle"])
@pytest.mark.parametrize("mode", MODES)
def test_fixed_budget_sums(agis, oracle_mod, graphs, name, mode):
    off, cols, g, nsum, hits = graphs["rmat12"]
    k, edges = I.PATTERNS[name]
    n = 40000  # 39 full tiles and a ragged one
    opts = agis.default_opts(mode=mode, seed=3, eps=0.0, max_trials=n, chunk_trials=8192)
    r = agis.estimate(g, agis.Pattern(k, edges), opts)
    q = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, c_min=CMIN, mode=mode, seed=3)
    s = q.sums(0, n)
    assert r["trials"] == n and r["hits"] == s["hits"] and r["sectors"] == s["sectors"]
    assert r["sectors_streamed"] == s["sectors_streamed"] and r["sectors_survey"] == s["sectors_survey"]
    assert r["sum_x"] == pytest.approx(s["sum_x"], rel=REL, abs=0)
    assert r["sum_x2"] == pytest.approx(s["sum_x2"], rel=REL, abs=0)


@pytest.mark.parametrize("name", ["triangle", "4-cycle", "tailed-triangle"])
def test_adaptive_matches_oracle(agis, oracle_mod, graphs, name):
    off, cols, g, nsum, hits = graphs["rmat12"]
    k, edges = I.PATTERNS[name]
    opts = agis.default_opts(mode=0, seed=5, eps=0.05, delta=0.05, chunk_trials=4096, min_trials=4096,
                             max_trials=1 << 21)
    r = agis.estimate(g, agis.Pattern(k, edges), opts)
    q = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, c_min=CMIN, mode=0, seed=5)
    o = q.estimate(eps=0.05, delta=0.05, chunk=4096, min_trials=4096, max_trials=1 << 21)
    assert r["trials"] == o["trials"] and r["converged"] == o["converged"] == 1
    assert r["hits"] == o["hits"] and r["sectors"] == o["sectors"]
    assert r["sectors_streamed"] == o["sectors_streamed"] and r["sectors_survey"] == o["sectors_survey"]
    assert r["estimate"] == pytest.approx(o["mean"], rel=REL)
    assert r["eps_hat"] == pytest.approx(o["eps_hat"], rel=1e-6)


def test_batch_equals_single(agis, graphs):
    off, cols, g, nsum, hits = graphs["rmat12"]
    names = ["triangle", "4-cycle", "4-clique", "house", "5-cycle", "tailed-triangle", "4-star"]
    pats = [agis.Pattern(*I.PATTERNS[n]) for n in names]
    opts = [agis.default_opts(mode=i % 3, seed=100 + i, eps=0.03 + 0.01 * (i % 2), delta=0.05,
                              chunk_trials=4096, min_trials=8192, max_trials=1 << 20)
            for i in range(len(names))]
    single = [agis.estimate(g, p, o) for p, o in zip(pats, opts)]
    batch = agis.estimate_batch(g, pats, opts)
    for a, b in zip(single, batch):
        for key in ("trials", "hits", "sectors", "sectors_streamed", "sectors_survey", "converged", "sum_x",
                    "sum_x2", "estimate"):
            assert a[key] == b[key], key


def test_sample_device_tiles(agis, oracle_mod, graphs):
    import torch
    off, cols, g, nsum, hits = graphs["rmat12"]
    k, edges = I.PATTERNS["house"]
    p = agis.Pattern(k, edges)
    opts = agis.default_opts(mode=0, seed=9)
    ntiles = 37
    out = torch.zeros(ntiles * agis.TILE_WORDS, dtype=torch.int64, device="cuda")
    agis.sample_device(g, p, opts, 2048, ntiles, out.data_ptr())
    torch.cuda.synchronize()
    ts = agis.tile_sums(out.cpu().numpy().view(np.uint64))
    h, sec, sx, sx2 = ts["hits"], ts["sectors"], ts["sum_x"], ts["sum_x2"]
    q = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, c_min=CMIN, mode=0, seed=9)
    T = agis.TILE
    for t in (0, 17, 36):
        s = q.sums(2048 + T * t, T)
        assert h[t] == s["hits"] and sec[t] == s["sectors"]
        assert ts["streamed"][t] == s["sectors_streamed"] and ts["survey"][t] == s["sectors_survey"]
        assert sx[t] == pytest.approx(s["sum_x"], rel=REL, abs=0)
        assert sx2[t] == pytest.approx(s["sum_x2"], rel=REL, abs=0)


# ------------------------------------------------------------------ errors

def test_invalid_graphs_rejected(agis, ctx):
    off, cols = I.cycle_graph(6)
    bad = cols.copy()
    bad[0], bad[1] = bad[1], bad[0]              # unsorted row
    with pytest.raises(agis.AgisError) as e:
        agis.Graph(ctx, off, bad, validate=True)
    assert e.value.status == agis.ERR_GRAPH
    asym = I.csr_from_edges(4, np.array([0, 1]), np.array([1, 2]))
    cols2 = asym[1].copy()
    cols2[-1] = 0                                 # 3 -> 0 without 0 -> 3... also breaks order
    with pytest.raises(agis.AgisError):
        agis.Graph(ctx, asym[0], cols2, validate=True)
    off3 = off.copy()
    off3[-1] += 1                                 # offsets disagree with nnz
    with pytest.raises(agis.AgisError):
        agis.Graph(ctx, off3, cols, validate=False)


def test_unpreprocessed_graph_is_state_error(agis, ctx):
    off, cols = I.cycle_graph(8)
    g = agis.Graph(ctx, off, cols)
    with pytest.raises(agis.AgisError) as e:
        agis.estimate(g, agis.Pattern(*I.PATTERNS["triangle"]), agis.default_opts())
    assert e.value.status == agis.ERR_STATE


def test_bad_opts_rejected(agis, graphs):
    g = graphs["k7"][2]
    with pytest.raises(agis.AgisError) as e:
        agis.estimate(g, agis.Pattern(*I.PATTERNS["triangle"]), agis.default_opts(chunk_trials=1000))
    assert e.value.status == agis.ERR_ARG


# ------------------------------------------------------------------ small configuration

@pytest.fixture(scope="module")
def rmat14(agis, ctx, oracle_mod):
    off, cols = I.rmat_graph(14, 16, 0.57, 0.19, 0.19, seed=1)
    g = make_graph(agis, ctx, off, cols)
    nsum, hits = oracle_mod.graph_stats(off, cols, 1)
    return off, cols, g, nsum, hits


@pytest.mark.parametrize("name", ["triangle", "4-cycle", "4-clique"])
@pytest.mark.parametrize("mode", [1, 2])
def test_scale14_estimates_cover_exact_counts(agis, oracle_mod, rmat14, name, mode):
    """R-MAT scale 14, 2^20 trials under f_approx (mode 1) and f_uniform (mode 2),
    Philox seed 1: the estimate lies within 4 standard errors of the exact count,
    and a prefix of the trials matches the oracle."""
    off, cols, g, nsum, hits = rmat14
    k, edges = I.PATTERNS[name]
    n = 1 << 20
    r = agis.estimate(g, agis.Pattern(k, edges), agis.default_opts(mode=mode, seed=1, eps=0.0, max_trials=n))
    truth = oracle_mod.exact_count(off, cols, name)
    se = (r["var"] / n) ** 0.5
    assert abs(r["estimate"] - truth) <= 4 * se + 1e-9 * truth, (r["estimate"], truth, se)
    q = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, c_min=CMIN, mode=mode, seed=1)
    s = q.sums(0, 8192)
    part = agis.estimate(g, agis.Pattern(k, edges), agis.default_opts(mode=mode, seed=1, eps=0.0, max_trials=8192))
    assert part["hits"] == s["hits"] and part["sectors"] == s["sectors"]
    assert part["sum_x"] == pytest.approx(s["sum_x"], rel=REL, abs=0)


# ------------------------------------------------------------------ every sampler path

def _policies(nnz):
    return {
        "bitmaps_for_degree_4_and_up": dict(bitmap_min_degree=4),
        "lists_of_64_entries": dict(list_entries=64),
        "no_row_prefix": dict(row_prefix_bytes=8),
        "row_prefix_of_top_rows": dict(row_prefix_bytes=8 * nnz // 3),
        "all_together": dict(bitmap_min_degree=16, list_entries=128, row_prefix_bytes=8 * nnz // 5),
    }


@pytest.mark.parametrize("policy", ["bitmaps_for_degree_4_and_up", "lists_of_64_entries", "no_row_prefix",
                                    "row_prefix_of_top_rows", "all_together"])
def test_trials_bit_exact_under_memory_policies(agis, ctx, oracle_mod, policy):
    """The memory policy picks among bitmap probes, merges and searches, listed and
    list-free intersections, full, partial or no row prefixes; none of it may
    change a trial."""
    off, cols = I.rmat_graph(12, 16, seed=3)
    nsum, hits = oracle_mod.graph_stats(off, cols, 1)
    g = agis.Graph(ctx, off, cols)
    g.set_memory_policy(**_policies(len(cols))[policy])
    g.preprocess(1, CMIN)
    for name in ["4-clique", "5-clique", "house", "5-cycle", "triangle", "4-path", "chordal-5-cycle",
                 "tailed-triangle", "4-star"]:
        for mode in MODES:
            compare_dumps(agis, oracle_mod, off, cols, g, nsum, hits, name, mode, 777, 1500)
    g.close()
