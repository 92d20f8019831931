"""The anchor draw for steps with several backward vertices: propose from the
shortest backward row minus the trajectory, with the step's weights, and fail the
trial unless the drawn vertex closes the other backward edges.  S_tau (Alg. 3) is
never built; Thm. 2 still makes the estimate unbiased because every extension
keeps a positive probability.  CPU: the oracle's variant against brute force and
against the exact S_tau draw.  GPU: bit-identical trials and sums."""
import numpy as np
import pytest

from paper_2601_01388_b300 import inputs as I
from tests.test_oracle_pins import TINY_GRAPHS

CMIN = 2.0 ** -10
MULTI = ["triangle", "4-cycle", "4-clique", "house", "diamond", "chordal-5-cycle", "5-clique"]


@pytest.mark.parametrize("gname", sorted(TINY_GRAPHS))
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_anchor_draw_unbiased(oracle_mod, gname, mode):
    off, cols = TINY_GRAPHS[gname]()
    for name in MULTI:
        k, edges = I.PATTERNS[name]
        truth = oracle_mod.bruteforce_count(off, cols, k, edges)
        a = oracle_mod.Query(off, cols, k, edges, mode=mode, anchor=True)
        mean, second, nsucc = a.enumerate()
        assert nsucc == truth
        assert mean == pytest.approx(truth, rel=1e-12, abs=1e-12), (name, gname)
        # per step the anchor's proposal total is at least S_tau's, so E[X^2] can only grow
        _, second_exact, _ = oracle_mod.Query(off, cols, k, edges, mode=mode).enumerate()
        assert second >= second_exact * (1 - 1e-12)


def test_anchor_draw_leaves_single_backward_patterns_alone(oracle_mod):
    """Trees (every step has one backward vertex) run the same trials either way."""
    off, cols = I.gnp_graph(40, 0.2, 6)
    for name in ("3-path", "4-path", "3-star", "4-star"):
        k, edges = I.PATTERNS[name]
        a = oracle_mod.Query(off, cols, k, edges, seed=5, anchor=True).trials(0, 2000)
        b = oracle_mod.Query(off, cols, k, edges, seed=5).trials(0, 2000)
        for u, v in zip(a, b):
            assert (u == v).all()


def test_anchor_draw_triangle_closed_form(oracle_mod):
    """Uniform triangle trials: v1 edge-uniform, v2 uniform in N(v1), v3 uniform in
    N(v1) \\ {v2} or N(v2) \\ {v1}, whichever row is shorter (v1's on ties), and it
    must be adjacent to the other: X = 2|E| (d_a - 1) on success."""
    off, cols = I.gnp_graph(30, 0.3, 2)
    deg = np.diff(off)
    k, edges = I.PATTERNS["triangle"]
    q = oracle_mod.Query(off, cols, k, edges, mode=2, seed=8, anchor=True)
    emb, hit, x, _ = q.trials(0, 4000)
    nbr = [set(cols[off[v]:off[v + 1]].tolist()) for v in range(len(deg))]
    plan = oracle_mod.compile_pattern(k, edges)
    assert plan["cfg"][2][0] == 2
    for t in range(len(x)):
        v1, v2, v3 = (int(e) for e in emb[t, :3])
        a = v1 if deg[v1] <= deg[v2] else v2
        if hit[t]:
            assert v3 in nbr[v1] and v3 in nbr[v2]
            assert x[t] == pytest.approx(len(cols) * (deg[a] - 1), rel=1e-13)
        else:
            assert x[t] == 0.0 and v3 == -1


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


@pytest.fixture(scope="module")
def graphs(agis, oracle_mod):
    ctx = agis.Context(0)
    out = {}
    for name, fn in {"rmat12": lambda: I.rmat_graph(12, 16, seed=3), "gnp60": lambda: I.gnp_graph(60, 0.15, 4),
                     "k7": lambda: I.complete_graph(7)}.items():
        off, cols = fn()
        g = agis.Graph(ctx, off, cols, validate=True)
        g.preprocess(1, CMIN)
        nsum, hits = oracle_mod.graph_stats(off, cols, 1)
        out[name] = (off, cols, g, nsum, hits)
    return out


def compare(agis, oracle_mod, gr, name, mode, first, count, seed=21):
    off, cols, g, nsum, hits = gr
    k, edges = I.PATTERNS[name]
    emb, hit, x, sec = agis.dump_trials(g, agis.Pattern(k, edges), agis.default_opts(mode=mode, seed=seed, anchor=1),
                                        first, count)
    q = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, c_min=CMIN, mode=mode, seed=seed, anchor=True)
    oemb, ohit, ox, osec = q.trials(first, count)
    bad = np.nonzero((emb != oemb).any(axis=1) | (hit != ohit) | (x != ox) | (sec != osec).any(axis=1))[0]
    assert len(bad) == 0, (name, mode, int(bad[0]), emb[bad[0]], oemb[bad[0]], sec[bad[0]], osec[bad[0]])
    return hit


@pytest.mark.gpu
@pytest.mark.parametrize("gname", ["rmat12", "gnp60", "k7"])
@pytest.mark.parametrize("name", MULTI + ["6-clique", "7-cycle"])
def test_anchor_trials_bit_exact(agis, oracle_mod, graphs, gname, name):
    for mode in (0, 1, 2):
        compare(agis, oracle_mod, graphs[gname], name, mode, 2000, 2100)


@pytest.mark.gpu
@pytest.mark.parametrize("policy", [dict(row_prefix_bytes=8), dict(bitmap_min_degree=4, list_entries=64),
                                    dict(row_prefix_bytes=1 << 14)])
def test_anchor_trials_bit_exact_under_memory_policies(agis, oracle_mod, policy):
    """Rows without a prefix take the scan path, hubs the bitmaps: same trials."""
    ctx = agis.Context(0)
    off, cols = I.rmat_graph(12, 16, seed=3)
    g = agis.Graph(ctx, off, cols)
    g.set_memory_policy(**policy)
    g.preprocess(1, CMIN)
    nsum, hits = oracle_mod.graph_stats(off, cols, 1)
    for name in ("4-clique", "house", "5-clique"):
        compare(agis, oracle_mod, (off, cols, g, nsum, hits), name, 1, 0, 2100)


@pytest.mark.gpu
def test_anchor_sums_and_batch(agis, oracle_mod, graphs):
    off, cols, g, nsum, hits = graphs["rmat12"]
    names = ["4-clique", "house", "5-cycle"]
    n = 30000
    for name in names:
        k, edges = I.PATTERNS[name]
        r = agis.estimate(g, agis.Pattern(k, edges), agis.default_opts(seed=4, anchor=1, eps=0.0, max_trials=n))
        s = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, c_min=CMIN, seed=4,
                             anchor=True).sums(0, n)
        assert r["hits"] == s["hits"] and r["sectors"] == s["sectors"]
        assert r["sum_x"] == pytest.approx(s["sum_x"], rel=1e-9, abs=0)
    pats = [agis.Pattern(*I.PATTERNS[nm]) for nm in names]
    opts = [agis.default_opts(seed=30 + i, anchor=1, eps=0.05, chunk_trials=1 << 14, min_trials=1 << 14)
            for i in range(len(names))]
    single = [agis.estimate(g, p, o) for p, o in zip(pats, opts)]
    batch = agis.estimate_batch(g, pats, opts)
    for a, b in zip(single, batch):
        assert a["trials"] == b["trials"] and a["estimate"] == b["estimate"]


@pytest.mark.gpu
def test_anchor_option_checked(agis, graphs):
    g = graphs["k7"][2]
    for bad in (dict(anchor=2), dict(reserved=1)):
        with pytest.raises(agis.AgisError) as e:
            agis.estimate(g, agis.Pattern(*I.PATTERNS["triangle"]), agis.default_opts(**bad))
        assert e.value.status == agis.ERR_ARG
