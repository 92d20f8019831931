"""The incremental versions of f_approx (Sec. 6.2: T[F1] only, + T[I1], + T[F2]) and
the decision threshold beta (Sec. 6.1).  CPU: the oracle with factors dropped is
still unbiased (Thm. 2 needs only positive probabilities on every embedding), is
exact where the dropped factors are constant, and n_(v) of Sec. 4.1 is pinned by
closed forms; the step-1 KL divergences to f_ideal behave as Sec. 6.2 reports.
GPU: sampling with any term mask and any beta is bit-identical to the oracle."""
import math

import numpy as np
import pytest

from paper_2601_01388_b300 import inputs as I
from tests.test_oracle_pins import TINY_GRAPHS, falling

CMIN = 2.0 ** -10
MASKS = (1, 3, 5, 7)     # T[F1] is kept in every version


def masked_cfg(cfg, terms):
    b, f1, ie, f2 = cfg
    return (b, f1 if terms & 1 else 0, ie if terms & 2 else 0, f2 if terms & 4 else 0)


# ---------------------------------------------------------------- n_(v), Sec. 4.1

@pytest.mark.parametrize("gname", sorted(TINY_GRAPHS))
def test_counts_by_first_vertex_sum_to_total(oracle_mod, gname):
    off, cols = TINY_GRAPHS[gname]()
    for name in ("triangle", "4-cycle", "house", "3-path", "tailed-triangle"):
        k, edges = I.PATTERNS[name]
        by = oracle_mod.bruteforce_by_first(off, cols, k, edges)
        assert (by >= 0).all()
        assert int(by.sum()) == oracle_mod.bruteforce_count(off, cols, k, edges)


def test_counts_by_first_vertex_closed_forms(oracle_mod):
    """Triangles: n_(v) = 2 T(v) (two orders of the other corners); a star is matched
    centre first (it has the largest score), so n_(v) = d(v)!/(d(v)-l)!."""
    off, cols = I.gnp_graph(30, 0.3, 5)
    deg = np.diff(off)
    nbr = [set(cols[off[v]:off[v + 1]].tolist()) for v in range(len(deg))]
    tri = [sum(1 for a in nbr[v] for b in nbr[v] if a < b and b in nbr[a]) for v in range(len(deg))]
    by = oracle_mod.bruteforce_by_first(off, cols, *I.PATTERNS["triangle"])
    assert by.tolist() == [2 * t for t in tri]
    for leaves in (2, 3, 4):
        k, edges = I.star(leaves)
        assert oracle_mod.compile_pattern(k, edges)["order"][0] == 0
        by = oracle_mod.bruteforce_by_first(off, cols, k, edges)
        assert by.tolist() == [falling(int(d), leaves) for d in deg]


# ---------------------------------------------------------------- masks keep Thm. 2

@pytest.mark.parametrize("gname", ["gnp10", "mixed", "k6"])
@pytest.mark.parametrize("terms", MASKS)
def test_masked_sampler_unbiased(oracle_mod, gname, terms):
    off, cols = TINY_GRAPHS[gname]()
    for name in ("triangle", "4-cycle", "4-clique", "house", "tailed-triangle", "3-star"):
        k, edges = I.PATTERNS[name]
        truth = oracle_mod.bruteforce_count(off, cols, k, edges)
        q = oracle_mod.Query(off, cols, k, edges, mode=1, terms=terms)
        mean, _, nsucc = q.enumerate()
        assert nsucc == truth
        assert mean == pytest.approx(truth, rel=1e-12, abs=1e-12), (name, terms)


def test_masks_without_first_term_rejected(oracle_mod):
    off, cols = I.gnp_graph(12, 0.4, 1)
    for bad in (2, 4, 6, 8, -1):
        with pytest.raises(ValueError):
            oracle_mod.Query(off, cols, *I.PATTERNS["triangle"], terms=bad)


def test_full_mask_is_the_method(oracle_mod):
    off, cols = I.gnp_graph(40, 0.2, 3)
    k, edges = I.PATTERNS["house"]
    a = oracle_mod.Query(off, cols, k, edges, mode=0, seed=4).trials(0, 3000)
    b = oracle_mod.Query(off, cols, k, edges, mode=0, seed=4, terms=7).trials(0, 3000)
    for u, v in zip(a, b):
        assert (u == v).all()


def test_triangle_first_term_only_closed_form(oracle_mod):
    """With T[F1] alone the triangle's draws are v1 ~ binom(d, 2), v2 ~ d(v2) - 1 over
    N(v1) and v3 uniform over N(v1) & N(v2), so a trajectory returns
    (sum_v binom(d_v, 2) / binom(d_v1, 2)) * (sum_{w in N(v1)} (d_w - 1) / (d_v2 - 1))
    * |N(v1) & N(v2)|."""
    off, cols = I.gnp_graph(35, 0.25, 8)
    deg = np.diff(off).astype(np.int64)
    k, edges = I.PATTERNS["triangle"]
    plan = oracle_mod.compile_pattern(k, edges)
    assert plan["cfg"][0] == (0, 2, 1, 0) and plan["cfg"][1][:2] == (1, 1)
    q = oracle_mod.Query(off, cols, k, edges, mode=1, terms=1)
    emb, hit, x, _ = q.trials(0, 4000)
    top = sum(math.comb(int(d), 2) for d in deg)
    assert hit.any()
    for t in np.nonzero(hit)[0]:
        v1, v2 = int(emb[t, 0]), int(emb[t, 1])
        row = cols[off[v1]:off[v1 + 1]]
        common = len(set(row.tolist()) & set(cols[off[v2]:off[v2 + 1]].tolist()))
        want = (top / math.comb(int(deg[v1]), 2) * float((deg[row] - 1).sum()) / float(deg[v2] - 1)
                * common)
        assert x[t] == pytest.approx(want, rel=1e-12)


# ---------------------------------------------------------------- Sec. 6.2, step-1 KL

def step1_kl(oracle_mod, off, cols, nsum, hits, name, terms):
    """KL(f_ideal(. | ()) || f) for the step-1 distribution f of the given mask
    (terms = 0: f_uniform of the first vertex)."""
    k, edges = I.PATTERNS[name]
    by = oracle_mod.bruteforce_by_first(off, cols, k, edges).astype(np.float64)
    ideal = by / by.sum()
    n = len(off) - 1
    if terms == 0:
        f = np.full(n, 1.0 / n)
    else:
        cfg = masked_cfg(oracle_mod.compile_pattern(k, edges)["cfg"][0], terms)
        deg = np.diff(off)
        w = np.array([oracle_mod.weight(int(deg[v]), int(nsum[v]), int(hits[v]), CMIN, cfg) for v in range(n)])
        f = w / w.sum()
    m = ideal > 0
    assert (f[m] > 0).all()
    return float((ideal[m] * np.log(ideal[m] / f[m])).sum())


def test_step1_kl_divergence_ablation(oracle_mod):
    """On a scale-8 R-MAT graph: f_approx is exact for wedges and stars (n_(v) is
    binom(d, l) up to a constant), every pattern's full f_approx is at least ten times
    closer to f_ideal than f_uniform, and adding terms never moves it away."""
    off, cols = I.rmat_graph(8, 16, seed=5)
    nsum, hits = oracle_mod.graph_stats(off, cols)
    for name in ("3-path", "3-star", "4-star"):
        assert step1_kl(oracle_mod, off, cols, nsum, hits, name, 7) == pytest.approx(0.0, abs=1e-12)
    for name in ("triangle", "4-cycle", "4-clique", "4-path", "tailed-triangle", "diamond"):
        kl = {t: step1_kl(oracle_mod, off, cols, nsum, hits, name, t) for t in (0, 1, 3, 7)}
        assert kl[7] <= kl[3] * (1 + 1e-9) and kl[3] <= kl[1] * (1 + 1e-9), (name, kl)
        assert kl[7] * 10 < kl[0], (name, kl)


# ---------------------------------------------------------------- GPU parity

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
def rmat12(agis, oracle_mod):
    ctx = agis.Context(0)
    off, cols = I.rmat_graph(12, 16, seed=3)
    g = agis.Graph(ctx, off, cols, validate=True)
    g.preprocess(1, CMIN)
    nsum, hits = oracle_mod.graph_stats(off, cols, 1)
    return off, cols, g, nsum, hits


def dump_pair(agis, oracle_mod, graph, name, first, count, **kw):
    off, cols, g, nsum, hits = graph
    k, edges = I.PATTERNS[name]
    emb, hit, x, sec = agis.dump_trials(g, agis.Pattern(k, edges), agis.default_opts(**kw), first, count)
    mode = kw.get("mode", 0)
    q = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, c_min=CMIN, mode=mode,
                         beta=kw.get("beta", 0.8), seed=kw["seed"], terms=kw.get("terms", 0))
    oemb, ohit, ox, osec = q.trials(first, count)
    bad = np.nonzero((emb != oemb).any(axis=1) | (hit != ohit) | (x != ox) | (sec != osec).any(axis=1))[0]
    assert len(bad) == 0, (name, kw, int(bad[0]))
    return hit


@pytest.mark.gpu
@pytest.mark.parametrize("terms", MASKS)
@pytest.mark.parametrize("name", ["triangle", "4-cycle", "4-clique", "house", "5-cycle", "4-path"])
def test_masked_trials_bit_exact(agis, oracle_mod, rmat12, name, terms):
    dump_pair(agis, oracle_mod, rmat12, name, 3000, 2100, mode=1, seed=13, terms=terms)


@pytest.mark.gpu
@pytest.mark.parametrize("beta", [-1.0, 0.25, 0.5, 0.8, 1.0, 1.5])
@pytest.mark.parametrize("name", ["house", "chordal-5-cycle", "tailed-triangle", "5-cycle"])
def test_beta_trials_bit_exact(agis, oracle_mod, rmat12, name, beta):
    dump_pair(agis, oracle_mod, rmat12, name, 0, 2100, mode=0, seed=17, beta=beta)


@pytest.mark.gpu
def test_masked_estimate_sums(agis, oracle_mod, rmat12):
    off, cols, g, nsum, hits = rmat12
    k, edges = I.PATTERNS["4-clique"]
    n = 30000
    for terms in (1, 3):
        r = agis.estimate(g, agis.Pattern(k, edges),
                          agis.default_opts(mode=1, seed=2, terms=terms, eps=0.0, max_trials=n))
        s = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, c_min=CMIN, mode=1, seed=2,
                             terms=terms).sums(0, n)
        assert r["hits"] == s["hits"] and r["sectors"] == s["sectors"]
        assert r["sum_x"] == pytest.approx(s["sum_x"], rel=1e-9, abs=0)


@pytest.mark.gpu
def test_bad_terms_rejected(agis, rmat12):
    g = rmat12[2]
    for bad in (-1, 2, 4, 6, 8):
        with pytest.raises(agis.AgisError) as e:
            agis.estimate(g, agis.Pattern(*I.PATTERNS["triangle"]), agis.default_opts(terms=bad))
        assert e.value.status == agis.ERR_ARG
    with pytest.raises(TypeError):
        agis.default_opts(term=1)
