"""Batching and serving invariance (a result is the same alone, batched and served),
memory admission of the server, and the device R-MAT generator."""
import time

import numpy as np
import pytest

from paper_2601_01388_b300 import inputs as I

pytestmark = pytest.mark.gpu
CMIN = 2.0 ** -10


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
def setup(agis):
    ctx = agis.Context(0)
    off, cols = I.rmat_graph(12, 16, seed=3)
    g = agis.Graph(ctx, off, cols)
    g.preprocess(1, CMIN)
    return ctx, g


def wait_all(srv, tickets, timeout=300):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets):
        assert time.time() - t0 < timeout, "server did not finish"
        for t in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
        time.sleep(0.001)
    return [done[t] for t in tickets]


def queries(agis, n=12):
    rng = np.random.Generator(np.random.Philox(key=[5, 0]))
    out = []
    for i in range(n):
        k, e = I.random_connected_pattern(rng, 3, 6, 0.3)
        o = agis.default_opts(mode=i % 3, seed=50 + i, eps=float(0.02 + 0.03 * rng.random()), delta=0.05,
                              chunk_trials=4096, min_trials=4096, max_trials=1 << 21)
        out.append((agis.Pattern(k, e), o))
    return out


KEYS = ("trials", "hits", "sectors", "sectors_streamed", "sectors_survey", "converged", "sum_x", "sum_x2", "estimate")


def test_served_equals_alone_and_batched(agis, setup):
    ctx, g = setup
    qs = queries(agis)
    alone = [agis.estimate(g, p, o) for p, o in qs]
    batched = agis.estimate_batch(g, [p for p, _ in qs], [o for _, o in qs])
    srv = agis.Server(g, 8 << 30, 5)
    tickets = []
    for j, (p, o) in enumerate(qs):             # staggered arrivals while others run
        tickets.append(srv.submit(p, o))
        if j % 3 == 2:
            time.sleep(0.002)
    served = wait_all(srv, tickets)
    st = srv.stats()
    srv.close()
    for a, b, c in zip(alone, batched, served):
        for k in KEYS:
            assert a[k] == b[k] == c[k], k
    assert st["completed"] == len(qs)
    assert 1 <= st["peak_slots"] <= 5


def test_continuous_admission_overlaps(agis, setup):
    """A query that arrives while another is on the GPU joins a later epoch while the
    first is still running (their epoch ranges overlap), finishes first, and both
    results equal what each gives alone."""
    ctx, g = setup
    long_q = (agis.Pattern(*I.PATTERNS["4-clique"]), agis.default_opts(mode=0, seed=71, eps=0.0, max_trials=1 << 23))
    short_q = (agis.Pattern(*I.PATTERNS["triangle"]),
               agis.default_opts(mode=0, seed=72, eps=0.0, max_trials=1 << 16))
    alone = [agis.estimate(g, p, o) for p, o in (long_q, short_q)]
    srv = agis.Server(g, 8 << 30, 4)
    tl = srv.submit(*long_q)
    t0 = time.time()
    while srv.stats()["epochs"] < 2:             # the long query is on the GPU
        assert time.time() - t0 < 60
        time.sleep(0.0005)
    ts = srv.submit(*short_q)
    rl, rs = wait_all(srv, [tl, ts])
    st = srv.stats()
    srv.close()
    assert rl["admit_epoch"] == 0
    assert rl["admit_epoch"] < rs["admit_epoch"] < rl["finish_epoch"]     # admitted mid-flight
    assert rs["finish_epoch"] < rl["finish_epoch"]
    for a, c in zip(alone, (rl, rs)):
        for k in KEYS:
            assert a[k] == c[k], k
    assert st["epochs"] >= rl["finish_epoch"] + 1
    # device time (events) within the host's busy span, up to the two clocks' skew
    assert 0.0 < st["gpu_busy_s"] <= st["busy_span_s"] * 1.001 + 1e-4


def test_admission_by_memory(agis, setup):
    ctx, g = setup
    g.drop_tables()
    nv, nnz = g.info()["nv"], g.info()["nnz"]
    qs = queries(agis, 6)
    alone = [agis.estimate(g, p, o) for p, o in qs]
    g.drop_tables()
    # room for the largest single query's tables (q per vertex, a vertex prefix for
    # step 1, a row prefix per single-backward f_approx step), not for all of them;
    # a later step whose configuration has no F1, I1 or F2 term weighs its candidates
    # equally and reads no table
    def need(p, o):
        info = p.info()
        use = p.decide(o.mode, o.beta)
        cfgs = {}
        for i in range(info["k"]):
            if use[i] and (i == 0 or any(info["cfg"][i][1:])):
                c = cfgs.setdefault(info["cfg"][i], [False, False])
                c[0] |= i == 0
                c[1] |= i > 0 and len(info["back"][i]) == 1
        return sum(8 * nv + (8 * nv if a else 0) + (8 * nnz if b else 0) for a, b in cfgs.values())
    budget = max(need(p, o) for p, o in qs)
    assert budget < sum(need(p, o) for p, o in qs)
    srv = agis.Server(g, budget, 6)
    served = wait_all(srv, [srv.submit(p, o) for p, o in qs])
    srv.close()
    for a, c in zip(alone, served):
        assert a["trials"] == c["trials"] and a["sum_x"] == c["sum_x"]


def test_query_that_cannot_fit_fails_cleanly(agis, setup):
    ctx, g = setup
    g.drop_tables()
    srv = agis.Server(g, 1024, 2)
    p = agis.Pattern(*I.PATTERNS["4-clique"])
    t = srv.submit(p, agis.default_opts(mode=1, max_trials=1 << 16))
    t0 = time.time()
    while True:
        try:
            r = srv.poll(t)
        except agis.AgisError as e:
            assert e.status == agis.ERR_NOMEM
            break
        assert r is None and time.time() - t0 < 60
        time.sleep(0.001)
    srv.close()


def test_device_rmat_is_a_valid_graph(agis):
    ctx = agis.Context(0)
    g = agis.Graph.rmat(ctx, 14, 16, 0.57, 0.19, 0.19, seed=1)
    g.validate()
    info = g.info()
    off, cols = g.csr()
    assert info["nv"] == 1 << 14 and len(cols) == info["nnz"] == off[-1]
    deg = np.diff(off)
    assert deg.max() == info["max_degree"]
    # same shape as the host generator's graph (different random streams)
    hoff, hcols = I.rmat_graph(14, 16, seed=1)
    assert abs(len(cols) - len(hcols)) / len(hcols) < 0.03
    assert 0.5 < deg.max() / np.diff(hoff).max() < 2.0
    g2 = agis.Graph.rmat(ctx, 14, 16, 0.57, 0.19, 0.19, seed=1)
    o2, c2 = g2.csr()
    assert (o2 == off).all() and (c2 == cols).all()          # reproducible
    g.preprocess(1, CMIN)
    r = agis.estimate(g, agis.Pattern(*I.PATTERNS["triangle"]), agis.default_opts(eps=0.0, max_trials=1 << 16))
    assert r["hits"] > 0


def test_device_chung_lu_is_a_valid_power_law_graph(agis):
    ctx = agis.Context(0)
    n = 200000
    g = agis.Graph.chung_lu(ctx, n, 2.1, 32.0, seed=3)
    g.validate()
    info = g.info()
    off, cols = g.csr()
    deg = np.diff(off)
    assert info["nv"] == n and len(cols) == info["nnz"]
    mean = deg.mean()
    assert 20.0 < mean < 34.0                      # duplicates and loops removed from n*32/2 draws
    assert deg.max() > 20 * mean                   # heavy tail
    assert deg.max() <= 2.0 * np.sqrt(32.0 * n)   # capped near sqrt(sum of expected degrees)
    g2 = agis.Graph.chung_lu(ctx, n, 2.1, 32.0, seed=3)
    o2, c2 = g2.csr()
    assert (o2 == off).all() and (c2 == cols).all()


def test_two_servers_on_two_graphs_concurrently(agis, setup):
    """Two servers (two scheduler threads, each building and replaying its own CUDA
    graph) on two resident graphs at once, with anchor-draw and term-mask queries
    in the mix: every result equals the same query run alone."""
    ctx, g = setup
    off2, cols2 = I.rmat_graph(11, 16, seed=9)
    g2 = agis.Graph(ctx, off2, cols2)
    g2.preprocess(1, CMIN)
    qs = queries(agis, 8)
    extra = agis.default_opts(seed=77, anchor=1, terms=3, eps=0.03, chunk_trials=4096, min_trials=4096,
                              max_trials=1 << 21)
    qs.append((agis.Pattern(*I.PATTERNS["house"]), extra))
    alone1 = [agis.estimate(g, p, o) for p, o in qs]
    alone2 = [agis.estimate(g2, p, o) for p, o in qs]
    s1 = agis.Server(g, 4 << 30, 4)
    s2 = agis.Server(g2, 4 << 30, 4)
    try:
        t1, t2 = [], []
        for p, o in qs:
            t1.append(s1.submit(p, o))
            t2.append(s2.submit(p, o))
        r1 = wait_all(s1, t1)
        r2 = wait_all(s2, t2)
    finally:
        s1.close()
        s2.close()
    for a, b in zip(alone1, r1):
        for k in KEYS:
            assert a[k] == b[k], k
    for a, b in zip(alone2, r2):
        for k in KEYS:
            assert a[k] == b[k], k
    g2.close()
