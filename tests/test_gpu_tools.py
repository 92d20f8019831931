"""The launch autotuner (results must not depend on the grid or the tiles per item
it picks) and the
random-access read probe."""
import numpy as np
import pytest

from paper_2601_01388_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def agis():
    from tests.conftest import has_gpu
    if not has_gpu():
        pytest.skip("needs a CUDA device")
    from paper_2601_01388_b300 import build
    build.build()
    from paper_2601_01388_b300 import agis as A
    return A


def test_autotune_keeps_results(agis):
    ctx = agis.Context(0)
    off, cols = I.rmat_graph(13, 16, seed=6)
    g = agis.Graph(ctx, off, cols)
    g.preprocess(1, 2.0 ** -10)
    pats = [agis.Pattern(*I.PATTERNS[n]) for n in ("4-clique", "house", "5-cycle")]
    opts = [agis.default_opts(mode=m, seed=3 + m, eps=0.0, max_trials=50000) for m in range(3)]
    before = [agis.estimate(g, p, o) for p, o in zip(pats, opts)]
    best, span = agis.autotune(g, pats, opts, 1 << 15)
    assert best >= 1 and span in (1, 2, 4)
    after = [agis.estimate(g, p, o) for p, o in zip(pats, opts)]
    batched = agis.estimate_batch(g, pats, opts)
    for a, b, c in zip(before, after, batched):
        assert a["sum_x"] == b["sum_x"] == c["sum_x"] and a["hits"] == b["hits"] == c["hits"]
        assert a["sectors"] == b["sectors"] == c["sectors"]


def test_random_read_probe_runs(agis):
    import torch
    buf = torch.zeros(1 << 26, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    agis.probe_random_read(buf.data_ptr(), buf.numel(), 1 << 20, 1, 0, sink.data_ptr())
    torch.cuda.synchronize()
    assert int(sink.item()) == 0          # all-zero buffer: the xor never hits the marker
    with pytest.raises(agis.AgisError):
        agis.probe_random_read(buf.data_ptr(), 100, 1, 1, 0, sink.data_ptr())


def test_multi_tile_items_keep_tile_sums(agis):
    """2^21 trials in one epoch run as items of several tiles; summing the per-tile
    outputs of single-tile items (sample_device) in order gives the same totals."""
    import torch
    ctx = agis.Context(0)
    off, cols = I.rmat_graph(13, 16, seed=6)
    g = agis.Graph(ctx, off, cols)
    g.preprocess(1, 2.0 ** -10)
    p = agis.Pattern(*I.PATTERNS["house"])
    n = 1 << 21
    for mode in (0, 2):
        o = agis.default_opts(mode=mode, seed=12, eps=0.0, max_trials=n, chunk_trials=n)
        r = agis.estimate(g, p, o)
        ntiles = n // agis.TILE
        out = torch.zeros(ntiles * agis.TILE_WORDS, dtype=torch.int64, device="cuda")
        agis.sample_device(g, p, o, 0, ntiles, out.data_ptr())
        torch.cuda.synchronize()
        ts = agis.tile_sums(out.cpu().numpy().view(np.uint64))
        acc = 0.0
        for v in ts["sum_x"]:
            acc += float(v)
        assert r["trials"] == n and r["hits"] == int(ts["hits"].sum()) and r["sectors"] == int(ts["sectors"].sum())
        assert r["sectors_streamed"] == int(ts["streamed"].sum()) and r["sectors_survey"] == int(ts["survey"].sum())
        assert r["sum_x"] == acc


def test_scatter_epochs_equal_tile_epochs(agis):
    """An epoch with no more tiles than the grid has CTAs runs in scatter mode (every
    warp takes single trials, a second kernel reduces each tile); its tile sums must
    be the main kernel's bits: an estimate of 2^13 trials (32 tiles, one scatter
    epoch) against agis_sample_device over the same trials (main kernel, one tile
    per item), for several patterns and modes, plus the batched form."""
    import torch
    ctx = agis.Context(0)
    off, cols = I.rmat_graph(13, 16, seed=6)
    g = agis.Graph(ctx, off, cols)
    g.preprocess(1, 2.0 ** -10)
    n = 1 << 13
    pats, opts, singles = [], [], []
    for name, mode in (("4-clique", 0), ("house", 0), ("5-cycle", 1), ("triangle", 2)):
        p = agis.Pattern(*I.PATTERNS[name])
        o = agis.default_opts(mode=mode, seed=21, eps=0.0, max_trials=n, chunk_trials=n)
        r = agis.estimate(g, p, o)
        assert r["launches"] == 1
        ntiles = n // agis.TILE
        out = torch.zeros(ntiles * agis.TILE_WORDS, dtype=torch.int64, device="cuda")
        agis.sample_device(g, p, o, 0, ntiles, out.data_ptr())
        torch.cuda.synchronize()
        ts = agis.tile_sums(out.cpu().numpy().view(np.uint64))
        acc = acc2 = 0.0
        for v, v2 in zip(ts["sum_x"], ts["sum_x2"]):
            acc += float(v)
            acc2 += float(v2)
        assert r["sum_x"] == acc and r["sum_x2"] == acc2, name
        assert r["hits"] == int(ts["hits"].sum()) and r["sectors"] == int(ts["sectors"].sum()), name
        assert r["sectors_streamed"] == int(ts["streamed"].sum()), name
        assert r["sectors_survey"] == int(ts["survey"].sum()), name
        pats.append(p)
        opts.append(o)
        singles.append(r)
    for a, b in zip(singles, agis.estimate_batch(g, pats, opts)):
        for key in ("trials", "hits", "sectors", "sum_x", "sum_x2"):
            assert a[key] == b[key], key
    g.close()
    ctx.close()


def _device_tile_sums(agis, g, p, o, ntiles):
    """The main kernel's tile sums of trials [0, ntiles * TILE), folded in tile order
    as the Alg. 1 loop folds them."""
    import torch
    out = torch.zeros(ntiles * agis.TILE_WORDS, dtype=torch.int64, device="cuda")
    agis.sample_device(g, p, o, 0, ntiles, out.data_ptr())
    torch.cuda.synchronize()
    ts = agis.tile_sums(out.cpu().numpy().view(np.uint64))
    acc = acc2 = 0.0
    for v, v2 in zip(ts["sum_x"], ts["sum_x2"]):
        acc += float(v)
        acc2 += float(v2)
    return {"sum_x": acc, "sum_x2": acc2, "hits": int(ts["hits"].sum()), "sectors": int(ts["sectors"].sum()),
            "sectors_streamed": int(ts["streamed"].sum()), "sectors_survey": int(ts["survey"].sum())}


def test_head_and_tail_epochs_equal_tile_epochs(agis, oracle_mod):
    """An epoch of more tiles than the grid has CTAs runs its last grid-full of tiles
    on the scatter kernel beside the main kernel; no tile's sums may depend on which
    of the two ran it.  One epoch of 1172 tiles (the grid has 740 CTAs on 148 SMs)
    against agis_sample_device over the same tiles, for several patterns and modes; a
    batch of three 400-tile queries, whose tail covers the second query's end and all
    of the third; and a ragged 300,000-trial epoch against the oracle's sums."""
    ctx = agis.Context(0)
    off, cols = I.rmat_graph(13, 16, seed=6)
    g = agis.Graph(ctx, off, cols)
    g.preprocess(1, 2.0 ** -10)
    T = agis.TILE
    keys = ("hits", "sectors", "sectors_streamed", "sectors_survey", "sum_x", "sum_x2")
    for name, mode in (("4-clique", 0), ("house", 1), ("5-cycle", 2)):
        p = agis.Pattern(*I.PATTERNS[name])
        o = agis.default_opts(mode=mode, seed=23, eps=0.0, max_trials=1172 * T, chunk_trials=1172 * T)
        r = agis.estimate(g, p, o)
        assert r["launches"] == 1 and r["trials"] == 1172 * T
        d = _device_tile_sums(agis, g, p, o, 1172)
        for key in keys:
            assert r[key] == d[key], (name, key)
        rb = agis.estimate_batch(g, [p], [o])[0]
        for key in keys:
            assert rb[key] == d[key], (name, key)
    pats = [agis.Pattern(*I.PATTERNS[n]) for n in ("4-clique", "house", "5-cycle")]
    opts = [agis.default_opts(mode=m, seed=30 + m, eps=0.0, max_trials=400 * T, chunk_trials=400 * T)
            for m in range(3)]
    batch = agis.estimate_batch(g, pats, opts)
    for p, o, b in zip(pats, opts, batch):
        d = _device_tile_sums(agis, g, p, o, 400)
        single = agis.estimate(g, p, o)
        for key in keys:
            assert b[key] == d[key] == single[key], key
    # ragged last tile, against the oracle
    nsum, hits = oracle_mod.graph_stats(off, cols, 1)
    k, edges = I.PATTERNS["house"]
    n = 300000
    o = agis.default_opts(mode=0, seed=41, eps=0.0, max_trials=n, chunk_trials=n // 1024 * 1024)
    r = agis.estimate(g, agis.Pattern(k, edges), o)
    s = oracle_mod.Query(off, cols, k, edges, nsum=nsum, hits=hits, mode=0, seed=41).sums(0, n)
    assert r["trials"] == n
    for key in keys[:4]:
        assert r[key] == s[key], key
    assert r["sum_x"] == pytest.approx(s["sum_x"], rel=1e-9, abs=0)
    assert r["sum_x2"] == pytest.approx(s["sum_x2"], rel=1e-9, abs=0)
    g.close()
    ctx.close()


def test_l2_window_keeps_results(agis):
    """The persisting-L2 window over the hub bitmaps is a cache hint: estimates (plain,
    batched, with and without epoch tails) and sampler tile sums are the same bits
    with the default window, a small one and none."""
    ctx = agis.Context(0)
    off, cols = I.rmat_graph(13, 16, seed=6)
    g = agis.Graph(ctx, off, cols)
    g.set_memory_policy(bitmap_min_degree=64)        # hub bitmaps on this small graph
    g.preprocess(1, 2.0 ** -10)
    pats = [agis.Pattern(*I.PATTERNS[n]) for n in ("4-clique", "house", "5-cycle")]
    T = agis.TILE
    opts = [agis.default_opts(mode=m, seed=40 + m, eps=0.0, max_trials=1000 * T, chunk_trials=1000 * T)
            for m in range(3)]
    keys = ("hits", "sectors", "sectors_streamed", "sectors_survey", "sum_x", "sum_x2")
    runs = []
    for nbytes in (48 << 20, 1 << 20, 0):
        g.set_l2_window(nbytes)
        single = [agis.estimate(g, p, o) for p, o in zip(pats, opts)]
        batch = agis.estimate_batch(g, pats, opts)
        sums = [_device_tile_sums(agis, g, p, o, 64) for p, o in zip(pats, opts)]
        runs.append((single, batch, sums))
    for single, batch, sums in runs[1:]:
        for a, b in zip(runs[0][0] + runs[0][1] + runs[0][2], single + batch + sums):
            for key in keys:
                assert a[key] == b[key], key
    g.close()
    ctx.close()
