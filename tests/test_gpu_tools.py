"""The grid autotuner (results must not depend on the grid it picks) and the
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
    best = agis.autotune(g, pats, opts, 1 << 15)
    assert best >= 1
    after = [agis.estimate(g, p, o) for p, o in zip(pats, opts)]
    for a, b in zip(before, after):
        assert a["sum_x"] == b["sum_x"] and a["hits"] == b["hits"] and a["sectors"] == b["sectors"]


def test_random_read_probe_runs(agis):
    import torch
    buf = torch.zeros(1 << 26, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    agis.probe_random_read(buf.data_ptr(), buf.numel(), 1 << 20, 1, 0, sink.data_ptr())
    torch.cuda.synchronize()
    assert int(sink.item()) == 0          # all-zero buffer: the xor never hits the marker
    with pytest.raises(agis.AgisError):
        agis.probe_random_read(buf.data_ptr(), 100, 1, 1, 0, sink.data_ptr())
