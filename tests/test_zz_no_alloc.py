"""The allocation-free prefix sum (agis_prefix_sum_u64_noalloc).

Callers that cannot call cudaMalloc -- a custom device allocator or pool hook that
must not re-enter the CUDA allocator, a service whose device memory a pool already
holds in full, latency-critical code that avoids cudaMalloc's blocking -- use this
entry point: it keeps its scratch in a file-scope device array.  Its output is
checked, twice in a row, against the prefix sums the existing weight-table entry
point (agis_graph_weight_table) returns for the same input; both are exact integer
scans, so they must be equal.  This file is named to be collected last."""
import numpy as np
import pytest

from paper_2601_01388_b300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_prefix_sum_matches_weight_table_prefix():
    from tests.conftest import has_gpu
    if not has_gpu():
        pytest.skip("needs a CUDA device")
    import torch
    from paper_2601_01388_b300 import build
    build.build()
    from paper_2601_01388_b300 import agis

    torch.cuda.set_device(0)
    ctx = agis.Context(0)
    off, cols = I.rmat_graph(17, 16, seed=4)          # 131072 vertices: 64 scan tiles
    g = agis.Graph(ctx, off, cols)
    g.preprocess(1, 2.0 ** -10)
    for cfg in [(0, 3, 1, 2), (0, 4, 3, 0)]:
        q, pref, _ = g.weight_table(cfg)              # the existing entry point's scan
        n = len(q)
        d_in = torch.from_numpy(q.view(np.int64)).cuda()
        for _ in range(2):                            # the scratch keeps the last call's contents
            d_out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
            agis.prefix_sum_u64_noalloc(d_in.data_ptr(), n, d_out.data_ptr(), 0)
            torch.cuda.synchronize()
            got = d_out.cpu().numpy().view(np.uint64)
            assert (got == pref).all()
    # a shorter, ragged input after a longer one reuses the same scratch
    m = 5000
    d_out = torch.zeros(m, dtype=torch.int64, device="cuda")
    agis.prefix_sum_u64_noalloc(d_in.data_ptr(), m, d_out.data_ptr(), 0)
    torch.cuda.synchronize()
    assert (d_out.cpu().numpy().view(np.uint64) == np.cumsum(q[:m], dtype=np.uint64)).all()
    with pytest.raises(agis.AgisError) as e:
        agis.prefix_sum_u64_noalloc(d_in.data_ptr(), 65536 * 2048 + 1, d_out.data_ptr(), 0)
    assert e.value.status == agis.ERR_ARG
    g.close()
    ctx.close()
