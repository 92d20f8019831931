"""The preprocessing cache (agis_graph_save_tables / agis_graph_load_tables).

CPU: a file written from the documented layout with the documented fingerprint is
read back by agis_tables_file_info; missing, truncated and foreign files are IO
errors.  GPU: statistics and tables saved from one handle and loaded into a fresh
handle of the same CSR give identical estimates; a different CSR is refused."""
import os
import struct

import numpy as np
import pytest

from paper_2601_01388_b300 import inputs as I

CMIN = 2.0 ** -10
KEYS = ("trials", "hits", "sectors", "sectors_streamed", "sectors_survey", "converged", "sum_x", "sum_x2",
        "estimate")


def _mix64(x):
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def csr_fingerprint(off, cols):
    """The fingerprint as include/agis.h defines it, in numpy's wrapping uint64."""
    g, s = np.uint64(0x9E3779B97F4A7C15), np.uint64(0xD1B54A32D192ED03)
    with np.errstate(over="ignore"):
        i = np.arange(len(cols), dtype=np.uint64)
        a = _mix64((i * g) ^ np.asarray(cols).astype(np.uint32).astype(np.uint64))
        v = np.arange(len(off), dtype=np.uint64)
        b = _mix64((v * g) ^ np.asarray(off).astype(np.uint64) ^ s)
        return int(a.sum(dtype=np.uint64) + b.sum(dtype=np.uint64))


@pytest.fixture(scope="module")
def agis():
    from paper_2601_01388_b300 import build
    build.build()
    from paper_2601_01388_b300 import agis as A
    return A


def test_file_header_read_back(agis, tmp_path):
    off, cols = I.rmat_graph(6, 8, seed=2)
    nv, nnz = len(off) - 1, len(cols)
    fp = csr_fingerprint(off, cols)
    head = b"AGISTAB1" + struct.pack("<IIqqQQd", 1, 1, nv, nnz, fp, 7, CMIN)
    body = np.zeros(nv, np.uint64).tobytes() + np.zeros(nv, np.uint32).tobytes()
    table = struct.pack("<4iiIQ", 0, 3, 2, 0, 5, 1, 123) + np.arange(nv, dtype=np.uint64).tobytes() * 2
    path = tmp_path / "g.tables"
    path.write_bytes(head + body + table)
    info = agis.tables_file_info(str(path))
    assert info == {"nv": nv, "nnz": nnz, "fingerprint": fp, "n_tables": 1}
    for bad in (b"AGISTAB2" + head[8:], head[:20], b""):
        path.write_bytes(bad)
        with pytest.raises(agis.AgisError) as e:
            agis.tables_file_info(str(path))
        assert e.value.status == agis.ERR_IO
    with pytest.raises(agis.AgisError) as e:
        agis.tables_file_info(str(tmp_path / "missing"))
    assert e.value.status == agis.ERR_IO


@pytest.mark.gpu
def test_save_load_gives_identical_estimates(agis, tmp_path):
    from tests.conftest import has_gpu
    if not has_gpu():
        pytest.skip("needs a CUDA device")
    off, cols = I.rmat_graph(13, 16, seed=3)
    qs = [("4-clique", 0), ("house", 0), ("5-cycle", 1), ("triangle", 2)]
    ctx = agis.Context(0)
    a = agis.Graph(ctx, off, cols)
    assert a.fingerprint() == csr_fingerprint(off, cols)
    a.preprocess(5, CMIN)
    opts = [agis.default_opts(mode=m, seed=40 + i, eps=0.0, max_trials=1 << 16) for i, (_, m) in enumerate(qs)]
    pats = [agis.Pattern(*I.PATTERNS[n]) for n, _ in qs]
    want = [agis.estimate(a, p, o) for p, o in zip(pats, opts)]
    path = str(tmp_path / "rmat13.tables")
    a.save_tables(path)
    info = agis.tables_file_info(path)
    assert info["nv"] == len(off) - 1 and info["nnz"] == len(cols) and info["n_tables"] >= 3
    nsum_a, hits_a = a.stats()
    cfg = (0, 3, 2, 0)
    qa, pa, sa = a.weight_table(cfg)

    # a fresh handle of the same CSR: no preprocessing, tables from the file
    b = agis.Graph(ctx, off, cols)
    b.load_tables(path)
    nsum_b, hits_b = b.stats()
    assert (nsum_a == nsum_b).all() and (hits_a == hits_b).all()
    qb, pb, sb = b.weight_table(cfg)
    assert (qa == qb).all() and (pa == pb).all() and sa == sb
    got = [agis.estimate(b, p, o) for p, o in zip(pats, opts)]
    for w, g_ in zip(want, got):
        for k in KEYS:
            assert w[k] == g_[k], k
    # under a memory policy that allows only partial row prefixes the saved full ones
    # are skipped and rebuilt on demand: the results stay the same
    c = agis.Graph(ctx, off, cols)
    c.set_memory_policy(row_prefix_bytes=1 << 16)
    c.load_tables(path)
    got = [agis.estimate(c, p, o) for p, o in zip(pats, opts)]
    for w, g_ in zip(want, got):
        for k in KEYS:
            assert w[k] == g_[k], k

    # another graph is refused and stays unpreprocessed
    off2, cols2 = I.rmat_graph(13, 16, seed=4)
    d = agis.Graph(ctx, off2, cols2)
    with pytest.raises(agis.AgisError) as e:
        d.load_tables(path)
    assert e.value.status == agis.ERR_GRAPH
    with pytest.raises(agis.AgisError) as e:
        agis.estimate(d, pats[0], opts[0])
    assert e.value.status == agis.ERR_STATE
    for g_ in (a, b, c, d):
        g_.close()
    ctx.close()
