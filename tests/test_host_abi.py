"""CPU-side checks of the C ABI: the library builds and loads without a GPU, it
exports every symbol include/agis.h declares, and its host-side pattern analysis
agrees with the oracle's.  No device compute is called here."""
import os
import re

import numpy as np
import pytest

from paper_2601_01388_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def agis():
    from paper_2601_01388_b300 import build
    build.build()
    from paper_2601_01388_b300 import agis as A
    return A


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(agis_[a-z_0-9]+)\s*\(", text, re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(agis):
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(agis._lib, n), n


def test_binding_covers_header(agis):
    assert set(declared_functions()) == set(agis.EXPORTS)


def test_status_strings(agis):
    for s in range(-8, 1):
        assert agis.status_str(s) not in ("", "unknown status")


def test_default_opts(agis):
    o = agis.default_opts()
    assert (o.eps, o.delta, o.beta, o.mode) == (0.1, 0.01, 0.8, 0)
    assert o.chunk_trials % 1024 == 0 and 1024 % agis.TILE == 0


def test_z_matches_scipy(agis):
    import scipy.stats
    for d in (0.5, 0.05, 0.01, 1e-4, 1e-9):
        assert agis.z_of_delta(d) == pytest.approx(scipy.stats.norm.isf(d / 2), rel=1e-12)


def test_pattern_analysis_matches_oracle(agis, oracle_mod):
    rng = np.random.Generator(np.random.Philox(key=[3, 0]))
    pats = list(I.PATTERNS.values()) + [I.random_connected_pattern(rng, 2, 8) for _ in range(200)]
    for k, e in pats:
        a = agis.Pattern(k, e)
        info = a.info()
        o = oracle_mod.compile_pattern(k, e)
        assert info["order"] == o["order"]
        assert info["cfg"] == o["cfg"]
        assert info["back"] == o["back"]
        assert info["aut"] == o["aut"]
        assert info["certainty"] == o["certainty"]
        for mode in (0, 1, 2):
            for beta in (0.5, 0.8, 1.0):
                assert a.decide(mode, beta) == oracle_mod.decide(k, e, mode, beta)


@pytest.mark.parametrize("bad", [(1, [(0, 0)]), (3, [(0, 1)]), (3, [(0, 1), (0, 1)]),
                                 (9, [(i, i + 1) for i in range(8)]), (3, [(0, 3)]),
                                 (4, [(0, 1), (2, 3), (0, 2)][:2])])
def test_invalid_patterns_rejected(agis, bad):
    with pytest.raises(agis.AgisError) as e:
        agis.Pattern(*bad)
    assert e.value.status == agis.ERR_PATTERN


def test_no_device_gives_cuda_error(agis):
    from tests.conftest import has_gpu
    if has_gpu():
        pytest.skip("a device is present")
    with pytest.raises(agis.AgisError) as e:
        agis.Context(0)
    assert e.value.status == agis.ERR_CUDA


def test_layout_constants_match_header(agis):
    """The binding's tile layout and result struct follow include/agis.h."""
    import ctypes
    text = open(os.path.join(ROOT, "include", "agis.h")).read()
    assert int(re.search(r"#define AGIS_TILE_WORDS (\d+)", text).group(1)) == agis.TILE_WORDS
    body = re.search(r"typedef struct \{([^}]*)\} agis_result;", text).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        words = decl.split()
        if words:
            fields += [n.strip() for n in " ".join(words[1:]).split(",")]
    assert fields == [f for f, _ in agis.Result._fields_]
    assert ctypes.sizeof(agis.Result) == 120     # 15 eight-byte slots, no padding


def test_null_handles_are_argument_errors(agis):
    """Every call named here checks its handles before touching the device, so a NULL
    handle is ARG (include/agis.h) on any host, with or without a GPU."""
    import ctypes
    lib = agis._lib
    res = agis.Result()
    opts = agis.default_opts()
    out = ctypes.c_void_p()
    fp = ctypes.c_uint64()
    calls = [
        ("agis_destroy", (None,)),
        ("agis_graph_free", (None,)),
        ("agis_graph_preprocess", (None, 1, 2.0 ** -10)),
        ("agis_graph_set_memory_policy", (None, 0, 0, 0, 0)),
        ("agis_graph_set_l2_window", (None, 1 << 20)),
        ("agis_graph_drop_tables", (None,)),
        ("agis_graph_orient", (None, ctypes.byref(out))),
        ("agis_graph_is_oriented", (None,)),
        ("agis_graph_fingerprint", (None, ctypes.byref(fp))),
        ("agis_estimate", (None, None, ctypes.byref(opts), ctypes.byref(res))),
        ("agis_server_destroy", (None,)),
    ]
    for name, args in calls:
        assert getattr(lib, name)(*args) == agis.ERR_ARG, name
