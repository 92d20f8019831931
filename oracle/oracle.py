"""ctypes front end of the CPU oracle (``agis_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is a plain single-threaded restatement of
AGIS's sampler (Alg. 3), its preprocessing (Sec. 4.4), pattern analysis (Alg. 2,
Def. decision function, Def. auxiliary arrays) and Alg. 1.  Only the tests, the
smoke check and the benchmark's CPU-baseline leg may import this module.  It
shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "agis_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MAXK = 8
MODE_AUTO, MODE_APPROX, MODE_UNIFORM = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (no FMA contraction, no fast math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-Wall", "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class Plan(C.Structure):
    _fields_ = [("k", C.c_int32), ("order", C.c_int32 * MAXK), ("nback", C.c_int32 * MAXK),
                ("back", (C.c_int32 * MAXK) * MAXK), ("f1", C.c_int32 * MAXK),
                ("i1", C.c_int32 * MAXK), ("ieff", C.c_int32 * MAXK), ("f2", C.c_int32 * MAXK),
                ("certainty", C.c_double * MAXK), ("aut", C.c_int64)]


class EstimateResult(C.Structure):
    _fields_ = [("trials", C.c_uint64), ("hits", C.c_uint64), ("sectors", C.c_uint64),
                ("sum_x", C.c_double), ("sum_x2", C.c_double), ("mean", C.c_double),
                ("var", C.c_double), ("eps_hat", C.c_double), ("converged", C.c_int32),
                ("sectors_streamed", C.c_uint64), ("sectors_survey", C.c_uint64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        L.orc_philox4x64_10.argtypes = [P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]
        L.orc_draw_below.argtypes = [C.c_uint64] * 5
        L.orc_draw_below.restype = C.c_uint64
        L.orc_plan_compile.argtypes = [C.c_int32, C.c_int32, P(C.c_int32), P(Plan)]
        L.orc_plan_compile.restype = C.c_int
        L.orc_plan_decide.argtypes = [P(Plan), C.c_int32, C.c_double, P(C.c_int32)]
        L.orc_cc_pair.argtypes = [C.c_uint64, C.c_uint64, P(C.c_uint64), P(C.c_uint64)]
        L.orc_graph_stats.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_uint64,
                                      C.c_void_p, C.c_void_p]
        L.orc_graph_stats_range.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_uint64,
                                            C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]
        L.orc_weight.argtypes = [C.c_int64, C.c_uint64, C.c_uint32, C.c_double,
                                 C.c_int32, C.c_int32, C.c_int32, C.c_int32]
        L.orc_weight.restype = C.c_double
        L.orc_quant_shift.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                      C.c_int32, C.c_int32, C.c_int32, C.c_int32]
        L.orc_quant_shift.restype = C.c_int32
        L.orc_quantise.argtypes = [C.c_double, C.c_int64, C.c_int32, C.c_int32, C.c_int32]
        L.orc_quantise.restype = C.c_uint64
        L.orc_weight_table.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                       C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]
        L.orc_weight_table.restype = C.c_int32
        L.orc_query_create.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_double, C.c_int32, C.c_int32, P(C.c_int32),
                                       C.c_int32, C.c_double, C.c_uint64]
        L.orc_query_create.restype = C.c_void_p
        L.orc_query_create_terms.argtypes = L.orc_query_create.argtypes + [C.c_int32]
        L.orc_query_create_terms.restype = C.c_void_p
        L.orc_query_create_ex.argtypes = L.orc_query_create.argtypes + [C.c_int32, C.c_int32, C.c_int32]
        L.orc_query_create_ex.restype = C.c_void_p
        L.orc_orient.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_orient.restype = C.c_int64
        L.orc_bruteforce_by_first.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                              P(C.c_int32), C.c_void_p]
        L.orc_bruteforce_by_first.restype = C.c_int
        L.orc_query_free.argtypes = [C.c_void_p]
        L.orc_query_info.argtypes = [C.c_void_p, P(Plan), P(C.c_int32), P(C.c_int32),
                                     P(C.c_uint64)]
        L.orc_trials.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
        L.orc_sums.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, P(C.c_uint64),
                               P(C.c_double), P(C.c_double), C.c_void_p]
        L.orc_z_of_delta.argtypes = [C.c_double]
        L.orc_z_of_delta.restype = C.c_double
        L.orc_estimate.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_uint64, C.c_uint64,
                                   C.c_uint64, P(EstimateResult)]
        L.orc_bruteforce_count.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_int32,
                                           C.c_int32, P(C.c_int32)]
        L.orc_bruteforce_count.restype = C.c_int64
        for fn in ("orc_exact_triangle", "orc_exact_4cycle", "orc_exact_4clique"):
            getattr(L, fn).argtypes = [C.c_int64, C.c_void_p, C.c_void_p]
            getattr(L, fn).restype = C.c_int64
        L.orc_enumerate.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double), P(C.c_uint64)]
        L.orc_trajectory_prob.argtypes = [C.c_void_p, P(C.c_int32)]
        L.orc_trajectory_prob.restype = C.c_double
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _edges_arr(edges):
    flat = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    return flat, flat.ctypes.data_as(C.POINTER(C.c_int32))


def philox(ctr, key):
    c = (C.c_uint64 * 4)(*[int(x) for x in ctr])
    k = (C.c_uint64 * 2)(*[int(x) for x in key])
    o = (C.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(x) for x in o]


def draw_below(W, a, b, stream, seed):
    return int(lib().orc_draw_below(W, a, b, stream, seed))


def cc_pair(d, r):
    a, b = C.c_uint64(), C.c_uint64()
    lib().orc_cc_pair(d, r, C.byref(a), C.byref(b))
    return a.value, b.value


def compile_pattern(k, edges):
    """Matching order, auxiliary arrays, Certainty and |Aut| (Alg. 2, Def. auxiliary
    arrays, Def. decision function).  Raises ValueError for an invalid pattern."""
    flat, p = _edges_arr(edges)
    plan = Plan()
    rc = lib().orc_plan_compile(k, len(flat) // 2, p, C.byref(plan))
    if rc != 0:
        raise ValueError("invalid pattern")
    k = plan.k
    return {
        "k": k,
        "order": list(plan.order)[:k],
        "back": [list(plan.back[i])[:plan.nback[i]] for i in range(k)],
        "cfg": [(plan.nback[i], plan.f1[i], plan.ieff[i], plan.f2[i]) for i in range(k)],
        "i1": list(plan.i1)[:k],
        "certainty": list(plan.certainty)[:k],
        "aut": plan.aut,
    }


def decide(k, edges, mode=MODE_AUTO, beta=0.8):
    flat, p = _edges_arr(edges)
    plan = Plan()
    if lib().orc_plan_compile(k, len(flat) // 2, p, C.byref(plan)) != 0:
        raise ValueError("invalid pattern")
    ua = (C.c_int32 * MAXK)()
    lib().orc_plan_decide(C.byref(plan), mode, beta, ua)
    return list(ua)[:plan.k]


def graph_stats(off, cols, seed=1):
    off = np.ascontiguousarray(off, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    nv = len(off) - 1
    nsum = np.zeros(nv, dtype=np.uint64)
    hits = np.zeros(nv, dtype=np.uint32)
    lib().orc_graph_stats(nv, _ptr(off), _ptr(cols), seed, _ptr(nsum), _ptr(hits))
    return nsum, hits


def graph_stats_range(off, cols, seed, v0, v1, nsum, hits):
    """Fills nsum[v0:v1], hits[v0:v1] in place (arrays of length nv)."""
    lib().orc_graph_stats_range(len(off) - 1, _ptr(off), _ptr(cols), seed, v0, v1, _ptr(nsum), _ptr(hits))


def weight(d, nsum, hits, c_min, cfg):
    b, f1, ie, f2 = cfg
    return float(lib().orc_weight(d, nsum, hits, c_min, b, f1, ie, f2))


def quant_shift(off, nsum, hits, c_min, cfg):
    off = np.ascontiguousarray(off, dtype=np.int64)
    return int(lib().orc_quant_shift(len(off) - 1, _ptr(off), _ptr(nsum), _ptr(hits), c_min, *cfg))


def quantise(w, d, cfg, shift):
    b, f1, _, _ = cfg
    return int(lib().orc_quantise(w, d, b, f1, shift))


def weight_table(off, nsum, hits, c_min, cfg):
    off = np.ascontiguousarray(off, dtype=np.int64)
    nsum = np.ascontiguousarray(nsum, dtype=np.uint64)
    hits = np.ascontiguousarray(hits, dtype=np.uint32)
    q = np.zeros(len(off) - 1, dtype=np.uint64)
    sh = lib().orc_weight_table(len(off) - 1, _ptr(off), _ptr(nsum), _ptr(hits), c_min, *cfg, _ptr(q))
    return q, int(sh)


def z_of_delta(delta):
    return float(lib().orc_z_of_delta(delta))


def orient(off, cols):
    """Degree-ordered orientation (Sec. 5.4): (off, cols) of the out-rows."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    oo = np.zeros(len(off), dtype=np.int64)
    oc = np.zeros(max(len(cols), 1), dtype=np.int32)
    n = lib().orc_orient(len(off) - 1, _ptr(off), _ptr(cols), _ptr(oo), _ptr(oc))
    return oo, oc[:n].copy()


def bruteforce_by_first(off, cols, k, edges):
    """n_(v) for every vertex v: embeddings whose first matched pattern vertex is v."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    flat, p = _edges_arr(edges)
    out = np.zeros(len(off) - 1, dtype=np.int64)
    if lib().orc_bruteforce_by_first(len(off) - 1, _ptr(off), _ptr(cols), k, len(flat) // 2, p, _ptr(out)) != 0:
        raise ValueError("invalid pattern")
    return out


def bruteforce_count(off, cols, k, edges):
    off = np.ascontiguousarray(off, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    flat, p = _edges_arr(edges)
    return int(lib().orc_bruteforce_count(len(off) - 1, _ptr(off), _ptr(cols), k, len(flat) // 2, p))


def exact_count(off, cols, name):
    """Exact C(G,P) for the triangle, 4-cycle or 4-clique on a larger graph."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    fn = {"triangle": "orc_exact_triangle", "4-cycle": "orc_exact_4cycle", "4-clique": "orc_exact_4clique"}[name]
    return int(getattr(lib(), fn)(len(off) - 1, _ptr(off), _ptr(cols)))


class Query:
    """One pattern query on one graph: keeps the oracle's per-query state."""

    def __init__(self, off, cols, k, edges, *, nsum=None, hits=None, graph_seed=1,
                 c_min=2.0 ** -10, mode=MODE_AUTO, beta=0.8, seed=1, terms=0, oriented=False,
                 anchor=False):
        self.off = np.ascontiguousarray(off, dtype=np.int64)
        self.cols = np.ascontiguousarray(cols, dtype=np.int32)
        if nsum is None or hits is None:
            nsum, hits = graph_stats(self.off, self.cols, graph_seed)
        self.nsum = np.ascontiguousarray(nsum, dtype=np.uint64)
        self.hits = np.ascontiguousarray(hits, dtype=np.uint32)
        self._flat, p = _edges_arr(edges)
        self.k = k
        self._h = lib().orc_query_create_ex(len(self.off) - 1, _ptr(self.off), _ptr(self.cols),
                                            _ptr(self.nsum), _ptr(self.hits), c_min, k,
                                            len(self._flat) // 2, p, mode, beta, seed, terms, int(oriented),
                                            int(anchor))
        if not self._h:
            raise ValueError("invalid pattern or out of memory")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_query_free(h)
            self._h = None

    def info(self):
        plan = Plan()
        ua = (C.c_int32 * MAXK)()
        sh = (C.c_int32 * MAXK)()
        w1 = C.c_uint64()
        lib().orc_query_info(self._h, C.byref(plan), ua, sh, C.byref(w1))
        k = plan.k
        return {"use_approx": list(ua)[:k], "shift": list(sh)[:k], "W1": w1.value,
                "order": list(plan.order)[:k], "aut": plan.aut,
                "cfg": [(plan.nback[i], plan.f1[i], plan.ieff[i], plan.f2[i]) for i in range(k)]}

    def trials(self, first, count):
        emb = np.zeros((count, MAXK), dtype=np.int32)
        hit = np.zeros(count, dtype=np.uint8)
        x = np.zeros(count, dtype=np.float64)
        sec = np.zeros((count, 3), dtype=np.uint64)     # model total, its streamed part, survey count
        lib().orc_trials(self._h, first, count, _ptr(emb), _ptr(hit), _ptr(x), _ptr(sec))
        return emb, hit, x, sec

    def sums(self, first, count):
        h = C.c_uint64()
        sec = (C.c_uint64 * 3)()
        sx, sx2 = C.c_double(), C.c_double()
        lib().orc_sums(self._h, first, count, C.byref(h), C.byref(sx), C.byref(sx2), sec)
        return {"trials": count, "hits": h.value, "sum_x": sx.value, "sum_x2": sx2.value,
                "sectors": sec[0], "sectors_streamed": sec[1], "sectors_survey": sec[2]}

    def estimate(self, eps=0.01, delta=0.05, chunk=1 << 16, min_trials=1 << 16,
                 max_trials=1 << 30):
        r = EstimateResult()
        lib().orc_estimate(self._h, eps, delta, chunk, min_trials, max_trials, C.byref(r))
        return {f: getattr(r, f) for f, _ in EstimateResult._fields_}

    def enumerate(self):
        m, s = C.c_double(), C.c_double()
        n = C.c_uint64()
        lib().orc_enumerate(self._h, C.byref(m), C.byref(s), C.byref(n))
        return m.value, s.value, n.value

    def trajectory_prob(self, tau):
        t = (C.c_int32 * MAXK)(*([int(v) for v in tau] + [-1] * (MAXK - len(tau))))
        return float(lib().orc_trajectory_prob(self._h, t))
