"""Thin Python binding of libagis.so (the C ABI in include/agis.h).

Functions carry the C names without the ``agis_`` prefix and only marshal
arguments: every step of the counting path runs in the library's CUDA kernels.
If the shared library is missing this module raises ImportError -- there is no
fallback implementation.  PyTorch is only used, where a caller passes tensors,
for device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libagis.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libagis.so is not built ({LIB_PATH}); run paper_2601_01388_b300/build.py")

_lib = C.CDLL(LIB_PATH)

OK, ERR_ARG, ERR_NOMEM, ERR_CUDA, ERR_GRAPH, ERR_PATTERN, ERR_TIMEOUT, ERR_BUSY, ERR_STATE, ERR_IO = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9
MODE_AUTO, MODE_APPROX, MODE_UNIFORM = 0, 1, 2

EXPORTS = [
    "agis_status_str", "agis_default_opts", "agis_create", "agis_destroy", "agis_graph_load_csr",
    "agis_graph_preprocess", "agis_graph_info", "agis_graph_stats_copy", "agis_graph_weight_table",
    "agis_graph_row_prefix", "agis_graph_orient", "agis_graph_is_oriented", "agis_graph_set_memory_policy", "agis_graph_set_l2_window", "agis_graph_validate", "agis_graph_copy_csr", "agis_graph_drop_tables", "agis_graph_free", "agis_graph_generate_rmat", "agis_graph_generate_chunglu",
    "agis_pattern_create", "agis_pattern_info", "agis_pattern_decide", "agis_pattern_free",
    "agis_estimate", "agis_estimate_batch", "agis_autotune", "agis_dump_trials", "agis_sample_device",
    "agis_prepare", "agis_tile_trials", "agis_z_of_delta", "agis_kernel_launches", "agis_prefix_sum_u64_noalloc", "agis_probe_random_read", "agis_step_timers", "agis_server_create", "agis_server_submit", "agis_server_poll",
    "agis_server_stats", "agis_server_destroy", "agis_graph_save_tables", "agis_graph_load_tables",
    "agis_graph_fingerprint", "agis_tables_file_info",
]


class Opts(C.Structure):
    _fields_ = [("eps", C.c_double), ("delta", C.c_double), ("beta", C.c_double),
                ("mode", C.c_int32), ("terms", C.c_int32), ("seed", C.c_uint64),
                ("min_trials", C.c_uint64), ("max_trials", C.c_uint64),
                ("chunk_trials", C.c_uint64), ("anchor", C.c_int32), ("reserved", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("estimate", C.c_double), ("subgraphs", C.c_double), ("mean", C.c_double),
                ("var", C.c_double), ("eps_hat", C.c_double), ("sum_x", C.c_double),
                ("sum_x2", C.c_double), ("trials", C.c_uint64), ("hits", C.c_uint64),
                ("sectors", C.c_uint64), ("converged", C.c_int32), ("launches", C.c_int32),
                ("t_prep_s", C.c_double), ("t_sample_s", C.c_double),
                ("sectors_streamed", C.c_uint64), ("sectors_survey", C.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


P = C.POINTER
VP = C.c_void_p
_sig = {
    "agis_status_str": ([C.c_int], C.c_char_p),
    "agis_default_opts": ([P(Opts)], None),
    "agis_create": ([C.c_int, VP, P(VP)], C.c_int),
    "agis_destroy": ([VP], C.c_int),
    "agis_graph_load_csr": ([VP, VP, C.c_int, VP, C.c_int64, C.c_int64, C.c_int, C.c_int, P(VP)], C.c_int),
    "agis_graph_preprocess": ([VP, C.c_uint64, C.c_double], C.c_int),
    "agis_graph_info": ([VP, P(C.c_int64), P(C.c_int64), P(C.c_int64), P(C.c_uint64)], C.c_int),
    "agis_graph_stats_copy": ([VP, VP, VP], C.c_int),
    "agis_graph_weight_table": ([VP, P(C.c_int32), VP, VP, P(C.c_int32)], C.c_int),
    "agis_graph_row_prefix": ([VP, P(C.c_int32), VP], C.c_int),
    "agis_graph_set_memory_policy": ([VP, C.c_uint64, C.c_uint64, C.c_int64, C.c_uint32], C.c_int),
    "agis_graph_set_l2_window": ([VP, C.c_uint64], C.c_int),
    "agis_graph_validate": ([VP], C.c_int),
    "agis_graph_orient": ([VP, P(VP)], C.c_int),
    "agis_graph_is_oriented": ([VP], C.c_int),
    "agis_graph_copy_csr": ([VP, VP, VP], C.c_int),
    "agis_graph_drop_tables": ([VP], C.c_int),
    "agis_graph_free": ([VP], C.c_int),
    "agis_graph_generate_rmat": ([VP, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_uint64, P(VP)], C.c_int),
    "agis_graph_generate_chunglu": ([VP, C.c_int64, C.c_double, C.c_double, C.c_uint64, P(VP)], C.c_int),
    "agis_pattern_create": ([C.c_int, C.c_int, P(C.c_int32), P(VP)], C.c_int),
    "agis_pattern_info": ([VP, P(C.c_int32), P(C.c_int32), P(C.c_int32), P(C.c_double), P(C.c_uint8), P(C.c_uint64)], C.c_int),
    "agis_pattern_decide": ([VP, C.c_int32, C.c_double, P(C.c_uint8)], C.c_int),
    "agis_pattern_free": ([VP], C.c_int),
    "agis_estimate": ([VP, VP, P(Opts), P(Result)], C.c_int),
    "agis_estimate_batch": ([VP, C.c_int, P(VP), P(Opts), P(Result)], C.c_int),
    "agis_dump_trials": ([VP, VP, P(Opts), C.c_uint64, C.c_uint64, VP, VP, VP, VP], C.c_int),
    "agis_sample_device": ([VP, VP, P(Opts), C.c_uint64, C.c_uint64, VP], C.c_int),
    "agis_prepare": ([VP, VP, P(Opts)], C.c_int),
    "agis_autotune": ([VP, C.c_int, P(VP), P(Opts), C.c_uint64, P(C.c_int32), P(C.c_int32)], C.c_int),
    "agis_z_of_delta": ([C.c_double], C.c_double),
    "agis_tile_trials": ([], C.c_int),
    "agis_kernel_launches": ([], C.c_uint64),
    "agis_prefix_sum_u64_noalloc": ([VP, C.c_int64, VP, VP], C.c_int),
    "agis_probe_random_read": ([VP, C.c_uint64, C.c_uint64, C.c_uint64, VP, VP], C.c_int),
    "agis_step_timers": ([VP, C.c_int], C.c_int),
    "agis_server_create": ([VP, C.c_size_t, C.c_int, P(VP)], C.c_int),
    "agis_server_submit": ([VP, VP, P(Opts), P(C.c_uint64)], C.c_int),
    "agis_server_poll": ([VP, C.c_uint64, P(Result), P(C.c_double), P(C.c_uint64)], C.c_int),
    "agis_server_stats": ([VP, P(C.c_uint64), P(C.c_uint64), P(C.c_int32), P(C.c_double), P(C.c_double)], C.c_int),
    "agis_server_destroy": ([VP], C.c_int),
    "agis_graph_save_tables": ([VP, C.c_char_p], C.c_int),
    "agis_graph_load_tables": ([VP, C.c_char_p], C.c_int),
    "agis_graph_fingerprint": ([VP, P(C.c_uint64)], C.c_int),
    "agis_tables_file_info": ([C.c_char_p, P(C.c_int64), P(C.c_int64), P(C.c_uint64), P(C.c_int32)], C.c_int),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name, None)
    if _f is None:
        continue
    _f.argtypes = _args
    _f.restype = _res


TILE = int(_lib.agis_tile_trials())    # trials per tile (the build's tile size)
TILE_WORDS = 6                         # AGIS_TILE_WORDS: uint64 words of one tile's output


class AgisError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({status})")


def status_str(s):
    return _lib.agis_status_str(s).decode()


def _check(rc, what):
    if rc != OK:
        raise AgisError(rc, what)


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def default_opts(**kw):
    o = Opts()
    _lib.agis_default_opts(C.byref(o))
    names = {f[0] for f in Opts._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


def prefix_sum_u64_noalloc(in_ptr: int, n: int, out_ptr: int, stream: int = 0):
    """Inclusive uint64 prefix sum of n entries between two device buffers; allocates
    nothing (see include/agis.h)."""
    _check(_lib.agis_prefix_sum_u64_noalloc(C.c_void_p(in_ptr), n, C.c_void_p(out_ptr),
                                            C.c_void_p(stream) if stream else None),
           "agis_prefix_sum_u64_noalloc")


def probe_random_read(buf_ptr: int, nbytes: int, reads: int, seed: int, stream: int, sink_ptr: int) -> int:
    """Enqueues the random 32-byte-sector read probe; returns the reads issued."""
    _check(_lib.agis_probe_random_read(C.c_void_p(buf_ptr), nbytes, reads, seed,
                                       C.c_void_p(stream) if stream else None, C.c_void_p(sink_ptr)),
           "agis_probe_random_read")
    return reads


def step_timers(reset=False):
    """Per-step-kind (cycles, steps) of the sampler (a -DAGIS_STEP_TIMERS build)."""
    out = np.zeros(16, dtype=np.uint64)
    _check(_lib.agis_step_timers(_ptr(out), int(reset)), "agis_step_timers")
    kinds = ["step1", "single_backward", "listed_intersection", "listed_reuse", "list_free_scan"]
    return {k: (int(out[2 * i]), int(out[2 * i + 1])) for i, k in enumerate(kinds)}


def kernel_launches():
    return int(_lib.agis_kernel_launches())


def z_of_delta(delta):
    return float(_lib.agis_z_of_delta(delta))


# ------------------------------------------------------------------ handles

class Context:
    def __init__(self, device=0, stream=None):
        h = VP()
        s = None if stream is None else C.c_void_p(int(stream))
        _check(_lib.agis_create(device, s, C.byref(h)), "agis_create")
        self.h = h

    def close(self):
        if self.h:
            _lib.agis_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pattern:
    def __init__(self, k, edges):
        flat = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
        h = VP()
        _check(_lib.agis_pattern_create(k, len(flat) // 2, flat.ctypes.data_as(P(C.c_int32)), C.byref(h)),
               "agis_pattern_create")
        self.h = h
        self.k = k
        self.edges = [tuple(e) for e in np.asarray(edges).reshape(-1, 2).tolist()]

    def info(self):
        k = C.c_int32()
        order = (C.c_int32 * 8)()
        cfg = (C.c_int32 * 32)()
        cert = (C.c_double * 8)()
        back = (C.c_uint8 * 8)()
        aut = C.c_uint64()
        _check(_lib.agis_pattern_info(self.h, C.byref(k), order, cfg, cert, back, C.byref(aut)), "agis_pattern_info")
        n = k.value
        return {"k": n, "order": list(order)[:n],
                "cfg": [tuple(cfg[4 * i:4 * i + 4]) for i in range(n)],
                "certainty": list(cert)[:n],
                "back": [[j for j in range(8) if back[i] >> j & 1] for i in range(n)],
                "aut": aut.value}

    def decide(self, mode=MODE_AUTO, beta=0.8):
        u = (C.c_uint8 * 8)()
        _check(_lib.agis_pattern_decide(self.h, mode, beta, u), "agis_pattern_decide")
        return list(u)[:self.k]

    def close(self):
        if self.h:
            _lib.agis_pattern_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A device-resident CSR graph (agis_graph)."""

    def __init__(self, ctx: Context, off, cols, validate=True, on_device=False):
        self.ctx = ctx
        h = VP()
        if on_device:
            # torch CUDA tensors: pass their device addresses
            nv = off.numel() - 1
            nnz = cols.numel()
            is64 = 1 if off.element_size() == 8 else 0
            rc = _lib.agis_graph_load_csr(ctx.h, C.c_void_p(off.data_ptr()), is64, C.c_void_p(cols.data_ptr()),
                                          nv, nnz, 1, int(validate), C.byref(h))
        else:
            off = np.ascontiguousarray(off)
            cols = np.ascontiguousarray(cols, dtype=np.int32)
            is64 = 1 if off.dtype.itemsize == 8 else 0
            if off.dtype not in (np.int64, np.int32):
                off = off.astype(np.int64)
                is64 = 1
            rc = _lib.agis_graph_load_csr(ctx.h, _ptr(off), is64, _ptr(cols), len(off) - 1, len(cols), 0,
                                          int(validate), C.byref(h))
        _check(rc, "agis_graph_load_csr")
        self.h = h

    @classmethod
    def rmat(cls, ctx, scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1):
        self = cls.__new__(cls)
        self.ctx = ctx
        h = VP()
        _check(_lib.agis_graph_generate_rmat(ctx.h, scale, edge_factor, a, b, c, seed, C.byref(h)),
               "agis_graph_generate_rmat")
        self.h = h
        return self

    @classmethod
    def chung_lu(cls, ctx, n, gamma=2.1, mean_degree=32.0, seed=1):
        self = cls.__new__(cls)
        self.ctx = ctx
        h = VP()
        _check(_lib.agis_graph_generate_chunglu(ctx.h, n, gamma, mean_degree, seed, C.byref(h)),
               "agis_graph_generate_chunglu")
        self.h = h
        return self

    def orient(self):
        """The degree-ordered orientation for clique patterns (a new Graph)."""
        o = Graph.__new__(Graph)
        o.ctx = self.ctx
        h = VP()
        _check(_lib.agis_graph_orient(self.h, C.byref(h)), "agis_graph_orient")
        o.h = h
        return o

    @property
    def oriented(self):
        return _lib.agis_graph_is_oriented(self.h) == 1

    def preprocess(self, seed=1, c_min=2.0 ** -10):
        _check(_lib.agis_graph_preprocess(self.h, seed, c_min), "agis_graph_preprocess")

    def info(self):
        nv, nnz, md = C.c_int64(), C.c_int64(), C.c_int64()
        b = C.c_uint64()
        _check(_lib.agis_graph_info(self.h, C.byref(nv), C.byref(nnz), C.byref(md), C.byref(b)), "agis_graph_info")
        return {"nv": nv.value, "nnz": nnz.value, "max_degree": md.value, "device_bytes": b.value}

    def stats(self):
        nv = self.info()["nv"]
        nsum = np.zeros(nv, dtype=np.uint64)
        hits = np.zeros(nv, dtype=np.uint32)
        _check(_lib.agis_graph_stats_copy(self.h, _ptr(nsum), _ptr(hits)), "agis_graph_stats_copy")
        return nsum, hits

    def weight_table(self, cfg):
        nv = self.info()["nv"]
        q = np.zeros(nv, dtype=np.uint64)
        pref = np.zeros(nv, dtype=np.uint64)
        sh = C.c_int32()
        c = (C.c_int32 * 4)(*cfg)
        _check(_lib.agis_graph_weight_table(self.h, c, _ptr(q), _ptr(pref), C.byref(sh)), "agis_graph_weight_table")
        return q, pref, sh.value

    def row_prefix(self, cfg):
        nnz = self.info()["nnz"]
        r = np.zeros(nnz, dtype=np.uint64)
        c = (C.c_int32 * 4)(*cfg)
        _check(_lib.agis_graph_row_prefix(self.h, c, _ptr(r)), "agis_graph_row_prefix")
        return r

    def set_memory_policy(self, row_prefix_bytes=0, bitmap_bytes=0, bitmap_min_degree=0, list_entries=0):
        _check(_lib.agis_graph_set_memory_policy(self.h, row_prefix_bytes, bitmap_bytes, bitmap_min_degree,
                                                 list_entries), "agis_graph_set_memory_policy")

    def set_l2_window(self, nbytes):
        """Bytes of hub bitmaps kept persisting in L2 by sampler launches (0: off)."""
        _check(_lib.agis_graph_set_l2_window(self.h, nbytes), "agis_graph_set_l2_window")

    def validate(self):
        _check(_lib.agis_graph_validate(self.h), "agis_graph_validate")

    def csr(self):
        i = self.info()
        off = np.zeros(i["nv"] + 1, dtype=np.int64)
        cols = np.zeros(i["nnz"], dtype=np.int32)
        _check(_lib.agis_graph_copy_csr(self.h, _ptr(off), _ptr(cols)), "agis_graph_copy_csr")
        return off, cols

    def drop_tables(self):
        _check(_lib.agis_graph_drop_tables(self.h), "agis_graph_drop_tables")

    def save_tables(self, path):
        """Writes the statistics and cached weight tables to `path` (see agis.h)."""
        _check(_lib.agis_graph_save_tables(self.h, os.fsencode(path)), "agis_graph_save_tables")

    def load_tables(self, path):
        """Reads statistics and tables saved from a graph with the same CSR."""
        _check(_lib.agis_graph_load_tables(self.h, os.fsencode(path)), "agis_graph_load_tables")

    def fingerprint(self):
        f = C.c_uint64()
        _check(_lib.agis_graph_fingerprint(self.h, C.byref(f)), "agis_graph_fingerprint")
        return f.value

    def close(self):
        if getattr(self, "h", None):
            _lib.agis_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tables_file_info(path) -> dict:
    """Header of a table file (host only)."""
    nv, nnz, fp, nt = C.c_int64(), C.c_int64(), C.c_uint64(), C.c_int32()
    _check(_lib.agis_tables_file_info(os.fsencode(path), C.byref(nv), C.byref(nnz), C.byref(fp), C.byref(nt)),
           "agis_tables_file_info")
    return {"nv": nv.value, "nnz": nnz.value, "fingerprint": fp.value, "n_tables": nt.value}


def estimate(graph: Graph, pattern: Pattern, opts: Opts) -> dict:
    r = Result()
    _check(_lib.agis_estimate(graph.h, pattern.h, C.byref(opts), C.byref(r)), "agis_estimate")
    return r.as_dict()


def estimate_batch(graph: Graph, patterns, opts_list) -> list:
    n = len(patterns)
    ph = (VP * n)(*[p.h for p in patterns])
    oa = (Opts * n)(*opts_list)
    ra = (Result * n)()
    _check(_lib.agis_estimate_batch(graph.h, n, ph, oa, ra), "agis_estimate_batch")
    return [ra[i].as_dict() for i in range(n)]


def dump_trials(graph: Graph, pattern: Pattern, opts: Opts, first: int, count: int):
    emb = np.zeros((count, 8), dtype=np.int32)
    hit = np.zeros(count, dtype=np.uint8)
    x = np.zeros(count, dtype=np.float64)
    sec = np.zeros((count, 3), dtype=np.uint64)    # sectors, sectors_streamed, sectors_survey
    _check(_lib.agis_dump_trials(graph.h, pattern.h, C.byref(opts), first, count, _ptr(emb), _ptr(hit),
                                 _ptr(x), _ptr(sec)), "agis_dump_trials")
    return emb, hit, x, sec


def autotune(graph: Graph, patterns, opts_list, trials_per_query=1 << 16):
    """Returns the chosen (CTAs per SM, tiles per work item)."""
    n = len(patterns)
    ph = (VP * n)(*[p.h for p in patterns])
    oa = (Opts * n)(*opts_list)
    b = C.c_int32()
    t = C.c_int32()
    _check(_lib.agis_autotune(graph.h, n, ph, oa, trials_per_query, C.byref(b), C.byref(t)), "agis_autotune")
    return b.value, t.value


def prepare(graph: Graph, pattern: Pattern, opts: Opts):
    _check(_lib.agis_prepare(graph.h, pattern.h, C.byref(opts)), "agis_prepare")


def sample_device(graph: Graph, pattern: Pattern, opts: Opts, first: int, ntiles: int, tile_out_ptr: int):
    """Enqueues fixed-budget sampling; tile_out_ptr is a device address of
    ntiles*TILE_WORDS uint64 words (e.g. a torch.int64 CUDA tensor's data_ptr())."""
    _check(_lib.agis_sample_device(graph.h, pattern.h, C.byref(opts), first, ntiles, C.c_void_p(tile_out_ptr)),
           "agis_sample_device")


def tile_sums(words: np.ndarray) -> dict:
    """Decodes tile output words (n x TILE_WORDS uint64): per-tile hits, sectors,
    sum_x, sum_x2, streamed (sectors_streamed) and survey (sectors_survey)."""
    w = np.ascontiguousarray(words, dtype=np.uint64).reshape(-1, TILE_WORDS)
    return {"hits": w[:, 0], "sectors": w[:, 1], "sum_x": w[:, 2].view(np.float64),
            "sum_x2": w[:, 3].view(np.float64), "streamed": w[:, 4], "survey": w[:, 5]}


class Server:
    def __init__(self, graph: Graph, scratch_bytes: int, max_slots: int):
        h = VP()
        _check(_lib.agis_server_create(graph.h, scratch_bytes, max_slots, C.byref(h)), "agis_server_create")
        self.h = h
        self.graph = graph

    def submit(self, pattern: Pattern, opts: Opts) -> int:
        t = C.c_uint64()
        _check(_lib.agis_server_submit(self.h, pattern.h, C.byref(opts), C.byref(t)), "agis_server_submit")
        return t.value

    def poll(self, ticket):
        r = Result()
        lat = C.c_double()
        ep = (C.c_uint64 * 2)()
        rc = _lib.agis_server_poll(self.h, ticket, C.byref(r), C.byref(lat), ep)
        if rc == ERR_BUSY:
            return None
        _check(rc, "agis_server_poll")
        d = r.as_dict()
        d["latency_s"] = lat.value
        d["admit_epoch"], d["finish_epoch"] = ep[0], ep[1]
        return d

    def stats(self):
        c, e = C.c_uint64(), C.c_uint64()
        p = C.c_int32()
        busy, span = C.c_double(), C.c_double()
        _check(_lib.agis_server_stats(self.h, C.byref(c), C.byref(e), C.byref(p), C.byref(busy), C.byref(span)),
               "agis_server_stats")
        return {"completed": c.value, "epochs": e.value, "peak_slots": p.value, "gpu_busy_s": busy.value,
                "busy_span_s": span.value,
                "gpu_idle_frac": (1.0 - busy.value / span.value) if span.value > 0 else None}

    def close(self):
        if getattr(self, "h", None):
            _lib.agis_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
