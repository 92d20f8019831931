#!/usr/bin/env python
"""Benchmark of the AGIS counting hot path on B300 (one JSON line on stdout).

Workload (plain per-query launches): R-MAT scale 22 (4.2M vertices, edge factor
16, a=0.57 b=0.19 c=0.19, symmetrised, deduplicated, int32 columns), patterns
4-clique, 5-cycle, house and 5-clique, 2^28 trials each under the decision
function D^pi (beta = 0.8), FP64 estimate and variance.  One step is one pass
of the whole path over that input: Sec. 4.4 preprocessing (neighbour-degree sums
and sampled clustering coefficients), the f_approx weight tables and prefix
sums, 2^28 Alg. 3 trials per pattern with per-tile FP64 reductions, and the
final sums.  Inputs are synthetic; the paper's data sets are not available.

Also reported: the same metric end to end through the C ABI from host buffers
(`e2e`), time to +-1% error at 95% confidence (Alg. 1, eps = 0.01, delta = 0.05)
for plain, batched and served forms, the sampler kernel's achieved bandwidth
against the measured HBM copy peak (`roofline`), and the CPU oracle on a bounded
sample of the same workload on this host's cores (`cpu_baseline`).

--impl reference times the CPU oracle instead (the reference arm of this
repository; the paper's own code is not available here).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "samples/s & time-to-±1% err (95% CI), batched/served vs plain, 1 B300"
PATTERN_NAMES = ["4-clique", "5-cycle", "house", "5-clique"]
CMIN = 2.0 ** -10


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="agis", choices=["agis", "reference"])
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--log2-trials", type=int, default=28)
    ap.add_argument("--patterns", default=",".join(PATTERN_NAMES))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tte", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--json-out", default="")
    ap.add_argument("--batch64", action="store_true",
                    help="also run the batching configuration: R-MAT scale 24 built on the device, 64 "
                         "queries with budgets 2^16..2^26, one autotuned persistent launch vs 64 plain launches")
    ap.add_argument("--batch-scale", type=int, default=24)
    ap.add_argument("--large", action="store_true",
                    help="also run the large-graph configuration: R-MAT scale 28, edge factor 32, built on the "
                         "device; 6-clique and 7-cycle to +-1%% under f_approx and f_uniform (2^30-trial budget)")
    ap.add_argument("--large-scale", type=int, default=28)
    ap.add_argument("--serve", action="store_true",
                    help="also run the serving configuration: Chung-Lu n=10M and R-MAT scale 24 resident on the "
                         "device, serving load on each (saturation, then Poisson at 50/80/95%%)")
    ap.add_argument("--serve-seconds", type=float, default=15.0)
    ap.add_argument("--concentration", action="store_true",
                    help="also run the concentration workload: all 6 four-vertex and 21 five-vertex "
                         "connected patterns as one batch each, to +-1%%")
    ap.add_argument("--anchor", action="store_true",
                    help="also compare the anchor draw with the S_tau build (time to +-1%%) on the bench patterns "
                         "and the 6-clique")
    ap.add_argument("--dag", action="store_true",
                    help="also run the 4/5/6-clique queries on the degree-ordered orientation vs the "
                         "undirected graph (time to +-1%%)")
    ap.add_argument("--ablation", action="store_true",
                    help="also run the f_approx term ablation and the beta sweep on the bench graph "
                         "(time and trials to +-1%%)")
    return ap.parse_args()


# ------------------------------------------------------------------ distributed (replicas only)

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"agis_bench_clocks_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ inputs

def workload_name(args, names):
    """The workload both arms report (the reference arm times a bounded sample of it)."""
    return (f"plain per-query launches: R-MAT scale {args.scale} (edge factor 16, a=0.57 b=0.19 c=0.19), "
            f"patterns {', '.join(names)}, 2^{args.log2_trials} trials each, D^pi (beta 0.8), "
            f"FP64 estimate and variance")


L2_BYTES = 126 * 1000 * 1000     # B300 L2


def l2_note(csr_bytes):
    """How the timed inputs compare with L2 (nothing is flushed between steps)."""
    rel = "larger" if csr_bytes > L2_BYTES else "not larger"
    return f"inputs {rel} than L2 (CSR {csr_bytes / 1e9:.2f} GB plus weight tables; L2 126 MB, not flushed)"


def make_workload(scale):
    from paper_2601_01388_b300 import inputs as I
    t = time.time()
    off, cols = I.rmat_graph(scale, 16, 0.57, 0.19, 0.19, seed=1)
    return off, cols, time.time() - t


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def kernel_source_hash():
    """sha256[:16] over the sampler's sources (kernel, shared definitions, RNG)."""
    h = hashlib.sha256()
    for f in ("sample.cu", "agis_internal.h", "philox.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2601_01388_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(trials_per_launch):
    """DRAM bytes per trial of the sampler from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "sample_kernel_rmat_s22.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    if f"kernel sources sha256[:16]: {kernel_source_hash()}" not in text:
        return None
    for line in text.splitlines():
        if line.strip().startswith("dram_bytes_per_trial:"):
            return float(line.split(":")[1].split()[0]) * trials_per_launch
    return None


# ------------------------------------------------------------------ CPU oracle

_ORC = {}


def _orc_init(shm_names, nv, nnz, nsum_name, hits_name):
    from multiprocessing import shared_memory
    from oracle import oracle as O
    O.build()
    shms = [shared_memory.SharedMemory(name=n) for n in shm_names + [nsum_name, hits_name]]
    _ORC["shms"] = shms
    _ORC["off"] = np.ndarray((nv + 1,), dtype=np.int64, buffer=shms[0].buf)
    _ORC["cols"] = np.ndarray((nnz,), dtype=np.int32, buffer=shms[1].buf)
    _ORC["nsum"] = np.ndarray((nv,), dtype=np.uint64, buffer=shms[2].buf)
    _ORC["hits"] = np.ndarray((nv,), dtype=np.uint32, buffer=shms[3].buf)
    _ORC["O"] = O


def _orc_stats(v0, v1):
    O = _ORC["O"]
    O.graph_stats_range(_ORC["off"], _ORC["cols"], 1, v0, v1, _ORC["nsum"], _ORC["hits"])
    return v1 - v0


def _orc_sample(name, seed, first, count):
    from paper_2601_01388_b300 import inputs as I
    O = _ORC["O"]
    key = (name, seed)
    q = _ORC.get(key)
    if q is None:
        k, edges = I.PATTERNS[name]
        q = O.Query(_ORC["off"], _ORC["cols"], k, edges, nsum=_ORC["nsum"], hits=_ORC["hits"],
                    c_min=CMIN, mode=0, seed=seed)
        _ORC[key] = q
    t = time.time()
    s = q.sums(first, count)
    return count, time.time() - t, s["sum_x"]


def host_cores():
    """Cores this process may run on (its CPU affinity), which may be fewer than the host has."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


class OraclePool:
    """The CPU oracle on all host cores: one spawn-started process per core, the CSR
    in shared memory, preprocessing split by vertex ranges and sampling split by
    disjoint trial ranges (the results are the single-process results)."""

    def __init__(self, off, cols, procs=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        self.nv, self.nnz = len(off) - 1, len(cols)
        self.procs = procs or host_cores()
        self.shm = []
        arrs = []
        for a in (off, cols):
            s = shared_memory.SharedMemory(create=True, size=max(a.nbytes, 1))
            np.ndarray(a.shape, dtype=a.dtype, buffer=s.buf)[:] = a
            self.shm.append(s)
        for dt in (np.uint64, np.uint32):
            s = shared_memory.SharedMemory(create=True, size=max(self.nv * np.dtype(dt).itemsize, 1))
            self.shm.append(s)
            arrs.append(s)
        ctx = mp.get_context("spawn")
        self.pool = ctx.Pool(self.procs, initializer=_orc_init,
                             initargs=([self.shm[0].name, self.shm[1].name], self.nv, self.nnz,
                                       self.shm[2].name, self.shm[3].name))

    def preprocess(self):
        t = time.time()
        parts = max(1, self.procs * 8)
        step = (self.nv + parts - 1) // parts
        ranges = [(v, min(self.nv, v + step)) for v in range(0, self.nv, step)]
        self.pool.starmap(_orc_stats, ranges)
        return time.time() - t

    def sample(self, names, per_pattern, seed_base=1):
        """per_pattern trials of each pattern, split across processes; returns
        (trials, wall seconds)."""
        jobs = []
        chunk = max(1, per_pattern // self.procs)
        for i, n in enumerate(names):
            for first in range(0, per_pattern, chunk):
                jobs.append((n, seed_base + i, first, min(chunk, per_pattern - first)))
        t = time.time()
        res = self.pool.starmap(_orc_sample, jobs)
        return sum(r[0] for r in res), time.time() - t

    def close(self):
        self.pool.terminate()
        for s in self.shm:
            s.close()
            s.unlink()


def cpu_rate(pool, names, seconds):
    """Samples/s of the oracle on a bounded sample sized to about `seconds`."""
    per = max(pool.procs, 64)
    n, dt = pool.sample(names, per)            # warms every process's query state
    while dt < seconds / 4 and per < (1 << 26):
        per *= 4
        n, dt = pool.sample(names, per)
    return n / dt, n, dt, per


# ------------------------------------------------------------------ serving load

def _serve_queries(agis, rng, n, seed_base):
    from paper_2601_01388_b300 import inputs as I
    qs = []
    for i in range(n):
        k, e = I.random_connected_pattern(rng, 3, 8, 0.3)
        o = agis.default_opts(mode=0, seed=seed_base + i, eps=float(rng.uniform(0.01, 0.05)), delta=0.05,
                              chunk_trials=1 << 16, min_trials=1 << 16, max_trials=1 << 24)
        qs.append((agis.Pattern(k, e), o))
    return qs


def _drive_server(srv, qs, arrivals):
    t0 = time.perf_counter()
    pending, lat, conv = {}, [], 0
    i, n = 0, len(qs)
    while i < n or pending:
        now = time.perf_counter() - t0
        while i < n and arrivals[i] <= now:
            pending[srv.submit(*qs[i])] = i
            i += 1
        for tk in list(pending):
            r = srv.poll(tk)
            if r is not None:
                lat.append(r["latency_s"])
                conv += r["converged"]
                del pending[tk]
        time.sleep(0.0002)
    return time.perf_counter() - t0, np.array(lat), conv


def serve_load(agis, g, seconds, seed=7, max_slots=64, budget=200 << 30, burst=64):
    """Serving on the resident graph: random connected 3-8-vertex patterns (Pruefer
    tree plus extra edges at p = 0.3), target relative error uniform in [1%, 5%] at
    95% confidence, at most 2^24 trials each.  The saturated rate is measured with
    a burst of queries submitted together; then Poisson arrivals at 50/80/95% of it
    for `seconds` each give p50/p99 latency and achieved queries/s."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x5345]))
    srv = agis.Server(g, budget, max_slots)
    qs = _serve_queries(agis, rng, burst, 10000)
    wall, lat, conv = _drive_server(srv, qs, np.zeros(burst))
    sat = burst / wall
    out = {"saturated_qps": sat, "burst": burst, "burst_wall_s": wall, "burst_converged": int(conv), "loads": []}
    for frac in (0.5, 0.8, 0.95):
        rate = frac * sat
        n = max(8, int(rate * seconds))
        qs = _serve_queries(agis, rng, n, 20000 + int(frac * 1000) * 1000)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
        wall, lat, conv = _drive_server(srv, qs, arrivals)
        out["loads"].append({"offered_qps": rate, "queries": n, "qps": n / wall, "p50_s": float(np.percentile(lat, 50)),
                             "p99_s": float(np.percentile(lat, 99)), "converged": int(conv)})
    st = srv.stats()
    srv.close()
    out["epochs"] = st["epochs"]
    out["peak_slots"] = st["peak_slots"]
    return out


def serving_configs(agis, ctx, seconds):
    """The serving configuration: a Chung-Lu power-law graph (10M vertices, degree
    exponent 2.1, mean degree 32) and the scale-24 R-MAT, both generated on the
    device and resident together; the serving load runs against each in turn."""
    import torch
    graphs = []
    t0 = time.perf_counter()
    cl = agis.Graph.chung_lu(ctx, 10_000_000, 2.1, 32.0, seed=1)
    cl.preprocess(1, CMIN)
    graphs.append(("Chung-Lu n=10M gamma=2.1 mean degree 32", cl, time.perf_counter() - t0))
    t0 = time.perf_counter()
    rm = agis.Graph.rmat(ctx, 24, 16, 0.57, 0.19, 0.19, seed=1)
    rm.preprocess(1, CMIN)
    graphs.append(("R-MAT scale 24 edge factor 16", rm, time.perf_counter() - t0))
    out = []
    for label, g, t_build in graphs:
        info = g.info()
        r = serve_load(agis, g, seconds)
        r.update({"graph": label, "nv": info["nv"], "nnz": info["nnz"], "max_degree": info["max_degree"],
                  "build_and_preprocess_s": t_build})
        out.append(r)
    for _, g, _ in graphs:
        g.close()
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ batching configuration

def batch64(agis, ctx, scale, stream):
    """64 pattern queries (cliques, cycles, paths, stars of 3-7 vertices, tailed
    triangle, diamond, chordal 5-cycle) with fixed trial budgets log-uniform in
    2^16..2^26 on an R-MAT graph generated on the device: all of them in one
    persistent launch (after the autotuner picks CTAs per SM and tiles per item)
    against 64 plain launches."""
    import torch
    from paper_2601_01388_b300 import inputs as I
    t0 = time.perf_counter()
    g = agis.Graph.rmat(ctx, scale, 16, 0.57, 0.19, 0.19, seed=1)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    g.preprocess(1, CMIN)
    t_prep = time.perf_counter() - t0
    qs = I.batch_queries(64, seed=1)
    pats = [agis.Pattern(*pat) for _, pat, _ in qs]
    opts = [agis.default_opts(mode=0, seed=500 + i, eps=0.0, max_trials=b) for i, (_, _, b) in enumerate(qs)]
    t0 = time.perf_counter()
    for p, o in zip(pats, opts):
        agis.prepare(g, p, o)
    t_tables = time.perf_counter() - t0
    best, span = agis.autotune(g, pats, opts, 1 << 15)
    total = sum(b for _, _, b in qs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [agis.estimate(g, p, o) for p, o in zip(pats, opts)]
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    batched = agis.estimate_batch(g, pats, opts)
    t_batch = time.perf_counter() - t0
    same = all(a["sum_x"] == b["sum_x"] and a["hits"] == b["hits"] for a, b in zip(plain, batched))
    info = g.info()
    g.close()
    return {"graph": f"R-MAT scale {scale} (device), nv {info['nv']}, nnz {info['nnz']}, max degree {info['max_degree']}",
            "generate_s": t_gen, "preprocess_s": t_prep, "tables_s": t_tables, "queries": len(qs),
            "trials": total, "autotuned_ctas_per_sm": best, "autotuned_tiles_per_item": span, "plain_s": t_plain, "batched_s": t_batch,
            "plain_samples_per_s": total / t_plain, "batched_samples_per_s": total / t_batch,
            "same_results": same}


# ------------------------------------------------------------------ large graph

def large_graph(agis, ctx, scale):
    """R-MAT scale 28 with edge factor 32 built on the device (int64 offsets, int32
    columns); time to +-1% at 95% confidence for the 6-clique and the 7-cycle under
    f_approx (D^pi) (at most 2^30 trials) and f_uniform (at most 2^28).  Row
    prefixes are kept to the highest-degree rows within 12 GB per configuration."""
    import torch
    from paper_2601_01388_b300 import inputs as I
    t0 = time.perf_counter()
    g = agis.Graph.rmat(ctx, scale, 32, 0.57, 0.19, 0.19, seed=1)
    t_gen = time.perf_counter() - t0
    g.set_memory_policy(row_prefix_bytes=12 << 30)
    t0 = time.perf_counter()
    g.preprocess(1, CMIN)
    t_prep = time.perf_counter() - t0
    info = g.info()
    out = {"graph": f"R-MAT scale {scale} edge factor 32 (device): nv {info['nv']}, nnz {info['nnz']}, "
                    f"max degree {info['max_degree']}", "generate_s": t_gen, "preprocess_s": t_prep, "runs": []}
    for name in ("6-clique", "7-cycle"):
        p = agis.Pattern(*I.PATTERNS[name])
        for mode, label, cap in ((0, "f_approx (D^pi)", 1 << 30), (2, "f_uniform", 1 << 28)):
            g.drop_tables()
            o = agis.default_opts(mode=mode, seed=7, eps=0.01, delta=0.05, chunk_trials=1 << 16,
                                  min_trials=1 << 16, max_trials=cap)
            t1 = time.perf_counter()
            agis.prepare(g, p, o)
            t_tab = time.perf_counter() - t1
            t1 = time.perf_counter()
            r = agis.estimate(g, p, o)
            dt = time.perf_counter() - t1
            out["runs"].append({"pattern": name, "distribution": label, "tables_s": t_tab, "s": dt,
                                "trials": r["trials"], "converged": r["converged"], "estimate": r["estimate"],
                                "eps_hat": r["eps_hat"], "samples_per_s": r["trials"] / dt})
    out["device_bytes"] = g.info()["device_bytes"]
    g.close()
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ ablation and beta

ABLATION_PATTERNS = ["4-clique", "4-path", "5-cycle", "house", "5-clique"]
# certainty below 1 on some steps (Def. decision_function), so beta changes the plan
BETA_PATTERNS = {
    "4-cycle": None, "5-cycle": None, "house": None, "7-cycle": None,
    "rand6-a": (6, [(0, 2), (0, 3), (0, 5), (1, 3), (1, 5), (2, 3), (2, 5), (3, 4), (4, 5)]),
    "rand7-b": (7, [(0, 2), (0, 3), (0, 5), (0, 6), (1, 3), (1, 5), (1, 6), (2, 4), (3, 5), (3, 6),
                    (4, 6)]),
}
BETAS = [("-inf", 1, 0.0), ("0.5", 0, 0.5), ("0.7", 0, 0.7), ("0.8", 0, 0.8), ("0.9", 0, 0.9),
         ("1.0", 0, 1.0), ("+inf", 2, 0.0)]


def ablation(agis, g, cap_log2=28):
    """Sec. 6.2 and Sec. 6.1 on the resident graph: trials and seconds to +-1% (95%)
    with the incremental versions of f_approx (T[F1]; + T[I1]; + T[F2]) and f_uniform,
    then across beta (-inf = f_approx on every step, +inf = f_uniform on every step).
    Runs stop at 2^cap_log2 trials; an unconverged run reports the trials it would
    need, trials * (eps_hat / eps)^2, since the half-width shrinks as 1/sqrt(n)."""
    from paper_2601_01388_b300 import inputs as I
    acc = dict(eps=0.01, delta=0.05, chunk_trials=1 << 16, min_trials=1 << 16, max_trials=1 << cap_log2)

    def run(p, o):
        g.drop_tables()
        t0 = time.perf_counter()
        agis.prepare(g, p, o)
        t_tab = time.perf_counter() - t0
        t0 = time.perf_counter()
        r = agis.estimate(g, p, o)
        dt = time.perf_counter() - t0
        need = r["trials"] if r["converged"] else int(r["trials"] * (r["eps_hat"] / 0.01) ** 2)
        return {"trials": r["trials"], "converged": r["converged"], "trials_needed": need,
                "estimate": r["estimate"], "eps_hat": r["eps_hat"], "tables_s": t_tab, "s": dt}

    out = {"cap_trials": 1 << cap_log2, "terms": [], "beta": []}
    for name in ABLATION_PATTERNS:
        p = agis.Pattern(*I.PATTERNS[name])
        for terms, label in ((1, "T[F1]"), (3, "T[F1]+T[I1]"), (7, "T[F1]+T[I1]+T[F2]"), (0, "f_uniform")):
            o = agis.default_opts(mode=2 if terms == 0 else 1, terms=terms, seed=31, **acc)
            out["terms"].append({"pattern": name, "f": label, **run(p, o)})
    for name, pat in BETA_PATTERNS.items():
        k, edges = pat if pat is not None else I.PATTERNS[name]
        p = agis.Pattern(k, edges)
        for label, mode, beta in BETAS:
            o = agis.default_opts(mode=mode, beta=beta, seed=37, **acc)
            uses = [int(u) for u in p.decide(mode, beta)]
            out["beta"].append({"pattern": name, "beta": label, "use_approx": uses, **run(p, o)})
    return out


# ------------------------------------------------------------------ concentration

def concentration_run(agis, g, cap_log2=28):
    """Sec. 6.3 on the resident graph: every connected 4-vertex (6) and 5-vertex (21)
    pattern as one batch, each to +-1% (95%); concentrations of the non-induced
    subgraph counts, and the variation distance between two independently seeded
    batches as an empirical accuracy figure."""
    from paper_2601_01388_b300 import concentration as K
    out = {}
    for k in (4, 5):
        pats = K.connected_patterns(k)
        ps = [agis.Pattern(*p) for p in pats]
        vecs = []
        for rep in range(2):
            opts = [agis.default_opts(eps=0.01, delta=0.05, seed=1000 * (rep + 1) + i, chunk_trials=1 << 16,
                                      min_trials=1 << 16, max_trials=1 << cap_log2) for i in range(len(ps))]
            g.drop_tables()
            t0 = time.perf_counter()
            rs = agis.estimate_batch(g, ps, opts)
            dt = time.perf_counter() - t0
            c = K.concentration(K.subgraph_counts([r["estimate"] for r in rs], k))
            vecs.append(c)
            if rep == 0:
                out[f"k{k}"] = {"patterns": len(ps), "s": dt, "trials": int(sum(r["trials"] for r in rs)),
                                "all_converged": all(r["converged"] for r in rs),
                                "concentration": [float(x) for x in c],
                                "edges": [p[1] for p in pats]}
        out[f"k{k}"]["variation_distance_between_seeds"] = K.variation_distance(vecs[0], vecs[1])
    return out


# ------------------------------------------------------------------ orientation for cliques

def cliques_oriented(agis, g, cap_log2=30):
    """Sec. 5.4's orientation for clique patterns on the resident graph: time to
    orient and preprocess the DAG, then time and trials to +-1% (95%) for the 4-, 5-
    and 6-clique on the undirected graph and on the orientation (same seeds)."""
    from paper_2601_01388_b300 import inputs as I
    t0 = time.perf_counter()
    o = g.orient()
    t_orient = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.preprocess(1, CMIN)
    t_prep = time.perf_counter() - t0
    info = o.info()
    out = {"orient_s": t_orient, "preprocess_s": t_prep, "nnz": info["nnz"], "max_out_degree": info["max_degree"],
           "runs": []}
    for name in ("4-clique", "5-clique", "6-clique"):
        p = agis.Pattern(*I.PATTERNS[name])
        for label, graph, anchor in (("undirected", g, 0), ("oriented", o, 0), ("oriented+anchor", o, 1)):
            opts = agis.default_opts(mode=0, seed=53, anchor=anchor, eps=0.01, delta=0.05, chunk_trials=1 << 16,
                                     min_trials=1 << 16, max_trials=1 << cap_log2)
            graph.drop_tables()
            t0 = time.perf_counter()
            agis.prepare(graph, p, opts)
            t_tab = time.perf_counter() - t0
            t0 = time.perf_counter()
            r = agis.estimate(graph, p, opts)
            dt = time.perf_counter() - t0
            out["runs"].append({"pattern": name, "graph": label, "tables_s": t_tab, "s": dt, "trials": r["trials"],
                                "converged": r["converged"], "estimate": r["estimate"], "eps_hat": r["eps_hat"],
                                "samples_per_s": r["trials"] / dt if dt > 0 else None})
    o.close()
    return out


# ------------------------------------------------------------------ anchor draw

def anchor_vs_exact(agis, g, names, cap_log2=30):
    """Time and trials to +-1% (95%) for each pattern with S_tau built as in Alg. 3
    and with the anchor draw (proposal from the shortest backward row, closing edges
    checked afterwards), same seeds."""
    from paper_2601_01388_b300 import inputs as I
    out = []
    for name in names:
        p = agis.Pattern(*I.PATTERNS[name])
        for anchor in (0, 1):
            o = agis.default_opts(mode=0, seed=61, anchor=anchor, eps=0.01, delta=0.05, chunk_trials=1 << 16,
                                  min_trials=1 << 16, max_trials=1 << cap_log2)
            g.drop_tables()
            t0 = time.perf_counter()
            agis.prepare(g, p, o)
            t_tab = time.perf_counter() - t0
            t0 = time.perf_counter()
            r = agis.estimate(g, p, o)
            dt = time.perf_counter() - t0
            out.append({"pattern": name, "draw": "anchor" if anchor else "S_tau", "tables_s": t_tab, "s": dt,
                        "trials": r["trials"], "hit_rate": r["hits"] / max(r["trials"], 1),
                        "converged": r["converged"], "estimate": r["estimate"],
                        "samples_per_s": r["trials"] / dt if dt > 0 else None})
    return out


# ------------------------------------------------------------------ GPU arm

def run_gpu(args, world, rank, local):
    import torch
    from paper_2601_01388_b300 import build
    build.build()
    from paper_2601_01388_b300 import agis
    from paper_2601_01388_b300 import inputs as I

    names = [n for n in args.patterns.split(",") if n]
    trials = 1 << args.log2_trials
    ntiles = (trials + agis.TILE - 1) // agis.TILE
    off, cols, t_gen = make_workload(args.scale)

    pool = None
    want_cpu = (rank == 0 and world == 1 and not args.no_cpu)
    if want_cpu:
        pool = OraclePool(off, cols)              # spawn-started processes

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = agis.Context(local, stream.cuda_stream)
    with torch.cuda.stream(stream):
        g = agis.Graph(ctx, off, cols, validate=True)
        info = g.info()
        pats = [agis.Pattern(*I.PATTERNS[n]) for n in names]
        opts = [agis.default_opts(mode=0, seed=1 + i, eps=0.0, max_trials=trials) for i in range(len(names))]
        outs = [torch.zeros(ntiles * 4, dtype=torch.int64, device="cuda") for _ in names]

        def step(record):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 + 2 * len(names))]
            ev[0].record(stream)
            g.preprocess(1, CMIN)                           # a1, a2 (Sec. 4.4)
            ev[1].record(stream)
            for p, o in zip(pats, opts):                    # a3, a4 (tables + prefix sums)
                agis.prepare(g, p, o)
            ev[2].record(stream)
            for j, (p, o) in enumerate(zip(pats, opts)):    # a5..a10 (Alg. 3 + reductions)
                ev[3 + 2 * j].record(stream)
                agis.sample_device(g, p, o, 0, ntiles, outs[j].data_ptr())
                ev[4 + 2 * j].record(stream)
            words = [o.cpu().numpy().view(np.uint64) for o in outs]   # step result to host
            stream.synchronize()
            res = []
            for w in words:
                h, sec, sx, sx2 = agis.tile_sums(w)
                res.append((int(h.sum()), int(sec.sum()), float(sx.sum()), float(sx2.sum())))
            t = {"preprocess": ev[0].elapsed_time(ev[1]), "tables": ev[1].elapsed_time(ev[2]),
                 "sample": [ev[3 + 2 * j].elapsed_time(ev[4 + 2 * j]) for j in range(len(names))]}
            if record is not None:
                record.append((t, res))
            return t, res

        for _ in range(args.warmup):
            step(None)
        stream.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        launches0 = agis.kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        recs = []
        e0.record(stream)
        for _ in range(args.steps):
            step(recs)
        e1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        barrier(world)
        launches = agis.kernel_launches() - launches0
        clk = clocks.stop()
        ms = e0.elapsed_time(e1) / args.steps
        ms = allreduce_max(ms, world)
        trials_per_step = trials * len(names)
        value = trials_per_step * world / (ms / 1000.0)

        # random 32-byte-sector read bandwidth over 16 GB (the random-access roofline)
        rand_gbs = None
        try:
            buf = torch.empty(16 << 30, dtype=torch.uint8, device="cuda")
            sink = torch.zeros(1, dtype=torch.int64, device="cuda")
            sms = torch.cuda.get_device_properties(local).multi_processor_count
            threads = sms * 2048
            reads = 1 << 30
            per = -(-reads // threads)
            per = -(-per // 8) * 8
            issued = threads * per
            best = None
            for rep in range(4):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                agis.probe_random_read(buf.data_ptr(), buf.numel(), reads, rep + 1, stream.cuda_stream, sink.data_ptr())
                b.record(stream)
                b.synchronize()
                ms_r = a.elapsed_time(b)
                if rep > 0 and (best is None or ms_r < best):
                    best = ms_r
            rand_gbs = issued * 32 / (best / 1000.0) / 1e9
            del buf
            torch.cuda.empty_cache()
        except Exception:
            rand_gbs = None

        # roofline of the sampler kernel: algorithmic sectors / its own event time
        samp_ms = [sum(t["sample"]) for t, _ in recs]
        sectors = [sum(r[1] for r in res) for _, res in recs]
        per_launch_ms = statistics.mean([x for t, _ in recs for x in t["sample"]])
        achieved = statistics.mean([s * 32 / (m / 1000.0) for s, m in zip(sectors, samp_ms)]) / 1e9
        peak, peak_kind = measured_peaks()
        traffic = profile_traffic(trials)
        last = recs[-1][1]
        phases = {k: statistics.mean([t[k] for t, _ in recs]) for k in ("preprocess", "tables")}
        phases["sample"] = statistics.mean(samp_ms)
        per_pattern = {n: {"estimate": r[2] / trials, "hits": r[0], "sectors_per_trial": r[1] / trials,
                           "ms": statistics.mean([t["sample"][j] for t, _ in recs])}
                       for j, (n, r) in enumerate(zip(names, last))}

        # ---- end to end through the C ABI from pinned host buffers
        e2e = None
        if not args.no_e2e:
            h_off = torch.from_numpy(off).pin_memory().numpy()
            h_cols = torch.from_numpy(cols).pin_memory().numpy()
            reps = 1
            d2h = 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                ge = agis.Graph(ctx, h_off, h_cols, validate=False)
                ge.preprocess(1, CMIN)
                for p, o in zip(pats, opts):
                    r = agis.estimate(ge, p, o)
                    d2h += ntiles * 32 + 136
                ge.close()
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / reps
            e2e = {"value": trials_per_step / dt, "unit": "samples/s",
                   "h2d_bytes_per_step": int(h_off.nbytes + h_cols.nbytes + len(names) * 600),
                   "d2h_bytes_per_step": int(d2h / reps), "s_per_step": dt}

        # ---- time to +-1% (95% CI): plain, batched, served; and f_uniform for contrast
        tte = None
        if not args.no_tte:
            tte = {}
            acc = dict(eps=0.01, delta=0.05, chunk_trials=1 << 16, min_trials=1 << 16)
            plain = []
            t0 = time.perf_counter()
            for i, p in enumerate(pats):
                o = agis.default_opts(mode=0, seed=101 + i, max_trials=1 << 34, **acc)
                t1 = time.perf_counter()
                r = agis.estimate(g, p, o)
                plain.append({"pattern": names[i], "s": time.perf_counter() - t1, "trials": r["trials"],
                              "converged": r["converged"], "estimate": r["estimate"]})
            tte["plain_total_s"] = time.perf_counter() - t0
            tte["plain"] = plain
            bo = [agis.default_opts(mode=0, seed=101 + i, max_trials=1 << 34, **acc) for i in range(len(pats))]
            t0 = time.perf_counter()
            br = agis.estimate_batch(g, pats, bo)
            tte["batched_total_s"] = time.perf_counter() - t0
            tte["batched_same_result"] = all(a["trials"] == b["trials"] and a["estimate"] == b["estimate"]
                                             for a, b in zip(plain, br))
            srv = agis.Server(g, 200 << 30, 64)
            t0 = time.perf_counter()
            tickets = [srv.submit(p, o) for p, o in zip(pats, bo)]
            done = {}
            while len(done) < len(tickets):
                for tk in tickets:
                    if tk not in done:
                        r = srv.poll(tk)
                        if r is not None:
                            done[tk] = r
                time.sleep(0.0005)
            tte["served_total_s"] = time.perf_counter() - t0
            tte["served_same_result"] = all(done[tk]["trials"] == a["trials"] for tk, a in zip(tickets, plain))
            srv.close()
            uni = []
            for i, p in enumerate(pats):
                o = agis.default_opts(mode=2, seed=101 + i, max_trials=1 << 30, **acc)
                t1 = time.perf_counter()
                r = agis.estimate(g, p, o)
                uni.append({"pattern": names[i], "s": time.perf_counter() - t1, "trials": r["trials"],
                            "converged": r["converged"]})
            tte["uniform_plain"] = uni

        large = None
        if args.large:
            large = large_graph(agis, ctx, args.large_scale)

        batching = None
        if args.batch64:
            batching = batch64(agis, ctx, args.batch_scale, stream)

        serving = None
        if args.serve:
            serving = serving_configs(agis, ctx, args.serve_seconds)

        abl = None
        if args.ablation:
            abl = ablation(agis, g)

        conc = None
        if args.concentration:
            conc = concentration_run(agis, g)

        dag = None
        if args.dag:
            dag = cliques_oriented(agis, g)

        anch = None
        if args.anchor:
            anch = anchor_vs_exact(agis, g, names + ["6-clique"])

    cpu = None
    if pool is not None:
        t_prep = pool.preprocess()
        rate, n, dt, per = cpu_rate(pool, names, args.cpu_seconds)
        cpu = {"value": rate, "unit": "samples/s", "cores": pool.procs, "kind": "oracle",
               "sample": f"{per} trials of each of {', '.join(names)} (AUTO, seeds 1..4) on the same "
                         f"scale-{args.scale} graph, split over {pool.procs} processes; {dt:.1f} s; "
                         f"oracle preprocessing {t_prep:.1f} s not included"}
        pool.close()

    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args, names),
                   "nv": info["nv"], "nnz": info["nnz"], "max_degree": info["max_degree"],
                   "trials_per_pattern": trials, "parallelism": f"replicas x{world}",
                   "l2": l2_note(off.nbytes + cols.nbytes),
                   "graph_generation_s": t_gen},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "sample_kernel",
                     "peak_kind": peak_kind, "per_launch_ms": per_launch_ms,
                     "random_access_gbs": rand_gbs,
                     "frac_of_random_access": (achieved / rand_gbs) if rand_gbs else None,
                     "algorithmic_bytes_per_launch": statistics.mean(sectors) * 32 / len(names)},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "phases_ms": phases,
        "per_pattern": per_pattern,
        "time_to_1pct": tte,
    }
    if serving is not None:
        line["serving"] = serving
    if batching is not None:
        line["batch64"] = batching
    if large is not None:
        line["large_graph"] = large
    if abl is not None:
        line["ablation"] = abl
    if conc is not None:
        line["concentration"] = conc
    if dag is not None:
        line["cliques_oriented"] = dag
    if anch is not None:
        line["anchor_draw"] = anch
    return line


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle on the host cores, same metric and workload."""
    if rank != 0:
        return None
    names = [n for n in args.patterns.split(",") if n]
    off, cols, _ = make_workload(args.scale)
    pool = OraclePool(off, cols)
    t_prep = pool.preprocess()
    rate, n, dt, per = cpu_rate(pool, names, max(2.0, args.cpu_seconds / 3))
    times = []
    for _ in range(args.warmup):
        pool.sample(names, per)
    for _ in range(args.steps):
        nn, d = pool.sample(names, per)
        times.append(d)
    pool.close()
    ms = 1000.0 * statistics.mean(times)
    value = n / (ms / 1000.0)
    cpu = {"value": value, "unit": "samples/s", "cores": pool.procs, "kind": "oracle",
           "sample": f"{per} trials of each of {', '.join(names)} per step on the scale-{args.scale} graph "
                     f"over {pool.procs} processes; oracle preprocessing {t_prep:.1f} s not included"}
    return {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(args, names), "trials_per_pattern": 1 << args.log2_trials,
                       "parallelism": "host processes", "sampled": f"{per} trials of each pattern per step"},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    world, rank, local = dist_init()
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    else:
        line = run_gpu(args, world, rank, local)
    if rank == 0 and line is not None:
        s = json.dumps(line)
        print(s, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(s + "\n")
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
