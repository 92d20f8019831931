#!/usr/bin/env python
"""Benchmark of the AGIS counting hot path on B300 (one JSON line on stdout).

Workload (plain per-query launches): R-MAT scale 22 (4.2M vertices, edge factor
16, a=0.57 b=0.19 c=0.19, symmetrised, deduplicated, int32 columns), patterns
4-clique, 5-cycle, house and 5-clique, 2^28 trials each under the decision
function D^pi (beta = 0.8), FP64 estimate and variance.  One step is one plain
per-query launch of the whole path for one pattern, the patterns taken in turn
(step j runs pattern j mod 4, so every four steps cover the workload once):
Sec. 4.4 preprocessing (neighbour-degree sums, sampled clustering coefficients,
hub bitmaps), the pattern's f_approx weight tables and prefix sums, its 2^28
Alg. 3 trials with per-tile FP64 reductions, and the tile sums read back to the
host.  Warm-up steps run the same path at a smaller trial budget (they only
have to build the kernel instances, scratch and tables once).  Inputs are
synthetic; the paper's data sets are not available.

Also reported: the same metric end to end through the C ABI from pinned host
buffers (`e2e`: graph upload, preprocessing, tables, the estimate call and its
result, one rotation over the patterns), time to +-1% error at 95% confidence
(Alg. 1, eps = 0.01, delta = 0.05) for plain, batched and served forms, the
batching configuration (64 queries on a scale-24 R-MAT, each to +-1% or its
budget, one persistent batched call against 64 plain calls), the sampler
kernel's algorithmic bandwidth against the measured HBM copy peak (`roofline`),
and the CPU oracle on a bounded sample of the same workload on this host's
cores (`cpu_baseline`).  Every leg after the timed loop is skipped, and says
so, if the run would pass its deadline.

--impl reference times the CPU oracle instead (the reference arm of this
repository; the paper's own code is not available here).
"""
from __future__ import annotations

import argparse
import ctypes
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
# Alg. 1 checkpoint spacing (and first checkpoint) of the optional legs that run
# queries to +-1% (the time-to-+-1% legs take theirs from --tte-chunk-log2)
CHECKPOINT = 1 << 12


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4,
                    help="timed steps; step j is the full query of pattern j mod (number of patterns)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="agis", choices=["agis", "reference"])
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--log2-trials", type=int, default=28)
    ap.add_argument("--warmup-log2-trials", type=int, default=22,
                    help="trials of a warm-up step (same path, smaller budget)")
    ap.add_argument("--patterns", default=",".join(PATTERN_NAMES))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="end-to-end steps (default: one per pattern)")
    ap.add_argument("--no-tte", action="store_true")
    ap.add_argument("--tte-chunk-log2", type=int, default=12,
                    help="Alg. 1 checkpoint spacing (and first checkpoint) of the time-to-+-1%% legs")
    ap.add_argument("--tte-cap-log2", type=int, default=24, help="trial cap of an f_approx time-to-+-1%% query")
    ap.add_argument("--uniform-cap-log2", type=int, default=24,
                    help="trial cap of an f_uniform time-to-+-1%% query (the trials it would need are extrapolated)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--deadline-s", type=float, default=1500.0,
                    help="legs after the timed loop are skipped when their planned time would pass this")
    ap.add_argument("--json-out", default="")
    ap.add_argument("--summarize-ncu", default="",
                    help="(no GPU) turn an ncu CSV of sampler launches into the committed JSON traffic summary")
    ap.add_argument("--summary-out", default="")
    ap.add_argument("--summarize-launches", default="",
                    help="(no GPU) print the per-kernel table of an ncu --csv launch list")
    ap.add_argument("--ncu-command", default="", help="the ncu command line recorded in the summary")
    ap.add_argument("--no-batch64", dest="batch64", action="store_false",
                    help="skip the batching configuration: R-MAT scale 24 built on the device, 64 queries to "
                         "+-1%% with budgets 2^16..2^26 as caps, one batched call vs 64 plain calls")
    ap.add_argument("--list-entries", type=int, default=0,
                    help="memory policy: per-warp candidate-list capacity (0 = library default)")
    ap.add_argument("--bitmap-bytes", type=int, default=0,
                    help="memory policy: bytes for hub membership structures (0 = library default)")
    ap.add_argument("--batch-scale", type=int, default=24)
    ap.add_argument("--batch-eps", type=float, default=0.01)
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
    return ap.parse_args(argv)


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
    """sha256[:16] over the sampler's sources (kernel, the definitions it reads, RNG,
    and its launches, which set the persisting-L2 window)."""
    h = hashlib.sha256()
    for f in ("sample.cu", "agis_device.h", "philox.cuh", "launch.cu"):
        h.update(open(os.path.join(ROOT, "paper_2601_01388_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "sample_kernel_dram_rmat_s22.json")


def profile_traffic(path=TRAFFIC_SUMMARY):
    """Per-pattern DRAM bytes per trial of the sampler from the committed ncu summary
    (written by --summarize-ncu), if it was taken on the current kernel sources and
    the same workload; else None."""
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("kernel_sources_sha16") != kernel_source_hash():
        return None
    return {n: v["dram_bytes_per_trial"] for n, v in d.get("per_pattern", {}).items()}


def summarize_ncu(csv_path, out_path, names, trials, command, workload):
    """Reads an ncu --csv log of sampler launches (metrics dram__bytes_read.sum,
    dram__bytes_write.sum, gpu__time_duration.sum), one launch per pattern in the
    benchmark's order, and writes the per-pattern JSON summary the benchmark reads."""
    import csv
    rows = []
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        rows.append(r)
    launches = {}
    for r in rows:
        if "sample_kernel" not in r.get("Kernel Name", ""):
            continue
        lid = int(r["ID"])
        m = launches.setdefault(lid, {"kernel": r["Kernel Name"]})
        val = float(r["Metric Value"].replace(",", ""))
        unit = r.get("Metric Unit", "")
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12,
                 "nsecond": 1, "usecond": 1e3, "msecond": 1e6, "second": 1e9}.get(unit, 1)
        m[r["Metric Name"]] = val * scale
    ids = sorted(launches)
    per = {}
    for j, lid in enumerate(ids):
        name = names[j % len(names)]
        m = launches[lid]
        rd, wr = m.get("dram__bytes_read.sum", 0.0), m.get("dram__bytes_write.sum", 0.0)
        e = per.setdefault(name, {"launches": 0, "trials": 0, "dram_read_bytes": 0.0, "dram_write_bytes": 0.0,
                                  "duration_ns": 0.0})
        e["launches"] += 1
        e["trials"] += trials
        e["dram_read_bytes"] += rd
        e["dram_write_bytes"] += wr
        e["duration_ns"] += m.get("gpu__time_duration.sum", 0.0)
    for e in per.values():
        e["dram_bytes_per_trial"] = (e["dram_read_bytes"] + e["dram_write_bytes"]) / e["trials"]
        e["dram_gbs"] = (e["dram_read_bytes"] + e["dram_write_bytes"]) / e["duration_ns"] if e["duration_ns"] else None
    out = {"kernel": "sample_kernel", "kernel_sources_sha16": kernel_source_hash(), "workload": workload,
           "trials_per_launch": trials, "command": command, "per_pattern": per,
           "note": "ncu serialises launches: durations are for comparison only"}
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    return out


def summarize_launches(csv_path, by="kernel"):
    """Launches, summed gpu__time_duration and share of the total from an ncu --csv
    launch list (one metric per launch), per kernel or (by="nvtx", for a capture
    taken with --nvtx) per innermost NVTX range of this library ("agis:...", else
    "(none)"); returns rows sorted by time."""
    import csv
    import re
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    per = {}
    scale = {"ns": 1e-6, "nsecond": 1e-6, "usecond": 1e-3, "us": 1e-3, "msecond": 1.0, "ms": 1.0, "second": 1e3}
    for r in csv.DictReader(lines):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        if by == "nvtx":
            stack = next((v for k, v in r.items() if k and "Push/Pop" in k), "") or ""
            ranges = re.findall(r"(agis:[a-z_.]+)", stack)
            name = ranges[-1] if ranges else "(none)"
        else:
            name = r["Kernel Name"].split("(")[0].strip()
        ms = float(r["Metric Value"].replace(",", "")) * scale.get(r.get("Metric Unit", "ns"), 1e-6)
        e = per.setdefault(name, [0, 0.0])
        e[0] += 1
        e[1] += ms
    total = sum(v[1] for v in per.values()) or 1.0
    return sorted(((k, v[0], v[1], v[1] / total) for k, v in per.items()), key=lambda x: -x[2])


# ------------------------------------------------------------------ wall-time plan

# Rates the plan below assumes (samples/s): floors under the measured rates of the
# committed sampler, on the benchmark graph and on the scale-24 batching graph.
RATE_FLOOR = {"bench": 8.0e6, "batch": 4.0e6}
FIXED_S = 150.0      # torch import, library build check, host graph generation, upload, oracle pool, probe


def batch_budget_trials(n=64, seed=1):
    from paper_2601_01388_b300 import inputs as I
    return sum(b for _, _, b in I.batch_queries(n, seed=seed))


def plan_seconds(args, rates=RATE_FLOOR):
    """Upper bounds, per leg, of the wall time of a default run with these arguments:
    every capped query is assumed to run to its cap at the floor rates."""
    names = [n for n in args.patterns.split(",") if n]
    full = float(1 << args.log2_trials)
    p = {"fixed": FIXED_S,
         "warmup": args.warmup * float(1 << args.warmup_log2_trials) / rates["bench"],
         "timed": args.steps * full / rates["bench"]}
    if not args.no_e2e:
        p["e2e"] = (args.e2e_steps or len(names)) * full / rates["bench"]
    if not args.no_tte:
        # plain, batched and served forms under f_approx, then f_uniform alone
        p["tte"] = (3 * len(names) * float(1 << args.tte_cap_log2) +
                    len(names) * float(1 << args.uniform_cap_log2)) / rates["bench"]
    if args.batch64:
        p["batch64"] = 20.0 + 2 * batch_budget_trials() / rates["batch"]
    if not args.no_cpu:
        p["cpu"] = 4 * args.cpu_seconds + 10.0
    return p


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
                              chunk_trials=CHECKPOINT, min_trials=CHECKPOINT, max_trials=1 << 24)
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

def batch64(agis, ctx, scale, eps=0.01, chunk_log2=12, deadline=None):
    """The batching configuration: 64 pattern queries (cliques, cycles, paths,
    stars of 3-7 vertices, tailed triangle, diamond, chordal 5-cycle) on an R-MAT
    graph generated on the device, each run to +-eps at 95% confidence by Alg. 1
    with its budget (log-uniform in 2^16..2^26) as a cap: 64 plain calls (one
    query at a time) against one batched call (all queries share every epoch's
    persistent launch, after the autotuner picks CTAs per SM and tiles per item),
    then the same 64 queries submitted at once to a server.  Every query's result
    must be identical in the three forms."""
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
    chunk = 1 << chunk_log2
    opts = [agis.default_opts(mode=0, seed=500 + i, eps=eps, delta=0.05, chunk_trials=chunk, min_trials=chunk,
                              max_trials=b) for i, (_, _, b) in enumerate(qs)]
    t0 = time.perf_counter()
    for p, o in zip(pats, opts):
        agis.prepare(g, p, o)
    t_tables = time.perf_counter() - t0
    best, span = agis.autotune(g, pats, opts, 1 << 15)
    torch.cuda.synchronize()
    out = {"generate_s": t_gen, "preprocess_s": t_prep, "tables_s": t_tables, "queries": len(qs),
           "eps": eps, "delta": 0.05, "chunk_trials": chunk, "budget_trials": int(sum(b for _, _, b in qs)),
           "autotuned_ctas_per_sm": best, "autotuned_tiles_per_item": span}
    warm_query(agis, g, pats[0])
    t0 = time.perf_counter()
    plain = []
    for p, o in zip(pats, opts):
        t1 = time.perf_counter()
        r = agis.estimate(g, p, o)
        r["s"] = time.perf_counter() - t1
        plain.append(r)
    out["plain_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    batched = agis.estimate_batch(g, pats, opts)
    out["batched_s"] = time.perf_counter() - t0
    served = None
    if deadline is None or time.perf_counter() + out["batched_s"] * 1.5 < deadline:
        srv, warm_epochs = warm_server(agis, g, pats[0])
        t0 = time.perf_counter()
        tickets = [srv.submit(p, o) for p, o in zip(pats, opts)]
        done = {}
        while len(done) < len(tickets):
            for tk in tickets:
                if tk not in done:
                    r = srv.poll(tk)
                    if r is not None:
                        done[tk] = r
            time.sleep(0.0005)
        out["served_s"] = time.perf_counter() - t0
        out["served_epochs"] = srv.stats()["epochs"] - warm_epochs
        srv.close()
        served = [done[tk] for tk in tickets]
    keys = ("trials", "hits", "sum_x", "sum_x2", "converged", "estimate")
    out["batched_same_result"] = all(all(a[k] == b[k] for k in keys) for a, b in zip(plain, batched))
    if served is not None:
        out["served_same_result"] = all(all(a[k] == b[k] for k in keys) for a, b in zip(plain, served))
    trials = sum(r["trials"] for r in plain)
    out.update({"trials": int(trials), "converged": int(sum(r["converged"] for r in plain)),
                "plain_samples_per_s": trials / out["plain_s"], "batched_samples_per_s": trials / out["batched_s"],
                "batched_speedup": out["plain_s"] / out["batched_s"],
                "plain_launches": int(sum(r["launches"] for r in plain)),
                "batched_epochs": int(max(r["launches"] for r in batched))})
    out["per_query"] = [{"pattern": name, "budget": b, "trials": int(r["trials"]), "converged": int(r["converged"]),
                         "eps_hat": r["eps_hat"], "plain_s": r["s"]}
                        for (name, _, b), r in zip(qs, plain)]
    info = g.info()
    out["graph"] = (f"R-MAT scale {scale} (device), nv {info['nv']}, nnz {info['nnz']}, "
                    f"max degree {info['max_degree']}")
    g.close()
    torch.cuda.empty_cache()
    return out


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
            o = agis.default_opts(mode=mode, seed=7, eps=0.01, delta=0.05, chunk_trials=CHECKPOINT,
                                  min_trials=CHECKPOINT, max_trials=cap)
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
    acc = dict(eps=0.01, delta=0.05, chunk_trials=CHECKPOINT, min_trials=CHECKPOINT, max_trials=1 << cap_log2)

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
            opts = [agis.default_opts(eps=0.01, delta=0.05, seed=1000 * (rep + 1) + i, chunk_trials=CHECKPOINT,
                                      min_trials=CHECKPOINT, max_trials=1 << cap_log2) for i in range(len(ps))]
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
            opts = agis.default_opts(mode=0, seed=53, anchor=anchor, eps=0.01, delta=0.05, chunk_trials=CHECKPOINT,
                                     min_trials=CHECKPOINT, max_trials=1 << cap_log2)
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
            o = agis.default_opts(mode=0, seed=61, anchor=anchor, eps=0.01, delta=0.05, chunk_trials=CHECKPOINT,
                                  min_trials=CHECKPOINT, max_trials=1 << cap_log2)
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

def random_access_gbs(agis, stream, local):
    """Random 32-byte-sector read bandwidth over 16 GB (far beyond L2): the random-
    access roofline of the sampler's dependent gathers and searches."""
    import torch
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
        del buf
        torch.cuda.empty_cache()
        return issued * 32 / (best / 1000.0) / 1e9
    except Exception:
        return None


def warm_query(agis, g, p):
    """One small fixed-budget query, run before any timed form so that none of them
    pays the one-time allocation of the sampler's scratch."""
    agis.estimate(g, p, agis.default_opts(mode=0, seed=1, eps=0.0, max_trials=4096, chunk_trials=4096))


def warm_server(agis, g, p):
    """A server that has run one small query to completion (its scratch allocated);
    returns it with its epoch count so far."""
    srv = agis.Server(g, 200 << 30, 64)
    tk = srv.submit(p, agis.default_opts(mode=0, seed=1, eps=0.0, max_trials=4096, chunk_trials=4096))
    while srv.poll(tk) is None:
        time.sleep(0.0005)
    return srv, srv.stats()["epochs"]


def time_to_1pct(agis, g, pats, names, args, deadline):
    """Time to +-1% at 95% confidence (Alg. 1) for the benchmark patterns, with their
    weight tables built beforehand: one plain call per pattern, one batched call, one
    server with all of them submitted at once (identical results required), then
    f_uniform plain calls for contrast."""
    chunk = 1 << args.tte_chunk_log2
    acc = dict(eps=0.01, delta=0.05, chunk_trials=chunk, min_trials=chunk)
    cap = 1 << args.tte_cap_log2
    out = {"chunk_trials": chunk, "cap_trials": cap}
    keys = ("trials", "hits", "sum_x", "sum_x2", "converged", "estimate")
    opts = [agis.default_opts(mode=0, seed=101 + i, max_trials=cap, **acc) for i in range(len(pats))]
    # weight tables are per-graph preprocessing: built once before any form is timed
    t0 = time.perf_counter()
    for p, o in zip(pats, opts):
        agis.prepare(g, p, o)
    out["tables_s"] = time.perf_counter() - t0
    warm_query(agis, g, pats[0])
    plain = []
    t0 = time.perf_counter()
    for i, (p, o) in enumerate(zip(pats, opts)):
        t1 = time.perf_counter()
        r = agis.estimate(g, p, o)
        r["s"] = time.perf_counter() - t1
        plain.append(r)
    out["plain_total_s"] = time.perf_counter() - t0
    out["plain"] = [{"pattern": n, "s": r["s"], "trials": int(r["trials"]), "converged": int(r["converged"]),
                     "launches": int(r["launches"]), "estimate": r["estimate"], "eps_hat": r["eps_hat"]}
                    for n, r in zip(names, plain)]
    t0 = time.perf_counter()
    br = agis.estimate_batch(g, pats, opts)
    out["batched_total_s"] = time.perf_counter() - t0
    out["batched_same_result"] = all(all(a[k] == b[k] for k in keys) for a, b in zip(plain, br))
    srv, _ = warm_server(agis, g, pats[0])
    t0 = time.perf_counter()
    tickets = [srv.submit(p, o) for p, o in zip(pats, opts)]
    done = {}
    while len(done) < len(tickets):
        for tk in tickets:
            if tk not in done:
                r = srv.poll(tk)
                if r is not None:
                    done[tk] = r
        time.sleep(0.0002)
    out["served_total_s"] = time.perf_counter() - t0
    out["served_same_result"] = all(all(done[tk][k] == a[k] for k in keys) for tk, a in zip(tickets, plain))
    srv.close()
    uni = []
    ucap = 1 << args.uniform_cap_log2
    for i, p in enumerate(pats):
        if time.perf_counter() + ucap / RATE_FLOOR["bench"] > deadline:
            uni.append({"pattern": names[i], "skipped": "deadline"})
            continue
        o = agis.default_opts(mode=2, seed=101 + i, max_trials=ucap, **acc)
        t1 = time.perf_counter()
        r = agis.estimate(g, p, o)
        need = r["trials"] if r["converged"] else int(r["trials"] * (r["eps_hat"] / 0.01) ** 2)
        uni.append({"pattern": names[i], "s": time.perf_counter() - t1, "trials": int(r["trials"]),
                    "converged": int(r["converged"]), "trials_needed": need, "eps_hat": r["eps_hat"]})
    out["uniform_plain"] = uni
    return out


def run_gpu(args, world, rank, local):
    import torch
    from paper_2601_01388_b300 import build
    build.build()
    from paper_2601_01388_b300 import agis
    from paper_2601_01388_b300 import inputs as I

    t_start = time.perf_counter()
    deadline = t_start + args.deadline_s
    names = [n for n in args.patterns.split(",") if n]
    trials = 1 << args.log2_trials
    ntiles = (trials + agis.TILE - 1) // agis.TILE
    warm_trials = min(trials, 1 << args.warmup_log2_trials)
    off, cols, t_gen = make_workload(args.scale)

    pool = None
    want_cpu = (rank == 0 and world == 1 and not args.no_cpu)
    if want_cpu:
        pool = OraclePool(off, cols)              # spawn-started processes

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = agis.Context(local, stream.cuda_stream)
    skipped = {}
    with torch.cuda.stream(stream):
        g = agis.Graph(ctx, off, cols, validate=True)
        if args.list_entries or args.bitmap_bytes:
            g.set_memory_policy(bitmap_bytes=args.bitmap_bytes, list_entries=args.list_entries)
        info = g.info()
        pats = [agis.Pattern(*I.PATTERNS[n]) for n in names]
        opts = [agis.default_opts(mode=0, seed=1 + i, eps=0.0, max_trials=trials) for i in range(len(names))]
        out = torch.zeros(ntiles * agis.TILE_WORDS, dtype=torch.int64, device="cuda")

        def step(j, n_trials):
            """Step j: the whole path for pattern j mod P (a plain per-query launch)."""
            i = j % len(names)
            nt = (n_trials + agis.TILE - 1) // agis.TILE
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            ev[0].record(stream)
            g.preprocess(1, CMIN)                           # a1, a2 (Sec. 4.4)
            ev[1].record(stream)
            agis.prepare(g, pats[i], opts[i])               # a3, a4 (tables + prefix sums)
            ev[2].record(stream)
            agis.sample_device(g, pats[i], opts[i], 0, nt, out.data_ptr())   # a5..a10
            ev[3].record(stream)
            words = out[:nt * agis.TILE_WORDS].cpu().numpy().view(np.uint64)  # step result to host
            ev[4].record(stream)
            stream.synchronize()
            s = agis.tile_sums(words)
            return {"pattern": i, "trials": n_trials, "preprocess": ev[0].elapsed_time(ev[1]),
                    "tables": ev[1].elapsed_time(ev[2]), "sample": ev[2].elapsed_time(ev[3]),
                    "readback": ev[3].elapsed_time(ev[4]), "hits": int(s["hits"].sum()),
                    "sectors": int(s["sectors"].sum()), "streamed": int(s["streamed"].sum()),
                    "survey": int(s["survey"].sum()), "sum_x": float(s["sum_x"].sum()),
                    "sum_x2": float(s["sum_x2"].sum())}

        for j in range(args.warmup):
            step(j, warm_trials)
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
        for j in range(args.steps):
            recs.append(step(j, trials))
        e1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        barrier(world)
        launches = agis.kernel_launches() - launches0
        clk = clocks.stop()
        ms = e0.elapsed_time(e1) / args.steps
        ms = allreduce_max(ms, world)
        value = trials * world / (ms / 1000.0)
        t_timed_end = time.perf_counter()

        rand_gbs = random_access_gbs(agis, stream, local)

        # roofline of the sampler kernel (the dominant launch): algorithmic sectors
        # counted by the kernel itself / its own event time, per launch
        peak, peak_kind = measured_peaks()
        per_launch_ms = statistics.mean([r["sample"] for r in recs])
        alg_bytes = statistics.mean([r["sectors"] * 32 for r in recs])
        achieved = statistics.mean([r["sectors"] * 32 / (r["sample"] / 1000.0) for r in recs]) / 1e9
        dram = profile_traffic()
        traffic = None
        if dram and all(names[r["pattern"]] in dram for r in recs):
            traffic = statistics.mean([dram[names[r["pattern"]]] * r["trials"] for r in recs])
        # time bound of the byte mix: streamed sectors at the copy peak, the rest at
        # the random-sector rate; frac_time = that bound / the measured kernel time
        model = None
        if rand_gbs:
            bounds = [(r["streamed"] * 32 / (peak * 1e9) + (r["sectors"] - r["streamed"]) * 32 / (rand_gbs * 1e9),
                       r["sample"] / 1000.0) for r in recs]
            model = {"streamed_sectors_per_trial": statistics.mean([r["streamed"] / r["trials"] for r in recs]),
                     "random_sectors_per_trial": statistics.mean([(r["sectors"] - r["streamed"]) / r["trials"]
                                                                  for r in recs]),
                     "bound_ms_per_launch": 1000.0 * statistics.mean([b for b, _ in bounds]),
                     "frac_time": sum(b for b, _ in bounds) / sum(t for _, t in bounds)}
        phases = {k: statistics.mean([r[k] for r in recs]) for k in ("preprocess", "tables", "sample", "readback")}
        per_pattern = {}
        for i, n in enumerate(names):
            rs = [r for r in recs if r["pattern"] == i]
            if not rs:
                continue
            tr = sum(r["trials"] for r in rs)
            per_pattern[n] = {"steps": len(rs), "estimate": rs[-1]["sum_x"] / rs[-1]["trials"],
                              "hits": rs[-1]["hits"], "sample_ms": statistics.mean([r["sample"] for r in rs]),
                              "step_ms": statistics.mean([r["preprocess"] + r["tables"] + r["sample"] + r["readback"]
                                                          for r in rs]),
                              "samples_per_s": tr / (sum(r["sample"] for r in rs) / 1000.0),
                              "sectors_per_trial": sum(r["sectors"] for r in rs) / tr,
                              "streamed_sectors_per_trial": sum(r["streamed"] for r in rs) / tr,
                              "survey_sectors_per_trial": sum(r["survey"] for r in rs) / tr,
                              "algorithmic_gbs": sum(r["sectors"] * 32 for r in rs) /
                                                 (sum(r["sample"] for r in rs) / 1000.0) / 1e9,
                              "dram_bytes_per_trial": dram.get(n) if dram else None}
        survey_gbs = statistics.mean([r["survey"] * 32 / (r["sample"] / 1000.0) for r in recs]) / 1e9

        # ---- end to end through the C ABI from pinned host buffers: every step uploads
        # the graph, preprocesses it, builds the pattern's tables, runs the estimate call
        # (its per-tile sums come back to the host) and returns the result
        e2e = None
        if not args.no_e2e:
            n_e2e = args.e2e_steps or len(names)
            per_s = statistics.mean([r["preprocess"] + r["tables"] + r["sample"] + r["readback"] for r in recs]) / 1000
            if time.perf_counter() + n_e2e * per_s * 1.2 > deadline:
                n_e2e = max(0, int((deadline - time.perf_counter()) / (per_s * 1.2)))
            if n_e2e > 0:
                h_off = torch.from_numpy(off).pin_memory()
                h_cols = torch.from_numpy(cols).pin_memory()
                ho, hc = h_off.numpy(), h_cols.numpy()
                d2h, h2d = 0, 0
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for j in range(n_e2e):
                    i = j % len(names)
                    ge = agis.Graph(ctx, ho, hc, validate=False)
                    ge.preprocess(1, CMIN)
                    r = agis.estimate(ge, pats[i], opts[i])
                    ge.close()
                    h2d += ho.nbytes + hc.nbytes + ctypes.sizeof(agis.Opts)
                    d2h += ntiles * agis.TILE_WORDS * 8
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                e2e = {"value": n_e2e * trials / dt, "unit": "samples/s", "h2d_bytes_per_step": int(h2d / n_e2e),
                       "d2h_bytes_per_step": int(d2h / n_e2e), "steps": n_e2e, "s_per_step": dt / n_e2e}
            else:
                skipped["e2e"] = "deadline"

        tte = None
        if not args.no_tte:
            tte = time_to_1pct(agis, g, pats, names, args, deadline)

        batching = None
        if args.batch64:
            plan = plan_seconds(args)["batch64"]
            if time.perf_counter() + plan * 0.5 > deadline:
                skipped["batch64"] = "deadline"
            else:
                batching = batch64(agis, ctx, args.batch_scale, eps=args.batch_eps, chunk_log2=args.tte_chunk_log2,
                                   deadline=deadline)

        large = large_graph(agis, ctx, args.large_scale) if args.large else None
        serving = serving_configs(agis, ctx, args.serve_seconds) if args.serve else None
        abl = ablation(agis, g) if args.ablation else None
        conc = concentration_run(agis, g) if args.concentration else None
        dag = cliques_oriented(agis, g) if args.dag else None
        anch = anchor_vs_exact(agis, g, names + ["6-clique"]) if args.anchor else None

    cpu = None
    if pool is not None:
        if time.perf_counter() + 4 * args.cpu_seconds > deadline + 200:
            skipped["cpu_baseline"] = "deadline"
        else:
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
                   "step": f"the full {trials}-trial query of one pattern (step j: pattern j mod {len(names)}), "
                           f"preprocessing and tables included; warm-up steps at {warm_trials} trials",
                   "nv": info["nv"], "nnz": info["nnz"], "max_degree": info["max_degree"],
                   "trials_per_pattern": trials, "parallelism": f"replicas x{world}",
                   "l2": l2_note(off.nbytes + cols.nbytes),
                   "graph_generation_s": t_gen},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "sample_kernel",
                     "peak_kind": peak_kind, "per_launch_ms": per_launch_ms,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "survey_model_gbs": survey_gbs,
                     "random_access_gbs": rand_gbs,
                     "byte_mix_bound": model},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "phases_ms": phases,
        "per_pattern": per_pattern,
        "time_to_1pct": tte,
        "batch64": batching,
        "timing": {"timed_loop_s": t_timed_end - t_start, "total_s": time.perf_counter() - t_start,
                   "skipped": skipped},
    }
    if serving is not None:
        line["serving"] = serving
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
    if args.summarize_launches:
        for by in ("kernel", "nvtx"):
            rows = summarize_launches(args.summarize_launches, by)
            print(f"| {'kernel' if by == 'kernel' else 'NVTX range'} | launches | total ms | share |\n|---|---|---|---|")
            for k, n, ms, sh in rows:
                print(f"| `{k}` | {n} | {ms:.1f} | {100 * sh:.2f}% |")
            print()
        return
    if args.summarize_ncu:
        names = [n for n in args.patterns.split(",") if n]
        s = summarize_ncu(args.summarize_ncu, args.summary_out or TRAFFIC_SUMMARY, names, 1 << args.log2_trials,
                          args.ncu_command, workload_name(args, names))
        print(json.dumps(s["per_pattern"]))
        return
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
