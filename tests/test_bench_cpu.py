"""The benchmark's reference arm (the CPU oracle on the host cores) end to end on a
small graph: it runs without a GPU and prints one JSON line with the keys the
benchmark contract asks for, the same workload name as the GPU arm, and a
cpu_baseline that describes the run."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--scale", "10",
           "--log2-trials", "20", "--steps", "2", "--warmup", "3", "--cpu-seconds", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "samples/s"
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    names = bench.PATTERN_NAMES
    assert d["config"]["workload"] == bench.workload_name(argparse.Namespace(scale=10, log2_trials=20), names)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == bench.host_cores() and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "samples/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_twenty_step_command_fits_its_time_limit():
    """The 20-step command (--gpus 1 --steps 20 --warmup 5) at the stated floor rates:
    every leg's upper bound (capped queries run to their caps) sums to less than the
    deadline after which optional legs are skipped, and the deadline leaves room
    under an 1800 s limit for the CPU baseline and the JSON line."""
    sys.path.insert(0, ROOT)
    import bench
    args = bench.parse_args(["--gpus", "1", "--steps", "20", "--warmup", "5"])
    plan = bench.plan_seconds(args)
    assert args.log2_trials == 28 and args.scale == 22 and args.batch64
    assert plan["timed"] == 20 * 2 ** 28 / bench.RATE_FLOOR["bench"]
    assert sum(plan.values()) <= args.deadline_s, plan
    assert args.deadline_s + 200 < 1800
    # the default (no flags) run finishes within minutes
    d = bench.parse_args([])
    assert d.steps * 2 ** d.log2_trials / bench.RATE_FLOOR["bench"] <= 180


def test_ncu_summary_round_trip(tmp_path):
    """--summarize-ncu turns an ncu CSV of sampler launches into the JSON summary that
    the benchmark reads back (keyed by the sampler's source hash)."""
    sys.path.insert(0, ROOT)
    import bench
    hdr = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",' \
          '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = []
    for lid, (rd, wr, ns) in enumerate([(4.0, 1.0, 2.0), (2.0, 0.5, 1.0)]):
        for name, unit, val in (("dram__bytes_read.sum", "Gbyte", rd), ("dram__bytes_write.sum", "Gbyte", wr),
                                ("gpu__time_duration.sum", "msecond", ns)):
            rows.append(f'"{lid}","1","python","h","void agis::sample_kernel<0, 0>(...)","1","7","(256, 1, 1)",'
                        f'"(592, 1, 1)","0","10.3","Command line profiler metrics","{name}","{unit}","{val}"\n')
    csv_path = tmp_path / "dram.csv"
    csv_path.write_text("==PROF== noise\n" + hdr + "".join(rows))
    out = tmp_path / "summary.json"
    s = bench.summarize_ncu(str(csv_path), str(out), ["4-clique", "5-cycle"], 1 << 20, "ncu ...", "w")
    assert s["per_pattern"]["4-clique"]["dram_bytes_per_trial"] == 5e9 / (1 << 20)
    assert s["per_pattern"]["5-cycle"]["dram_gbs"] == 2.5e9 / 1e6
    got = bench.profile_traffic(str(out))
    assert got == {"4-clique": 5e9 / (1 << 20), "5-cycle": 2.5e9 / (1 << 20)}


def test_launch_list_summary(tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    hdr = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = ['"0","void agis::sample_kernel<0, 0>(GraphView)","gpu__time_duration.sum","msecond","3"\n',
            '"1","k_scan_apply(const unsigned long *)","gpu__time_duration.sum","usecond","500"\n',
            '"2","void agis::sample_kernel<0, 0>(GraphView)","gpu__time_duration.sum","msecond","0.5"\n']
    p = tmp_path / "l.csv"
    p.write_text(hdr + "".join(rows))
    got = bench.summarize_launches(str(p))
    assert [(k, n) for k, n, _, _ in got] == [("void agis::sample_kernel<0, 0>", 2), ("k_scan_apply", 1)]
    assert abs(got[0][2] - 3.5) < 1e-9 and abs(got[0][3] - 0.875) < 1e-9
    nv = tmp_path / "n.csv"
    nv.write_text('"ID","thread Domain:Push/Pop_Range:PL_Type","Kernel Name","Metric Name","Metric Unit",'
                  '"Metric Value"\n'
                  '"0","1 ""<default domain>:agis:load:none"" ","k1(int)","gpu__time_duration.sum","ns","2000000"\n'
                  '"1","1 ""<default domain>:agis:epoch:none"" ","k2(int)","gpu__time_duration.sum","ns","6000000"\n'
                  '"2","","k3(int)","gpu__time_duration.sum","ns","2000000"\n')
    got = bench.summarize_launches(str(nv), by="nvtx")
    assert [(k, n, round(ms, 6)) for k, n, ms, _ in got] == [("agis:epoch", 1, 6.0), ("agis:load", 1, 2.0),
                                                            ("(none)", 1, 2.0)]
