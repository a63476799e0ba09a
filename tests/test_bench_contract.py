"""The benchmark's CPU-side contract: the reference arm (the oracle on the host
cores) prints one JSON line with the fields the line format needs, workloads
without a timed reference arm say so, and the smaller profiling cases keep
the micro problems of the full workload.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_prints_one_line():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "1")
    assert d["impl"] == "reference"
    assert d["metric"] == "micro DOF-CG-iters/s" and d["unit"] == "DOF-iter/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_of_an_untimed_workload_says_so():
    d = _run("--impl", "reference", "--workload", "t1", "--steps", "1", "--warmup", "1")
    assert d["impl"] == "reference" and "unavailable" in d


def test_profiling_case_keeps_the_micro_problems():
    sys.path.insert(0, ROOT)
    import bench
    full, small = bench.workload("c3"), bench.workload("c3", macro_cells=8)
    assert (full.NM, small.NM) == (128, 8)
    assert small.Nm == full.Nm and small.family == full.family and small.D == full.D
    assert small.dt == full.dt and small.tol == full.tol
    # measured DRAM bytes per launch exist for the full-size timed workloads only
    for (wl, prec, short_strip, coupling), traffic in bench.MICRO_TRAFFIC.items():
        assert wl in ("c2", "c3") and prec == "mixed" and coupling in ("elimination", "partitioned")
        assert traffic > 1e8
