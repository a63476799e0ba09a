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
    assert d["impl"] == "reference" and d["same_config"] is True
    assert d["metric"] == "two-scale steps/s" and d["unit"] == "steps/s"
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
    # measured counters exist for the full-size timed workloads only, and only
    # counters of the current kernel revision are ever used
    for (wl, prec, tiling, coupling, rev), ctr in bench.MICRO_COUNTERS.items():
        assert wl in ("c2", "c3") and prec == "mixed" and coupling in ("elimination", "partitioned")
        assert 0 <= tiling < len(bench.KERNEL_NAMES) and ctr["dram_bytes"] > 1e8
        assert ctr["warp_insts_fixed"] > 1e6 and ctr["warp_insts_per_problem_iter"] > 100


def test_roofline_entry_without_counters_reports_null_traffic():
    """A kernel revision without an ncu capture gets traffic, dram_frac and the
    on-chip entry as null, never a stale number."""
    sys.path.insert(0, ROOT)
    import bench
    sp = {"micro_kernel_ms": 6.0, "micro_launches": 10, "dof_cg_iters": 10 * 4225 * 1089 * 25,
          "refine_sweeps": 10 * 4225, "tiling": 4, "macro_kernel_ms": 1.0, "inner_iters": 10 * 4225 * 25}
    r = bench.micro_roofline(None, "mixed", "elimination", sp, 1089, {"sm_mhz": 2070.0})
    assert r["traffic"] is None and r["dram_frac"] is None and "onchip" not in r
    old_rev = dict(sp)
    r2 = bench.micro_roofline("c2", "mixed", "elimination", old_rev, 1089, {"sm_mhz": 2070.0}, nsm=152)
    has = ("c2", "mixed", 4, "elimination", bench.KERNEL_REV) in bench.MICRO_COUNTERS
    assert (r2["traffic"] is not None) == has and ("onchip" in r2) == has
    if has:
        on = r2["onchip"]
        assert on["peak"] == 4 * 152 * 2070e6 and abs(on["frac"] - on["achieved"] / on["peak"]) < 1e-12
    assert r["frac"] == r["achieved"] / r["peak"] and r["frac_kind"].startswith("algorithmic")
