#!/usr/bin/env python
"""Benchmark of the two-scale micro-solve hot path on GB300.

Workload (default): 64x64 macro Q1 mesh -> 4225 micro problems, each a 32x32
Q1 mesh on the reference cell (1089 DoFs, 4.60M micro DoFs in total), bump
deformation a ~ U[0, 0.2] (seeded), D = I, kappa = 1, u0 = 1, v0 = 0,
dt = 0.005, relative tolerance 1e-8 (micro solves, FP64 residual),
coupling tolerance 1e-10.  One benchmark step = one implicit Euler step of
the coupled system: every coupling iteration solves all micro problems
(FP32 CG + FP64 refinement) and the macro problem.

Metric: micro DOF-CG-iterations per second (sum over micro problems of
DoFs x inner CG iterations, divided by the time of the timed steps), with the
two-scale steps/s beside it.  Under torchrun every rank advances its own
independent replica of the workload (weak scaling, no collective on the data
path); the value is the sum over ranks divided by the slowest rank's time.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# algorithmic bytes of the micro solve (streaming accounting, stencil stored):
# an FP32 PCG iteration moves 11 vector words + 5 stencil words per DoF,
# an FP64 iteration the same in 8-byte words; an FP64 refinement residual
# reads v, b and 5 stencil words and writes r (8 words of 8 bytes).
BYTES_PER_DOF_ITER = {"mixed": 64, "fp64": 128}
BYTES_PER_DOF_SWEEP = 64

KERNEL_NAMES = ["k_micro_solve<1>", "k_micro_solve<2>", "k_micro_solve<4>", "k_micro_solve<8>",
                "k_micro_strip<3>", "k_micro_strip<5>", "k_micro_strip<7>",
                "k_micro_strip_tall<9>", "k_micro_strip_tall<11>", "k_micro_strip_tall<13>",
                "direct band solve (three-field only)",
                "k_micro_cluster<5> x2", "k_micro_cluster<5> x4", "k_micro_cluster_tall<9> x4",
                "k_micro_cluster_tall<9> x8", "k_micro_warp<3>", "k_micro_warp<5>"]
# Source revision of the column-strip kernels that the ncu counters below were
# taken on.  A kernel change gets a new revision, so counters of an older
# kernel no longer match and read as null.
KERNEL_REV = "ff6"
# Per-launch ncu counters of the micro-solve kernel, taken with `bench.py
# --iteration-log 5 --tiling T` under ncu after a plain run of it: DRAM bytes
# (read + write) of a steady pipelined launch, and the executed warp
# instructions as a fixed part plus a part per micro-problem CG iteration (a
# least-squares line through the four steady launches, which it fits to the
# instruction), keyed by (workload, precision, tiling, coupling, revision).
# The 128x128/64x64 workload holds 19 GB on the device, beyond what a capture
# should hold, so its counters come from the same micro problems on 32x32
# macro cells (`--workload c3 --macro-cells 32`, 1089 problems, 1.1 GB of
# DRAM traffic a launch): every problem is solved by its own block from its
# own data, so the DRAM bytes and the fixed instructions scale with the
# number of problems (x 16641 / 1089) and the part per problem-iteration
# does not change.
C3_SCALE = 16641 / 1089
MICRO_COUNTERS = {
    ("c2", "mixed", 4, "elimination", "ff6"): {"dram_bytes": 1.0491e9, "warp_insts_fixed": 166.45e6,
                                               "warp_insts_per_problem_iter": 2222.0},
    ("c3", "mixed", 9, "elimination", "ff6"): {"dram_bytes": 1.135e9 * C3_SCALE, "warp_insts_fixed": 152.7e6 * C3_SCALE,
                                               "warp_insts_per_problem_iter": 7260.0,
                                               "captured_on": "32x32 macro cells (1089 problems), scaled x 16641/1089"},
}
# warp instructions one SM can issue per clock (four schedulers)
ISSUE_PER_SM_CLK = 4
def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "t1", "p43a", "p43b"],
                    help="t1: the stationary three-field system (manufactured solution, 128x128 / 64x64); "
                         "p43a / p43b: the two shapes of the paper's parallel benchmark (Sec. 4.3), 64x64 macro "
                         "with 8x8 micro cells and 8x8 macro with 64x64 micro cells, with the 64x64/32x32 "
                         "workload's data")
    ap.add_argument("--tiling-sweep", action="store_true",
                    help="also time every micro-solve variant that fits (steps/s per variant)")
    ap.add_argument("--fd-dirs", type=int, default=20, help="c5: finite-difference directions per family")
    ap.add_argument("--tiling", type=int, default=-1,
                    help="micro-kernel variant of the main timed problem (-1: the library's autotuner; a fixed "
                         "variant keeps a profiled run on the kernel the plain run chose)")
    ap.add_argument("--coupling", default="elimination", choices=["elimination", "partitioned"],
                    help="how each step reaches the coupled solution (the other way is timed beside it)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--macro-cells", type=int, default=None,
                    help="macro cells per side of a smaller case for profiling (c3 and t1; default: the full size)")
    ap.add_argument("--problems", type=int, default=32,
                    help="c4: the first N of the 32 problems (a smaller case for profiling)")
    ap.add_argument("--no-extras", action="store_true", help="skip fp64 comparison, e2e, cpu baseline")
    ap.add_argument("--iteration-log", type=int, default=0, metavar="N",
                    help="profiling aid: take N single steps of the workload (one micro-solve launch each after "
                         "the first, which also solves the pipeline's head) and print the inner CG iterations of "
                         "each, to pair with ncu's per-launch counters")
    return ap.parse_args()


def workload(name, seed=0, macro_cells=None):
    import workloads as W
    if name == "c2":
        return W.c2(seed=seed)
    if name == "p43a":   # fine macro mesh, coarse micro meshes: 4225 micro problems of 81 DoFs
        return W.c2(NM=64, Nm=8, seed=seed)
    if name == "p43b":   # coarse macro mesh, fine micro meshes: 81 micro problems of 4225 DoFs
        return W.c2(NM=8, Nm=64, seed=seed)
    return W.c3(seed=seed) if macro_cells is None else W.c3(NM=macro_cells, seed=seed)


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


COUPLING = {"elimination": 1, "partitioned": 0}


def make_problem(T, w, precision, stream, **opts):
    prec = T.TSF_MIXED if precision == "mixed" else T.TSF_FP64
    P = T.TwoScale(w.Nm, w.NM, bc=w.bc, precision=prec, stream=stream, cg_tol=w.tol, coupling_tol=w.coupling_tol,
                   **opts)
    P.set_physics(w.D, w.kappa, w.Du)
    P.set_deformation(w.family, w.params)
    P.set_state(w.u0, None)
    return P


def timed_steps(torch, P, w, steps, barrier):
    """device time (ms) of `steps` graph-launched steps on the current stream"""
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    P.step(w.dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1)


def other_coupling(torch, T, E, w, args, uP, vP, barrier, allmax, allsum, K, Wm):
    """The same steps with the other way of reaching the coupled solution."""
    E.step(w.dt, Wm)
    E.synchronize()
    E.reset_stats()
    msE = timed_steps(torch, E, w, K, barrier)
    E.synchronize()
    sE = E.stats()
    msE_max = allmax(msE)
    out = {
        "value": allsum(float(sE["dof_cg_iters"])) / (msE_max / 1e3), "unit": "DOF-iter/s",
        "ms_per_step": msE_max / K, "steps_per_s": int(os.environ.get("WORLD_SIZE", "1")) * K / (msE_max / 1e3),
        "inner_iters_per_solve": sE["inner_iters"] / max(sE["micro_solves"], 1),
        "coupling_iters_per_step": sE["coupling_iters_total"] / K,
        "rel_diff_vs_main": {"u": float(np.linalg.norm(E.u() - uP) / np.linalg.norm(uP)),
                             "v": float(np.linalg.norm(E.v() - vP) / np.linalg.norm(vP))},
    }
    E.close()
    return out


def rank_env():
    """(world, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_over_ranks(x, op, world, device="cpu"):
    """All-reduce one number over the ranks ("max" or "sum"); the identity at
    world size 1.  Every rank runs its own replica of the workload, so the
    only collectives are these two on the timing and the work counters."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_per_rank, ms_per_rank, world, device="cpu"):
    """Whole-job throughput: the units all ranks processed divided by the
    slowest rank's time; also returns (slowest ms, total units)."""
    ms_max = reduce_over_ranks(ms_per_rank, "max", world, device)
    total = reduce_over_ranks(units_per_rank, "sum", world, device)
    return total / (ms_max / 1e3), ms_max, total


def run_iteration_log(args):
    """One JSON line: the inner CG iterations (summed over the micro
    problems) of each of N single steps, in launch order.  The micro-solve
    launches of this run are: phi and psi (set-up), then per step one
    pipelined solve (the first step also the head solve)."""
    import torch
    import paper_2103_17040_gb300 as T
    torch.cuda.set_device(0)
    T.load_library()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    w = workload(args.workload, macro_cells=args.macro_cells)
    P = make_problem(T, w, args.precision, stream, coupling=COUPLING[args.coupling], tiling=args.tiling)
    rows, last = [], 0
    for _ in range(args.iteration_log):
        P.step(w.dt, 1)
        P.synchronize()
        st = P.stats()
        rows.append({"micro_solves": st["micro_solves"], "inner_iters": st["inner_iters"] - last,
                     "refine_sweeps": st["refine_sweeps"]})
        last = st["inner_iters"]
    print(json.dumps({"workload": args.workload, "tiling": P.stats()["tiling"], "steps": rows}))


def run_gb300(args):
    import torch
    import torch.distributed as dist
    import paper_2103_17040_gb300 as T

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    T.load_library()

    def barrier():
        if world > 1:
            dist.barrier()

    def allmax(x):
        return reduce_over_ranks(x, "max", world, "cuda")

    def allsum(x):
        return reduce_over_ranks(x, "sum", world, "cuda")

    # the library enqueues on this (non-default) torch stream, so torch's CUDA
    # events on it bracket exactly the library's work
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    w = workload(args.workload, seed=rank, macro_cells=args.macro_cells)
    nm, nM = w.nm, w.nM
    K, Wm = args.steps, args.warmup

    # ---- main timed region (graph-launched steps, inputs resident) ----
    other = "partitioned" if args.coupling == "elimination" else "elimination"
    P = make_problem(T, w, args.precision, stream, coupling=COUPLING[args.coupling], tiling=args.tiling)
    P.step(w.dt, Wm)
    P.synchronize()
    P.reset_stats()
    clk = Clocks(local)
    clk.start()
    ms = timed_steps(torch, P, w, K, barrier)
    clocks = clk.stop()
    P.synchronize()
    st = P.stats()
    dof_rate, ms_max, dof_iters = whole_job_rate(float(st["dof_cg_iters"]), ms, world, "cuda")
    steps_per_s = world * K / (ms_max / 1e3)
    # partitioned: 2 prologues + (micro, macro) per coupling iteration; pipelined elimination: start,
    # macro prologue, micro solve, macro solve (+ k_elim_pre with the one-block-per-problem variants),
    # and the commit of v in the last step of the call
    if args.coupling == "elimination":
        launches = (4 if st["tiling"] >= 4 else 5) * K + 1
    else:
        launches = 2 * K + 2 * st["coupling_iters_total"]

    line = {
        "metric": "two-scale steps/s",
        "value": steps_per_s,
        "unit": "steps/s",
        "n_gpus": world,
        "steps": K,
        "warmup": Wm,
        "ms_per_step": ms_max / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: macro {w.NM}x{w.NM} Q1 ({nM} micro problems), micro "
                               f"{w.Nm}x{w.Nm} Q1 ({nm} DoFs each, {nM * nm} micro DoFs), "
                               f"dt={w.dt}, tol={w.tol}, {args.precision}, coupling by {args.coupling}",
                   "macro_mesh": w.NM, "micro_mesh": w.Nm, "micro_dofs": nM * nm, "dt": w.dt, "tol": w.tol,
                   "coupling_tol": w.coupling_tol, "precision": args.precision, "coupling": args.coupling,
                   "replicas": world,
                   "l2": "working set > L2 (operators + vectors over 1 GB), no flush"},
        "dof_cg_iters_per_s": dof_rate,
        "coupling_iters_per_step": st["coupling_iters_total"] / K,
        "inner_iters_per_solve": st["inner_iters"] / max(st["micro_solves"], 1),
        "refine_sweeps_per_solve": st["refine_sweeps"] / max(st["micro_solves"], 1),
        "macro_iters_per_solve": st["macro_iters"] / max(st["coupling_iters_total"], 1),
        "tiling": st["tiling"],
        "gpu_launches": launches,
        "clocks": clocks,
    }

    # ---- every micro-solve variant that fits, timed on the same steps ----
    if args.tiling_sweep or args.workload in ("p43a", "p43b"):
        sweep = {}
        for t in [t for t in range(len(KERNEL_NAMES)) if t != 10]:
            try:
                Q = make_problem(T, w, args.precision, stream, coupling=COUPLING[args.coupling], tiling=t)
                Q.step(w.dt, Wm)
                Q.synchronize()
            except T.TsfError:
                continue   # does not fit this micro mesh / precision
            msq = timed_steps(torch, Q, w, K, lambda: None)
            sweep[KERNEL_NAMES[t]] = {"tiling": t, "ms_per_step": msq / K}
            Q.close()
        line["tiling_sweep"] = sweep
        line["tiling_sweep_note"] = "steps/s of the same workload with each variant fixed; the line's own value " \
                                    "uses the variant the library's autotuner picked (key tiling)"

    # ---- the same steps with the other way of reaching the coupled solution:
    # exact elimination (one micro solve per step) or the partitioned
    # iteration of the paper (micro and macro solves until u settles) ----
    uP, vP = P.u(), P.v()
    E = make_problem(T, w, args.precision, stream, coupling=COUPLING[other]) if not args.no_extras else None
    if E is not None:
        line[other] = other_coupling(torch, T, E, w, args, uP, vP, barrier, allmax, allsum, K, Wm)

    # ---- per-kernel timing of the micro solve (plain launches, CUDA events) ----
    opts = T.tsf_default_options()
    opts.precision = T.TSF_MIXED if args.precision == "mixed" else T.TSF_FP64
    opts.cg_tol, opts.coupling_tol = w.tol, w.coupling_tol
    opts.coupling = COUPLING[args.coupling]
    opts.use_graph, opts.profile = 0, 1
    opts.tiling = st["tiling"]
    opts.cuda_stream = stream.cuda_stream
    T.tsf_set_options(P.ctx, opts)
    P.reset_stats()
    P.step(w.dt, min(K, 10))
    P.synchronize()
    sp = P.stats()
    line["roofline"] = micro_roofline(args.workload if not args.macro_cells else None, args.precision, args.coupling,
                                      sp, nm, clocks)

    # ---- push-forward of the micro fields for visualisation (device buffer) ----
    xyv = torch.empty(nM * nm * 3, dtype=torch.float32, device="cuda")
    P.pushforward(0.8 / w.NM, xyv)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    pe0.record(stream)
    for _ in range(5):
        P.pushforward(0.8 / w.NM, xyv)
    pe1.record(stream)
    torch.cuda.synchronize()
    pf_ms = pe0.elapsed_time(pe1) / 5
    pf_gbs = 20.0 * nM * nm / (pf_ms / 1e3) / 1e9   # write (X1, X2, v) FP32, read v FP64: 20 B per micro DoF
    peak = line["roofline"]["peak"]
    line["pushforward"] = {"ms": pf_ms, "achieved_GBs": pf_gbs, "frac": pf_gbs / peak,
                           "note": "includes the getter's stream synchronisation"}
    del xyv
    P.close()

    if not args.no_extras and rank == 0:
        # ---- FP64 path at equal tolerance (comparison) ----
        if args.precision == "mixed":
            Q = make_problem(T, w, "fp64", stream, coupling=COUPLING[args.coupling])
            Q.step(w.dt, 2)
            Q.synchronize()
            Q.reset_stats()
            k64 = max(2, min(K, 10))
            ms64 = timed_steps(torch, Q, w, k64, lambda: None)
            s64 = Q.stats()
            line["fp64_path"] = {"value": k64 / (ms64 / 1e3), "unit": "steps/s",
                                 "dof_cg_iters_per_s": s64["dof_cg_iters"] / (ms64 / 1e3),
                                 "ms_per_step": ms64 / k64, "steps": k64,
                                 "speedup_mixed_vs_fp64_per_step": (ms64 / k64) / (ms_max / K)}
            Q.close()
        # ---- end to end through the public API with host buffers ----
        line["e2e"] = run_e2e(torch, T, w, args, stream, float(st["dof_cg_iters"]))
        # ---- CPU baseline: the oracle on this host's cores; errors against the tight oracle ----
        if world == 1:
            line["cpu_baseline"] = run_cpu_baseline(T, w, args, stream)
            line["error_vs_tight_oracle"] = run_tight_errors(T, w, args, stream)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def micro_roofline(workload_key, precision, coupling, sp, nm, clocks, nsm=None):
    """Roofline entry of the micro-solve kernel from its CUDA-event launch time
    (plain launches, profiled by the library) and, where an ncu capture of the
    same kernel revision exists, its measured DRAM bytes and instructions.

    * frac: algorithmic bytes (64 B per FP32 DoF-iteration of the inner CG and
      64 B per DoF and refinement sweep; 128 B per FP64 DoF-iteration) per
      launch / launch time / HBM peak.  The CG state stays on chip, so this is
      an algorithmic-equivalent rate that can exceed 1, not an HBM fraction.
    * dram_frac: the measured DRAM bytes per launch / launch time / HBM peak.
    * onchip: the issue-rate roofline -- executed warp instructions per launch
      over the time the SMs would need at four instructions per clock each --
      the bound of a kernel limited by instruction issue and latency rather
      than by memory."""
    micro_ms = sp["micro_kernel_ms"] / max(sp["micro_launches"], 1)
    bytes_launch = (BYTES_PER_DOF_ITER[precision] * sp["dof_cg_iters"] +
                    (BYTES_PER_DOF_SWEEP * sp["refine_sweeps"] * nm if precision == "mixed" else 0)) \
        / max(sp["micro_launches"], 1)
    achieved = bytes_launch / (micro_ms / 1e3) / 1e9
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    ctr = MICRO_COUNTERS.get((workload_key, precision, sp["tiling"], coupling, KERNEL_REV)) if workload_key else None
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "frac_kind": "algorithmic-equivalent (streaming accounting; the CG state stays on chip)",
           "traffic": ctr["dram_bytes"] if ctr else None,
           "dram_frac": (ctr["dram_bytes"] / (micro_ms / 1e3) / 1e9 / peak) if ctr else None,
           "kernel": KERNEL_NAMES[sp["tiling"]], "kernel_rev": KERNEL_REV, "bytes_per_launch": bytes_launch,
           "avg_launch_ms": micro_ms, "launches_timed": sp["micro_launches"],
           "macro_kernel_share": sp["macro_kernel_ms"] / max(sp["macro_kernel_ms"] + sp["micro_kernel_ms"], 1e-30),
           "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6800 GB/s"}
    if ctr:
        if nsm is None:
            import torch
            nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        mhz = clocks.get("sm_mhz") or (peaks or {}).get("sm_max_mhz") or 2070.0
        ipeak = ISSUE_PER_SM_CLK * nsm * mhz * 1e6
        insts = ctr["warp_insts_fixed"] + ctr["warp_insts_per_problem_iter"] * sp["inner_iters"] / max(
            sp["micro_launches"], 1)
        ach = insts / (micro_ms / 1e3)
        out["onchip"] = {"bound": "issue", "achieved": ach, "peak": ipeak, "unit": "warp-inst/s",
                         "frac": ach / ipeak, "warp_insts_per_launch": insts,
                         "note": f"{ISSUE_PER_SM_CLK} warp instructions per clock per SM at {mhz:.0f} MHz, "
                                 f"{nsm} SMs; instructions per launch from ncu (smsp__inst_executed.sum: fixed "
                                 f"part + part per micro-problem CG iteration) at this run's iteration count"}
    return out


def run_e2e(torch, T, w, args, stream, dof_iters_device):
    """End to end through the public API: every step uploads that step's
    input -- the macro source term (zero for this workload) -- from pinned
    host memory, takes one step and reads the macro field and the micro
    averages back into pinned host memory.  Each loop runs on a fresh problem
    over the same trajectory steps as the device-resident timing (the same
    warm-up, then the same number of steps), so the work per step is the same
    and ms per step compares directly.  The main loop uses the asynchronous
    getters (queued behind the step, one synchronisation at the end, checked
    against a synchronous read); beside it the same loop with synchronous
    reads after every step, and the loop that uploads the whole state (u, v)
    every step, which restarts the solver's history each step."""
    k, Wm = args.steps, args.warmup
    fu_h = torch.zeros(w.nM, dtype=torch.float64).pin_memory()
    u_out = torch.empty(w.nM, dtype=torch.float64).pin_memory()
    vbar_out = torch.empty(w.nM, dtype=torch.float64).pin_memory()
    fu_np, uo_np, vo_np = fu_h.numpy(), u_out.numpy(), vbar_out.numpy()

    def fresh():
        P = make_problem(T, w, args.precision, stream, coupling=COUPLING[args.coupling])
        P.step(w.dt, Wm)
        P.synchronize()
        return P

    def run(P, upload, reads):
        P.reset_stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            upload()
            P.step(w.dt, 1)
            reads(P)
        P.synchronize()
        return time.perf_counter() - t0, P.stats()

    def async_reads(P):
        P.u_async(uo_np)
        P.vbar_async(vo_np)

    def sync_reads(P):
        P.u(uo_np)
        P.vbar(vo_np)

    ips = lambda s: s["inner_iters"] / max(s["micro_solves"], 1)
    P = fresh()
    el, st = run(P, lambda: P.set_sources(fu=fu_np), async_reads)
    if not (np.array_equal(uo_np, P.u()) and np.array_equal(vo_np, P.vbar())):
        raise RuntimeError("asynchronous reads differ from the state")
    P.close()
    out = {"value": k / el, "unit": "steps/s", "steps": k, "warmup": Wm,
           "ms_per_step": 1e3 * el / k, "dof_cg_iters_per_s": st["dof_cg_iters"] / el,
           "h2d_bytes_per_step": 8 * w.nM, "d2h_bytes_per_step": 8 * 2 * w.nM,
           "inner_iters_per_solve": ips(st),
           "dof_iters_vs_device_loop": st["dof_cg_iters"] / max(dof_iters_device, 1.0),
           "inputs": "macro source term per step (pinned host -> device), macro field and averages back "
                     "(asynchronous getters into pinned memory, one synchronisation at the end)"}
    P = fresh()
    el1, st1 = run(P, lambda: P.set_sources(fu=fu_np), sync_reads)
    P.close()
    out["sync_reads"] = {"value": k / el1, "unit": "steps/s", "ms_per_step": 1e3 * el1 / k,
                         "inner_iters_per_solve": ips(st1),
                         "note": "the same loop, reading the results synchronously after every step"}
    P = fresh()
    u_h = torch.empty(w.nM, dtype=torch.float64).pin_memory()
    v_h = torch.empty(w.nM * w.nm, dtype=torch.float64).pin_memory()
    u_h.copy_(torch.from_numpy(P.u()))
    v_h.copy_(torch.from_numpy(P.v().ravel()))
    u_np, v_np = u_h.numpy(), v_h.numpy()
    el2, st2 = run(P, lambda: P.set_state(u_np, v_np), sync_reads)
    P.close()
    out["state_roundtrip"] = {"value": k / el2, "unit": "steps/s", "ms_per_step": 1e3 * el2 / k,
                              "inner_iters_per_solve": ips(st2),
                              "h2d_bytes_per_step": 8 * (w.nM + w.nM * w.nm), "d2h_bytes_per_step": 8 * 2 * w.nM}
    return out


def run_cpu_baseline(T, w, args, stream):
    """The FP64 oracle on the host cores for a bounded sample of the same
    workload: full-size steps from the initial state, at the benchmark
    tolerances, until the time budget is spent."""
    import oracle
    R = oracle.Problem(w.Nm, w.NM, w.bc, w.family, w.params, D=w.D, kappa=w.kappa, Du=w.Du)
    R.set_state(w.u0, None)
    t0 = time.perf_counter()
    n = 0
    while True:
        R.step(w.dt, 1, cg_tol=w.tol, coupling_tol=w.coupling_tol, macro_tol=1e-12)
        n += 1
        if time.perf_counter() - t0 > args.cpu_seconds or n >= 50:
            break
    el = time.perf_counter() - t0
    rs = R.stats()
    return {"value": n / el, "unit": "steps/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} full-size steps of the workload from u0=1, v0=0 (FP64, CSR Jacobi-PCG, partitioned "
                      f"coupling iteration, OpenMP over micro problems), {el:.1f} s",
            "dof_cg_iters_per_s": rs["inner_iters"] * w.nm / el}


def run_tight_errors(T, w, args, stream, nsteps=10):
    """Error of the GPU paths as benchmarked (mixed and FP64, the benchmark's
    tolerances and coupling) against the oracle solved tightly (relative
    residual 1e-13, coupling 1e-13), after nsteps full-size steps."""
    import oracle
    R = oracle.Problem(w.Nm, w.NM, w.bc, w.family, w.params, D=w.D, kappa=w.kappa, Du=w.Du)
    R.set_state(w.u0, None)
    t0 = time.perf_counter()
    R.step(w.dt, nsteps, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    el = time.perf_counter() - t0
    ru, rv = R.u, R.v
    out = {"steps": nsteps, "oracle": "FP64, relative residual 1e-13, coupling 1e-13", "oracle_s": el}
    for prec in ("mixed", "fp64"):
        P = make_problem(T, w, prec, stream, coupling=COUPLING[args.coupling])
        P.step(w.dt, nsteps)
        P.synchronize()
        u, v = P.u(), P.v()
        P.close()
        out[prec] = {"rel_l2_u": float(np.linalg.norm(u - ru) / np.linalg.norm(ru)),
                     "rel_l2_v": float(np.linalg.norm(v - rv) / np.linalg.norm(rv)),
                     "tol": w.tol, "coupling": args.coupling}
    return out


def run_reference(args):
    """The oracle, as it stands, on the host cores, on the same workload as the
    GPU arm (full size): the paper's partitioned coupling iteration (Sec. 3.3)
    with FP64 CSR micro problems and Jacobi-PCG, OpenMP over the micro
    problems, at the benchmark's tolerances; the same metric (steps/s)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload not in ("c2", "c3", "p43a", "p43b"):
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm (the oracle on the host cores) "
                          "is timed on the two-field time-stepping workloads"}))
        return
    import oracle
    w = workload(args.workload)
    R = oracle.Problem(w.Nm, w.NM, w.bc, w.family, w.params, D=w.D, kappa=w.kappa, Du=w.Du)
    R.set_state(w.u0, None)
    R.step(w.dt, args.warmup, cg_tol=w.tol, coupling_tol=w.coupling_tol, macro_tol=1e-12)
    R.reset_stats()
    t0 = time.perf_counter()
    R.step(w.dt, args.steps, cg_tol=w.tol, coupling_tol=w.coupling_tol, macro_tol=1e-12)
    el = time.perf_counter() - t0
    rs = R.stats()
    value = args.steps / el
    sample = f"{args.steps} full-size steps after {args.warmup} warm-up steps"
    line = {"metric": "two-scale steps/s", "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "same_config": True,
            "config": {"workload": f"{args.workload}: macro {w.NM}x{w.NM}, micro {w.Nm}x{w.Nm}, dt={w.dt}, "
                                   f"tol={w.tol}, FP64, partitioned coupling (coupling tol {w.coupling_tol})",
                       "precision": "fp64"},
            "dof_cg_iters_per_s": rs["inner_iters"] * w.nm / el,
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_c5(args):
    """Differentiation workload: the gradient of J = mean of u at the final time
    with respect to the per-node deformation parameters, after the 50-step FP64
    march of the 64x64 macro / 32x32 micro bump workload with checkpoints every
    10 steps (discrete adjoint on the GPU).  Timed at the workload's
    tolerances; then checked against Richardson-extrapolated central
    differences (h = 1e-2 and 5e-3) of the GPU forward march along seeded unit
    directions, both sides at tolerance 1e-14 with a fixed micro-solve
    variant, on the bump family and on the shear+bump family (64x64 / 32x32,
    D = diag(1, 0.1))."""
    import torch
    import paper_2103_17040_gb300 as T
    import workloads as W

    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    T.load_library()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    w = W.c5()
    ckpt = 10

    def ev_time(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, out

    # ---- timing at the workload's tolerances ----
    P = make_problem(T, w, "fp64", stream, coupling=COUPLING[args.coupling])
    P.step(w.dt, 2)
    P.set_state(w.u0, None)
    P.adjoint_mean_u(w.dt, 3, 2)
    P.set_state(w.u0, None)
    t_fwd, _ = ev_time(lambda: P.step(w.dt, w.nsteps))
    t_grad_l = []
    for _ in range(3):
        P.set_state(w.u0, None)
        t, (J, g) = ev_time(lambda: P.adjoint_mean_u(w.dt, w.nsteps, ckpt))
        t_grad_l.append(t)
    tiling = P.stats()["tiling"]
    P.close()

    x1, x2 = W.macro_coords(w.NM)
    mH = 0.25 * np.where((x1 == 0) | (x1 == 1), 1.0, 2.0) * np.where((x2 == 0) | (x2 == 1), 1.0, 2.0) / w.NM ** 2

    def fd_check(fam, prm, D, ndirs, seed):
        tight = dict(cg_tol=1e-14, coupling_tol=1e-14, macro_tol=1e-14, tiling=tiling, cg_maxit=20000,
                     coupling_maxit=100)
        Q = T.TwoScale(w.Nm, w.NM, bc=w.bc, precision=T.TSF_FP64, stream=stream, coupling=COUPLING[args.coupling],
                       **tight)
        Q.set_physics(D, w.kappa, w.Du)

        def J_at(p):
            Q.set_deformation(fam, p)
            Q.set_state(w.u0, None)
            Q.step(w.dt, w.nsteps)
            return float(np.dot(mH, Q.u()))

        Q.set_deformation(fam, prm)
        Q.set_state(w.u0, None)
        t0 = time.perf_counter()
        J0, g0 = Q.adjoint_mean_u(w.dt, w.nsteps, ckpt)
        t_adj = time.perf_counter() - t0
        # noise floor: change of J when the tolerances are loosened tenfold
        L = T.TwoScale(w.Nm, w.NM, bc=w.bc, precision=T.TSF_FP64, stream=stream, coupling=COUPLING[args.coupling],
                       **dict(tight, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13))
        L.set_physics(D, w.kappa, w.Du)
        L.set_deformation(fam, prm)
        L.set_state(w.u0, None)
        L.step(w.dt, w.nsteps)
        epsJ = abs(float(np.dot(mH, L.u())) - J0)
        L.close()
        # Richardson-extrapolated central difference: D(h) and D(h/2) have
        # the same h^2 truncation term, (4 D(h/2) - D(h)) / 3 cancels it
        h = 1e-2
        rows = []
        t0 = time.perf_counter()
        for k in range(ndirs):
            e = W.rng(1000 + seed + k).standard_normal(prm.shape)
            e /= np.linalg.norm(e)
            d1 = (J_at(prm + h * e) - J_at(prm - h * e)) / (2 * h)
            d2 = (J_at(prm + 0.5 * h * e) - J_at(prm - 0.5 * h * e)) / h
            fd = (4.0 * d2 - d1) / 3.0
            ad = float(np.sum(g0 * e))
            rows.append((ad, fd))
        t_fd = time.perf_counter() - t0
        Q.close()
        ad = np.array([r[0] for r in rows])
        fd = np.array([r[1] for r in rows])
        rel = np.abs(fd - ad) / np.abs(ad)
        return {"family": fam, "directions": ndirs, "h": h,
                "method": "Richardson-extrapolated central difference (4 D(h/2) - D(h)) / 3, truncation O(h^4)",
                "J": J0, "grad_norm": float(np.linalg.norm(g0)),
                "median_abs_directional": float(np.median(np.abs(ad))),
                "rel_err_max": float(rel.max()), "rel_err_median": float(np.median(rel)),
                "abs_err_max": float(np.abs(fd - ad).max()),
                "noise_floor_abs": epsJ / h, "J_change_tol_1e-13_vs_1e-14": epsJ,
                "adjoint_s": t_adj, "fd_s": t_fd,
                "per_direction": [[float(a), float(b)] for a, b in rows]}

    bump = fd_check(W.FAMILY_BUMP, w.params, w.D, args.fd_dirs, 0)
    w3 = W.c3(NM=w.NM, Nm=w.Nm)
    shear = fd_check(w3.family, w3.params, w3.D, args.fd_dirs, 500)
    t_grad = statistics.median(t_grad_l)
    line = {"metric": "gradient wall time (dJ/da, 4225 parameters)", "value": t_grad, "unit": "s",
            "n_gpus": 1, "steps": w.nsteps, "warmup": 1, "higher_is_better": False, "dtype": "f64",
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": f"c5: macro {w.NM}x{w.NM} ({w.nM} micro problems), micro {w.Nm}x{w.Nm}, "
                                   f"bump a ~ U[0,0.2], FP64, dt={w.dt} x {w.nsteps} steps, checkpoints every "
                                   f"{ckpt}, tol {w.tol}, coupling tol {w.coupling_tol}, coupling by {args.coupling}"},
            "forward_s": t_fwd, "gradient_over_forward": t_grad / t_fwd, "J": J, "grad_norm": float(np.linalg.norm(g)),
            "tiling": tiling, "fd_check": {"bump": bump, "shear_bump": shear}}
    print(json.dumps(line))


def run_c4(args):
    """32 independent two-scale problems of uneven sizes (macro 16..96 cells,
    micro 16..48 cells per side, 200M micro DoFs in all), mixed precision,
    each with its autotuned micro-solve variant; one batch step is one CUDA
    graph launch with one branch per problem (the library's default batch
    mode).  Beside it, over the same steps: the persistent batch mode (the
    micro solves of all problems in work-queue launches, one per class of micro mesh, eliminated
    coupling only) and the same problems stepped one after another (each
    problem through all the steps, its own step graph)."""
    import torch
    import paper_2103_17040_gb300 as T
    import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    T.load_library()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ws = W.c4(seed=rank)[:max(1, args.problems)]
    dt = ws[0].dt
    K, Wm = args.steps, args.warmup

    def build(persistent=False):
        B = T.TwoScaleBatch([(w.Nm, w.NM, w.bc) for w in ws], precision=T.TSF_MIXED, stream=stream,
                            cg_tol=ws[0].tol, coupling_tol=ws[0].coupling_tol, coupling=COUPLING[args.coupling],
                            persistent=persistent)
        for k, w in enumerate(ws):
            B[k].set_physics(w.D, w.kappa, w.Du)
            B[k].set_deformation(w.family, w.params)
            B[k].set_state(w.u0, None)
        return B

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    B = build()
    B.step(dt, Wm)
    B.synchronize()
    B.reset_stats()
    barrier = (lambda: torch.distributed.barrier()) if world > 1 else (lambda: None)
    clk = Clocks(local)
    clk.start()
    barrier()
    ms = timed(lambda: B.step(dt, K))
    barrier()
    clocks = clk.stop()
    B.synchronize()
    st = B.stats()
    tilings = [B[k].stats()["tiling"] for k in range(len(ws))]
    if world > 1:
        t = torch.tensor([ms, float(st["dof_cg_iters"])], dtype=torch.float64, device="cuda")
        mx = t.clone()
        torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
        ms_max, dof_iters = float(mx[0]), float(t[1])
    else:
        ms_max, dof_iters = ms, float(st["dof_cg_iters"])

    # the persistent mode over the same steps (micro solves of every problem
    # in work-queue launches beside one macro branch per problem)
    persistent = None
    if args.coupling == "elimination":
        B3 = build(persistent=True)
        B3.step(dt, Wm)
        B3.synchronize()
        B3.reset_stats()
        pm = timed(lambda: B3.step(dt, K))
        nq = B3.persistent_launches()  # micro-solve launches a step, one per class of micro mesh
        persistent = {"ms_per_step": pm / K, "dof_cg_iters_per_step": B3.stats()["dof_cg_iters"] / K,
                      "tilings": [B3[k].stats()["tiling"] for k in range(len(ws))], "micro_launches_per_step": nq,
                      "gpu_launches": (3 * len(ws) + nq) * K + len(ws)}
        B3.close()

    # the same problems one after another: a second, identical batch whose
    # problems are stepped through the same step range one problem at a time,
    # each with its own step graph (the solves get cheaper as the march
    # settles, so both are timed over the same steps)
    B2 = build()
    for k in range(len(ws)):
        B2[k].step(dt, Wm)
    torch.cuda.synchronize()
    for k in range(len(ws)):
        B2[k].reset_stats()

    def seq():
        for k in range(len(ws)):
            B2[k].step(dt, K)
    seq_ms = timed(seq)
    seq_iters = sum(B2[k].stats()["dof_cg_iters"] for k in range(len(ws)))
    B2.close()
    if persistent is not None:
        persistent["speedup_vs_sequential"] = (seq_ms / K) / persistent["ms_per_step"]
    ks = K

    # per-kernel timing of the micro solves (plain launches, one problem at a time)
    bytes_total, micro_ms, launches = 0.0, 0.0, 0
    for k, w in enumerate(ws):
        P = B[k]
        o = T.tsf_default_options()
        o.precision, o.cg_tol, o.coupling_tol = T.TSF_MIXED, w.tol, w.coupling_tol
        o.coupling = COUPLING[args.coupling]
        o.use_graph, o.profile, o.tiling = 0, 1, tilings[k]
        o.cuda_stream = stream.cuda_stream
        T.tsf_set_options(P.ctx, o)
        P.reset_stats()
        P.step(dt, 2)
        P.synchronize()
        sp = P.stats()
        bytes_total += BYTES_PER_DOF_ITER["mixed"] * sp["dof_cg_iters"] + BYTES_PER_DOF_SWEEP * sp["refine_sweeps"] * w.nm
        micro_ms += sp["micro_kernel_ms"]
        launches += sp["micro_launches"]
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = bytes_total / (micro_ms / 1e3) / 1e9
    B.close()
    ndof = sum(w.nM * w.nm for w in ws)
    line = {
        "metric": "micro DOF-CG-iters/s", "value": dof_iters / (ms_max / 1e3), "unit": "DOF-iter/s",
        "n_gpus": world, "steps": K, "warmup": Wm, "ms_per_step": ms_max / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"c4: {len(ws)} independent two-scale problems, macro 16..96 / micro 16..48 cells "
                               f"per side, {ndof} micro DoFs, dt={dt}, tol={ws[0].tol}, mixed, coupling by "
                               f"{args.coupling}, one graph per batch step with one branch per problem",
                   "problems": len(ws), "micro_dofs": ndof, "batch_mode": "branches",
                   "l2": "working set > L2, no flush"},
        "persistent": persistent,
        "batch_steps_per_s": world * K / (ms_max / 1e3),
        "sequential_ms_per_step": seq_ms / ks, "batch_speedup_vs_sequential": (seq_ms / ks) / (ms / K),
        "sequential_dof_cg_iters_per_step": seq_iters / ks, "batch_dof_cg_iters_per_step": st["dof_cg_iters"] / K,
        "coupling_iters_per_problem_step": st["coupling_iters_total"] / (K * len(ws)),
        "tilings": tilings, "coupling": args.coupling,
        "gpu_launches": ((4 * K + 1) * len(ws) if args.coupling == "elimination"
                         else 2 * K * len(ws) + 2 * st["coupling_iters_total"]),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "frac_kind": "algorithmic-equivalent (streaming accounting; the CG state stays on chip)",
                     "traffic": None, "dram_frac": None,
                     "kernel": "micro solves (each problem's autotuned variant, plain launches one problem at a time)",
                     "launches_timed": launches,
                     "avg_launch_ms": micro_ms / max(launches, 1),
                     "bytes_per_launch": bytes_total / max(launches, 1),
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6800 GB/s"},
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_c1(args):
    """The manufactured-solution workload: 8x8 macro (Dirichlet) / 8x8 micro,
    bump a = 0.1 x1, manufactured sources uploaded every step, dt = 0.01 x 10
    steps, tolerance 1e-12, FP64 and mixed.  Times the whole march through the
    public API (source upload per step included); errors against the
    manufactured solution at the nodes, and (oracle leg) against the oracle."""
    import torch
    import paper_2103_17040_gb300 as T
    import workloads as W
    from workloads import mms

    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    T.load_library()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    w = W.c1()
    a = w.params[:, 0]
    data = [mms.nodal_data(w.NM, w.Nm, a, n * w.dt) for n in range(w.nsteps + 1)]

    def march(prec):
        P = T.TwoScale(w.Nm, w.NM, bc=1, precision=prec, stream=stream, cg_tol=w.tol, coupling_tol=w.coupling_tol,
                       macro_tol=1e-13)
        P.set_deformation(w.family, w.params)
        best = None
        for rep in range(max(3, args.warmup) + 1):
            P.set_state(data[0]["u"], data[0]["v"].ravel())
            P.reset_stats()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for n in range(w.nsteps):
                d = data[n + 1]
                P.set_sources(fv=d["fv"].ravel(), g=d["g"].ravel(), fu=d["fu"], ud=d["ud"])
                P.step(w.dt, 1)
            P.synchronize()
            el = time.perf_counter() - t0
            if rep >= 1:  # the first march captures graphs and tunes
                best = el if best is None else min(best, el)
        st = P.stats()
        u, v = P.u(), P.v()
        P.close()
        ex = data[-1]
        return {"steps_per_s": w.nsteps / best, "ms_per_step": 1e3 * best / w.nsteps,
                "dof_cg_iters_per_s": st["dof_cg_iters"] / best,
                "max_nodal_error_u": float(np.max(np.abs(u - ex["u"]))),
                "max_nodal_error_v": float(np.max(np.abs(v - ex["v"])))}, u, v

    r64, u64, v64 = march(T.TSF_FP64)
    rmx, _, _ = march(T.TSF_MIXED)
    line = {"metric": "two-scale steps/s", "value": r64["steps_per_s"], "unit": "steps/s", "n_gpus": 1,
            "steps": w.nsteps, "warmup": max(3, args.warmup), "ms_per_step": r64["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "c1: macro 8x8 (Dirichlet, manufactured data), micro 8x8, bump a = 0.1 x1, "
                                   "dt = 0.01 x 10 steps, tol 1e-12, FP64; sources uploaded every step"},
            "fp64": r64, "mixed": rmx,
            "note": "81 micro problems of 81 DoFs: launch- and latency-bound, no roofline"}
    if not args.no_extras:
        import oracle
        R = oracle.Problem(w.Nm, w.NM, 1, w.family, w.params)
        t0 = time.perf_counter()
        R.set_state(data[0]["u"], data[0]["v"].ravel())
        for n in range(w.nsteps):
            d = data[n + 1]
            R.set_sources(fv=d["fv"].ravel(), g=d["g"].ravel(), fu=d["fu"], ud=d["ud"])
            R.step(w.dt, 1, cg_tol=w.tol, coupling_tol=w.coupling_tol, macro_tol=1e-13)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": w.nsteps / el, "unit": "steps/s", "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": "the whole 10-step march"}
        line["error_vs_oracle"] = {"rel_l2_u": float(np.linalg.norm(u64 - R.u) / np.linalg.norm(R.u)),
                                   "rel_l2_v": float(np.linalg.norm(v64 - R.v) / np.linalg.norm(R.v))}
    print(json.dumps(line))


def run_t1(args):
    """The stationary three-field system (u, v, w; Eq. (5)) on the manufactured
    solution of Eqs. (18)-(19): Omega = Z = [-1,1]^2, 128 x 128 macro cells
    (16641 nodes, the largest macro mesh of Table 1), 64 x 64 micro cells
    (4225 DoFs each, 70.3 M micro DoFs), mixed precision, tolerance 1e-10.
    Times (i) the complete solve: geometry, the three micro solves (v0, phi_I,
    phi_O; direct: the band factorisation and the refinement sweeps), the
    coupled macro solve and the commit; (ii) a re-solve for new sources,
    which re-uses phi_I, phi_O and the factor (one right-hand side).  The
    default micro solve is the direct banded Cholesky one; the fastest
    iterative variant (tall strips) is timed beside it.  Nodal errors against
    the manufactured solution; CPU baseline: the oracle's monolithic sparse
    solve of the same problem at 16 x 16 / 16 x 16."""
    import torch
    import paper_2103_17040_gb300 as T
    from workloads import three_field as T3

    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    T.load_library()
    stream = torch.cuda.Stream()
    NM, Nm = args.macro_cells or 128, 64
    wl = T3.manufactured(NM, Nm, Dv=1.0, Dw=0.5, kappa=(0.5, 1.0, 0.25, 1.0), tol=1e-10)
    K = max(3, min(args.steps, 10))
    dofs = wl.nM * wl.nm

    def measure(tiling):
        P = T.ThreeField(Nm, NM, x0=wl.x0, L=wl.L, dir_mask=wl.dir_mask, precision=T.TSF_MIXED, stream=stream,
                         cg_tol=wl.tol, macro_tol=1e-12, tiling=tiling)
        P.set_physics(wl.D, wl.Dw, wl.kappa)
        P.set_deformation(wl.family, wl.params)
        P.set_sources(**wl.sources())
        P.solve()                               # allocates, tunes
        full, resolve = [], []
        for rep in range(K):
            P.set_physics(wl.D, wl.Dw, wl.kappa)    # forces geometry, factor and the phi solves again
            s0 = P.stats()
            t0 = time.perf_counter()
            P.solve()
            full.append((time.perf_counter() - t0, P.stats(), s0))
            t0 = time.perf_counter()
            P.solve()                               # same sources: phi (and the factor) re-used
            resolve.append((time.perf_counter() - t0, P.stats()))
        u, w, v, _ = P.fields()
        P.close()
        med = lambda xs: statistics.median(xs)
        st = full[-1][1]
        r = {"tiling": st["tiling"], "complete_solve_ms": 1e3 * med(x[0] for x in full),
             "resolve_ms": 1e3 * med(x[0] for x in resolve),
             "device_ms": {"micro_3_solves": med(x[1]["micro_ms"] for x in full),
                           "macro": med(x[1]["macro_ms"] for x in full),
                           "total": med(x[1]["total_ms"] for x in full),
                           "resolve_micro": med(x[1]["micro_ms"] for x in resolve),
                           "resolve_total": med(x[1]["total_ms"] for x in resolve)},
             "refine_sweeps_per_problem": (st["refine_sweeps"] - full[-1][2]["refine_sweeps"]) / wl.nM,
             "fields": (u, w, v)}
        if st["tiling"] == T.TSF3_TILING_DIRECT:
            r["device_ms"]["factor"] = med(x[1]["factor_ms"] for x in full)
            r["device_ms"]["band_solves"] = med(x[1]["band_solve_ms"] for x in full)
            r["band_launches"] = st["band_launches"]
            r["band_solve_ms_per_launch"] = {
                "3_rhs": med(x[1]["band_solve_ms"] / x[1]["band_launches"] for x in full),
                "1_rhs": med(x[1]["band_solve_ms"] / x[1]["band_launches"] for x in resolve)}
        else:
            iters = st["dof_cg_iters"] - full[-1][2]["dof_cg_iters"]
            r["micro_dof_cg_iters_per_s"] = iters / (r["device_ms"]["micro_3_solves"] * 1e-3)
        return r

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    d = measure(-1)
    ck = clocks.stop()
    u, w, v = d.pop("fields")
    ue, we, ve = T3.mms_exact(NM, Nm)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    # k_band_solve, algorithmic bytes per launch: the factor twice (forward and
    # backward substitution, nm (Nm+3) FP32 values a problem), and per DoF and
    # right-hand side: r (8 B), y written and read (4 + 4 B), x updated (16 B)
    B = Nm + 3
    bytes_3 = wl.nM * wl.nm * (2 * B * 4 + 3 * 32)
    ms3 = d["band_solve_ms_per_launch"]["3_rhs"]
    achieved = bytes_3 / (ms3 * 1e-3) / 1e9
    line = {"metric": "micro DoFs solved/s (stationary three-field solve)", "value": dofs / (1e-3 * d["complete_solve_ms"]),
            "unit": "DoF/s", "n_gpus": 1, "steps": K, "warmup": 1, "ms_per_step": d["complete_solve_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"t1: manufactured three-field problem of Eqs. (18)-(19), macro {NM}x{NM} on "
                                   "[-1,1]^2 (Dirichlet u), micro 64x64, mixed, tol 1e-10; direct micro solves; "
                                   "inputs larger than L2"},
            **d,
            "roofline": {"bound": "hbm", "kernel": "k_band_solve<3>", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": None},
            "max_nodal_error": {"u": float(np.abs(u - ue).max()), "w": float(np.abs(w - we).max()),
                                "v": float(np.abs(v - ve).max())},
            "clocks": ck,
            # complete solve: expand, geometry, set-up, factor, sweeps x (solve, residual), moments, macro,
            # commit, vbar; re-solve: set-up, sweeps x (solve, residual), moments, macro, commit, vbar
            "gpu_launches": K * (8 + 2 * d["band_launches"] + 5 + 2 * d["band_launches"])}
    if not args.no_extras:
        it = measure(9)
        it.pop("fields")
        line["iterative"] = it
        from oracle.three_field import ThreeField
        s = T3.manufactured(16, 16, Dv=1.0, Dw=0.5, kappa=(0.5, 1.0, 0.25, 1.0))
        t0 = time.perf_counter()
        R = ThreeField(s.Nm, s.NM, s.family, s.params, D=s.D, Dw=s.Dw, kappa=s.kappa, x0=s.x0, L=s.L,
                       dir_mask=s.dir_mask)
        R.solve(**s.sources())
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": s.nM * s.nm / el, "unit": "DoF/s", "cores": 1, "kind": "oracle",
                                "sample": "monolithic sparse LU of the same problem at 16x16 / 16x16 "
                                          "(83521 micro DoFs), assembly included"}
    print(json.dumps(line))


def main():
    args = parse()
    if args.iteration_log:
        run_iteration_log(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "t1":
        run_t1(args)
    elif args.workload == "c1":
        run_c1(args)
    elif args.workload == "c4":
        run_c4(args)
    elif args.workload == "c5":
        run_c5(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
