#!/usr/bin/env python3
"""Benchmark of the heat + CG hot path on GB300.

One step = one pass of the whole path over one batch of synthetic input:
  heat: upload u0 (512^3 interior, 8 sine modes + 1e-3 noise), 1000 FTCS steps
        at r = 0.15 in FP64 (Boundary + Interior kernels, pointer swap), read back;
  CG:   solve the 256^3 7-point Dirichlet Laplacian system, b ~ N(0,1),
        rtol 1e-8, FP64, once matrix-free and once with the CSR int32 matrix.
``value`` is heat GLUP/s over the heat segment of the timed steps (device time
from CUDA events on the launching stream); CG iterations/s and p50/p99 solve
latencies are reported beside it.  All inputs are larger than L2 (129 MB).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU
(independent replicas: the path has no exchange step on one box), the timed
region is bracketed by barriers, and the slowest rank's time is used.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUP/s & % of HBM peak (heat 512³ FP64/FP32); CG it/s; p50/p99 solve latency"
SEED = 20261202
FP64_INSTR_PER_LUP = 7          # 5 DADD + 2 DFMA in the Interior kernel
BYTES_PER_LUP_F64 = 16          # read u once, write u' once
# FP64 issue peak derived from the nominal 1.25 TFLOP/s (FMA = 2 flops): 0.625e12 instr/s
FP64_INSTR_PEAK_T = 0.625

# heat arithmetic modes: Heat() keywords, the arithmetic type, algorithmic bytes per LUP,
# and the roof that binds the Interior kernel
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e nominal bandwidth (the measured copy rate is the roofline peak)
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel, from one ncu capture of the kernel as it stands, keyed by
# (arithmetic, grid edge, steps per launch): the FP64 exact-sum Interior kernel
# (two rows per thread, one point in four converted on the FP64 pipe) on 512^3
# read 1187.2 MB and wrote 1025.9 MB per launch (mean of 2 launches); the FP32
# blocked kernel at depth 2 (34-thread rows, plane loop unrolled by three) on
# 512^3 read 626.5 MB and wrote 494.2 MB per pass (mean of 2 passes); the FIXED64
# streaming kernel (plane loop unrolled by three) on 512^3 read 1149.5 MB and
# wrote 1025.9 MB per launch (mean of 2 launches).
# Re-capture after any change to that kernel; sizes not listed report null.
KERNEL_TRAFFIC_BYTES = {("f64", 512, 1): 2213105024, ("f32", 512, 2): 1120694016,
                        ("fixed64", 512, 1): 2175355904}
HEAT_MODES = {
    # plain FP64 handle: FP64 fields, exact int64 neighbour sum, one FP64 FMA per point
    "f64": {"dtype": "f64", "flags": "", "arith": "f64", "bytes": 16, "bound": "hbm",
            "desc": "FP64 fields; exact 64-bit fixed-point neighbour sum, one FP64 FMA per point"},
    # every operation on the FP64 pipe (5 DADD + 2 DFMA per point)
    "f64pipe": {"dtype": "f64", "flags": "HS_FP64_PIPE", "arith": "f64", "bytes": 16, "bound": "alu",
                "desc": "FP64 fields; 5 DADD + 2 DFMA per point on the FP64 pipe"},
    "fixed64": {"dtype": "f64", "flags": "HS_FIXED64", "arith": "int64", "bytes": 16, "bound": "hbm",
                "desc": "int64 fixed-point fields (FP64 interface), one rounding per point"},
    "f32": {"dtype": "f32", "flags": "", "arith": "f32", "bytes": 8, "bound": "hbm",
            "desc": "FP32 fields and arithmetic"},
}


# Algorithmic bytes of the other rows (read each input once, write each output once):
#  * batched heat: 16 B per lattice-point update of an FP64 grid, 8 B of an FP32 grid;
#  * the paper's variable-coefficient update: u, kappa and dt f read, u' written --
#    32 B (FP64) / 16 B (FP32) per update; the FP64 form is bound by the FP64 pipe
#    at 23 operations per update (per axis 4 additions, a multiply and an FMA for
#    the face differences; 5 to add dt f and the three scaled differences);
#  * CG per unknown and iteration: SpMV 16 B (read p, write q), x/r update 48 B
#    (read x, p, r, q; write x, r), p update 24 B (read r, p; write p) = 88 B
#    matrix-free; CSR adds 12 B per stored entry and 4 B of row pointer per row;
#  * mixed-precision CG per inner iteration and unknown: matrix-free (nx a multiple
#    of 4), the p update folded into the SpMV 16 B (read r, p; write p', q) and the
#    update 24 B = 40 B; CSR: SpMV 8 B + 8 B per entry and 4 B per row, update 24 B,
#    p update 12 B; per refinement:
#    FP64 SpMV 16 B (+ 12 B per entry, 4 B per row for CSR), residual 36 B
#    (read b, A x; write r in FP64 and r, p, d in FP32), correction 20 B.
VK_FP64_OPS_PER_LUP = 2    # FP64 variable-kappa update, exact-sum form: u + dt f, then one FMA
CG_BYTES_PER_ROW = 88
MIXED_INNER_BYTES_PER_ROW = {"matrix_free": 40, "csr": 44}
MIXED_REFINE_BYTES_PER_ROW = 72


def hbm_roofline(kernel, bytes_moved, ms, hbm_gbs, peak_kind, traffic=None, **extra):
    """Roofline object of an HBM-bound measurement: algorithmic bytes moved in
    `ms` milliseconds against the measured copy rate."""
    ach = bytes_moved / (ms * 1e-3) / 1e9
    out = {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": hbm_gbs, "unit": "GB/s",
           "frac": ach / hbm_gbs, "traffic": traffic, "peak_kind": peak_kind,
           "frac_of_nominal": ach / NOMINAL_HBM_GBS, "algorithmic_bytes": bytes_moved}
    out.update(extra)
    return out


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--heat-n", type=int, default=512)
    ap.add_argument("--heat-steps", type=int, default=1000)
    ap.add_argument("--r", type=float, default=0.15)
    ap.add_argument("--cg-n", type=int, default=256)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--heat-mode", choices=sorted(HEAT_MODES), default="f64",
                    help="arithmetic of the timed heat segment")
    ap.add_argument("--workload", choices=["default", "precision", "serving"], default="default",
                    help="default: the timed heat + CG step; precision: the 1024^3 FP32 heat "
                         "and 512^3 mixed-precision CG comparison; serving: the continuous-"
                         "batching request stream (these two: one run, no timing contract)")
    ap.add_argument("--requests", type=int, default=2000, help="serving: requests in the trace")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving workload in the default run")
    ap.add_argument("--tdepth", type=int, default=0,
                    help="steps per pass of the timed heat handle (0: library choice)")
    ap.add_argument("--paper-n", type=int, default=510,
                    help="paper side: interior points per axis (510 = the paper's N = 512)")
    ap.add_argument("--paper-steps", type=int, default=500, help="paper side: steps")
    ap.add_argument("--no-side", action="store_true",
                    help="skip every side measurement (same as --sides none)")
    ap.add_argument("--sides", default="all",
                    help="comma list of side measurements after the timed steps: modes, batching, "
                         "paper, mixed, precision, serving; 'all' or 'none'")
    return ap.parse_args()


SIDES = ("modes", "batching", "paper", "mixed", "precision", "serving")


def sides_of(args) -> set:
    """The side measurements to run after the timed steps."""
    if args.no_side or args.sides == "none":
        return set()
    if args.sides == "all":
        out = set(SIDES)
    else:
        out = {x.strip() for x in args.sides.split(",") if x.strip()}
        bad = out - set(SIDES)
        if bad:
            raise SystemExit(f"unknown --sides entries: {sorted(bad)}")
    if args.no_serving:
        out.discard("serving")
    return out


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows, self.proc, self.thread = [], None, None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[4 + i].lower() in ("active", "yes", "1")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def paper_problem_side(pkg, stream, hbm_gbs, peak_kind, n=510, steps=500):
    """The paper's variable-coefficient problem at its N = 512 (510^3 interior
    nodes, dt = h^2/(12 kappa_max)), 500 steps, FP64 and FP32 (n and steps:
    another size, for small profiling runs).  The paper's
    measured k = 6.4042e-11 s per point-step for OpenMP offload on one H100
    (Table of used measurements) is 15.6 GLUP/s -- another GPU's number, for
    context."""
    import torch

    from workloads import heat_u0_single_mode
    u0 = heat_u0_single_mode(n, n, n)
    out = {"grid": f"{n}^3 interior" + (" (paper N = 512)" if n == 510 else ""), "steps": steps,
           "r": 1.0 / (12 * 0.95),
           "paper_h100_openmp_glups": 1.0 / 6.4042e-11 / 1e9}
    for dtype in ("f64", "f32"):
        src = torch.from_numpy(u0).cuda()
        if dtype == "f32":
            src = src.float()
        with pkg.Heat(n, n, n, 1.0 / (12 * 0.95), dtype=dtype, flags=pkg.HS_VARKAPPA, stream=stream) as h:
            h.upload(src).step(20)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h.upload(src)
            e0.record(stream)
            h.step(steps)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
        lups = float(n) ** 3 * steps
        out[dtype] = {"glups": lups / (ms * 1e-3) / 1e9, "ms": ms}
        # FP64: u read and written, three face-sum arrays of kappa, dt f (48 B);
        # FP32: u read and written, kappa, dt f (16 B).  The cubic FP64 grid
        # runs the exact-sum form (2 FP64 instructions per update, the operator
        # sum in 128-bit integers), bound by integer issue and load latency:
        # its roofline object is HBM at 48 B per update, with the FP64 pipe's
        # share beside it
        bpl = 48 if dtype == "f64" else 16
        kname = "k_vk_interior_xs + k_vk_boundary_xs (exact sum)" if dtype == "f64" else \
            "k_vk_interior_f4 + k_vk_boundary<float>"
        hbm = hbm_roofline(kname, lups * bpl, ms, hbm_gbs, peak_kind, bytes_per_lup=bpl)
        if dtype == "f64":
            rate = lups * VK_FP64_OPS_PER_LUP / (ms * 1e-3) / 1e12
            hbm.update({"fp64_ops_per_lup": VK_FP64_OPS_PER_LUP, "fp64_achieved_t": rate,
                        "fp64_frac": rate / FP64_INSTR_PEAK_T})
        out[dtype]["roofline"] = hbm
        del src
    return out


def batching_side(pkg, stream, hbm_gbs, peak_kind):
    """The batching workload: 256 heat grids (edges log-uniform in [16, 128],
    FP64/FP32, r ~ U[0.05, 0.16], steps ~ U{50..500}) in one persistent launch
    replayed from a CUDA graph, against the same grids stepped one handle at a
    time; and 64 CG solves (edges in [32, 128], rtol 1e-8) batched against one
    at a time."""
    import numpy as np
    import torch

    from workloads import cg_batch_specs, heat_batch_specs

    def ev():
        return torch.cuda.Event(enable_timing=True)

    specs = heat_batch_specs(256)
    heats = []
    for s in specs:
        nz, ny, nx = s["shape"]
        h = pkg.Heat(nx, ny, nz, s["r"], dtype=s["dtype"], stream=stream, tdepth=1)
        h.upload(s["u0"].astype(h.np_dtype))
        heats.append(h)
    out = {}
    with pkg.HeatBatch(heats, [s["steps"] for s in specs], stream=stream) as b:
        b.run(use_graph=True).wait()                      # warm-up (captures the graph)
        e0, e1 = ev(), ev()
        e0.record(stream)
        b.run(use_graph=True)
        e1.record(stream)
        b.wait()
        ms = e0.elapsed_time(e1)
        nbytes = sum(int(np.prod(sp["shape"])) * sp["steps"] * (16 if sp["dtype"] == "f64" else 8)
                     for sp in specs)
        out["heat_256"] = {"lups": b.lups, "ms": ms, "glups": b.lups / (ms * 1e-3) / 1e9,
                           "blocks": b.blocks, "launches_per_run": 1,
                           "roofline": hbm_roofline("k_heat_batch (persistent, all grids and steps)",
                                                    nbytes, ms, hbm_gbs, peak_kind,
                                                    bytes_per_lup="16 (FP64 grids) / 8 (FP32 grids)")}
    e0, e1 = ev(), ev()
    e0.record(stream)
    for s, h in zip(specs, heats):
        h.step(s["steps"])
    e1.record(stream)
    e1.synchronize()
    ms1 = e0.elapsed_time(e1)
    out["heat_256"]["alone_ms"] = ms1
    out["heat_256"]["speedup_vs_alone"] = ms1 / out["heat_256"]["ms"]
    for h in heats:
        h.close()
    cg_specs = cg_batch_specs(64)
    ops = [pkg.Operator.stencil(nx, ny, nz) for (nz, ny, nx), _ in cg_specs]
    bs = [torch.from_numpy(b).cuda() for _, b in cg_specs]
    with pkg.CGBatch(ops, stream=stream) as cb:
        cb.run(bs, rtol=1e-8, max_iter=20000)             # warm-up
        e0, e1 = ev(), ev()
        e0.record(stream)
        _, infos = cb.run(bs, rtol=1e-8, max_iter=20000)
        e1.record(stream)
        e1.synchronize()
        msb = e0.elapsed_time(e1)
    e0, e1 = ev(), ev()
    e0.record(stream)
    iters = 0
    for op, b in zip(ops, bs):
        with pkg.CG(op, stream=stream) as cg:
            _, inf = cg.run(b, rtol=1e-8, max_iter=20000)
            iters += inf["iters"]
    e1.record(stream)
    e1.synchronize()
    msa = e0.elapsed_time(e1)
    out["cg_64"] = {"ms": msb, "alone_ms": msa, "speedup_vs_alone": msa / msb,
                    "total_iters": sum(i["iters"] for i in infos),
                    "all_converged": all(i["converged"] for i in infos)}
    return out


def interior_roofline(mode_name, n, int_ms, hbm_gbs, peak_kind, tdepth=1):
    """Roofline object of the dominant heat kernel from its mean launch time
    (ms): the streaming Interior kernel (tdepth 1, planes 1..n-2) or the
    temporally blocked kernel (tdepth L: all n planes, L steps per launch;
    algorithmic bytes = one read and one write of the field per launch)."""
    spec = HEAT_MODES[mode_name]
    lup = float(n) * n * (max(n - 2, 0) if tdepth == 1 else n)
    hbm_rate = lup * spec["bytes"] / (int_ms * 1e-3) / 1e9
    tname = {"f64": "double", "f64pipe": "double", "fixed64": "long long", "f32": "float"}[mode_name]
    # FP64 temporal blocking computes on the FP64 pipe
    alu = spec["bound"] == "alu" or (mode_name == "f64" and tdepth > 1)
    if tdepth > 1:
        name = f"k_heat_tb<{tname}, L={tdepth}>"
    elif mode_name == "f64pipe":
        name = "k_heat_interior<double> (Interior, register z-march, one step)"
    elif mode_name == "f64":
        name = "k_heat_stream_xs (Interior, TMA-staged, one step, FP64 exact sum)"
    else:
        name = f"k_heat_stream<{tname}> (Interior, TMA-staged, one step)"
    if alu:
        rate = lup * tdepth * FP64_INSTR_PER_LUP / (int_ms * 1e-3) / 1e12
        return {"bound": "alu", "kernel": name, "achieved": rate, "peak": FP64_INSTR_PEAK_T,
                "unit": "T FP64-instr/s", "frac": rate / FP64_INSTR_PEAK_T, "traffic": None,
                "hbm_achieved_gbs": hbm_rate, "hbm_peak_gbs": hbm_gbs, "hbm_frac": hbm_rate / hbm_gbs,
                "hbm_peak_kind": peak_kind, "interior_ms_per_launch": int_ms}
    traffic = KERNEL_TRAFFIC_BYTES.get((mode_name, n, tdepth))
    return {"bound": "hbm", "kernel": name, "achieved": hbm_rate, "peak": hbm_gbs, "unit": "GB/s",
            "frac": hbm_rate / hbm_gbs, "traffic": traffic,
            "traffic_per_algorithmic": None if traffic is None else traffic / (lup * spec["bytes"]),
            "peak_kind": peak_kind,
            "frac_of_nominal": hbm_rate / NOMINAL_HBM_GBS, "nominal_gbs": NOMINAL_HBM_GBS,
            "bytes_per_lup": spec["bytes"], "steps_per_launch": tdepth,
            "effective_gbs": hbm_rate * tdepth, "interior_ms_per_launch": int_ms}


# ---------------------------------------------------------------------------------
def cpu_baseline(args, threads):
    """The oracle as it stands, on this host's cores, on a bounded sample of the
    workload: a few 512^3 FP64 steps (timed step loop only) and a few CG
    iterations on 256^3."""
    import numpy as np

    import oracle
    from workloads import cg_rhs, heat_u0_modes

    oracle.build()
    n = args.heat_n
    u0, _, _ = heat_u0_modes(n, n, n, seed=SEED)
    _, t1 = oracle.heat_run(u0, args.r, 1, threads=threads, return_seconds=True)
    steps = int(max(2, min(200, 12.0 / max(t1, 1e-3))))
    _, secs = oracle.heat_run(u0, args.r, steps, threads=threads, return_seconds=True)
    glups = n ** 3 * steps / secs / 1e9
    _, secs1 = oracle.heat_run(u0, args.r, 2, threads=1, return_seconds=True)   # one core, two steps
    m = args.cg_n
    b = cg_rhs(m ** 3, seed=SEED)
    cg_iters = 20
    _, info = oracle.cg_solve(b, 1e-30, cg_iters, shape=(m, m, m), threads=threads)
    return {"value": glups, "unit": "GLUP/s", "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"heat {n}^3 FP64 r={args.r}, {steps} of {args.heat_steps} steps, timed step "
                      f"loop only; CG matrix-free {m}^3, {cg_iters} iterations",
            "cg_matrix_free_its_per_s": cg_iters / info["loop_seconds"],
            "single_core_glups": n ** 3 * 2 / secs1 / 1e9}


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, each step a bounded
    sample (a few 512^3 heat steps) of the same workload and metric."""
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401

    import oracle
    from workloads import heat_u0_modes

    oracle.build()
    threads = host_cores()
    n = args.heat_n
    u0, _, _ = heat_u0_modes(n, n, n, seed=SEED)
    _, t1 = oracle.heat_run(u0, args.r, 1, threads=threads, return_seconds=True)
    per = int(max(1, min(50, 8.0 / max(t1, 1e-3))))   # heat steps per sample
    times = []
    for s in range(args.warmup + args.steps):
        _, secs = oracle.heat_run(u0, args.r, per, threads=threads, return_seconds=True)
        if s >= args.warmup:
            times.append(secs)
    total = sum(times)
    value = n ** 3 * per * len(times) / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GLUP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"heat {n}^3 FP64 r={args.r} (sample: {per} steps per bench step)",
                       "seed": SEED},
            "cpu_baseline": {"value": value, "unit": "GLUP/s", "cores": threads, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"{per} heat steps of {n}^3 per bench step"},
            "e2e": {"value": value, "unit": "GLUP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)

    from paper_2608_11882_gb300.build import build
    build()
    import paper_2608_11882_gb300 as pkg
    from paper_2608_11882_gb300 import _native as nat
    from workloads import cg_rhs, heat_u0_modes, lap7_csr

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    n, m = args.heat_n, args.cg_n
    stream = torch.cuda.current_stream()

    # ---- inputs (seeded, synthetic), resident in HBM before timing -------------
    u0_np, _, _ = heat_u0_modes(n, n, n, seed=SEED)
    u0_host = torch.from_numpy(u0_np).pin_memory()
    u0_dev = u0_host.to("cuda", non_blocking=False)
    u_out_dev = torch.empty_like(u0_dev)
    b_np = cg_rhs(m ** 3, seed=SEED)
    b_host = torch.from_numpy(b_np).pin_memory()
    b_dev = b_host.cuda()
    rowptr, col, val = lap7_csr(m, m, m)
    csr_dev = [torch.from_numpy(a).cuda() for a in (rowptr, col, val)]
    nnz = int(col.size)
    del rowptr, col, val
    x_mf = torch.zeros(m ** 3, dtype=torch.float64, device="cuda")
    x_csr = torch.zeros_like(x_mf)

    def make_heat(mode):
        spec = HEAT_MODES[mode]
        flags = getattr(pkg, spec["flags"]) if spec["flags"] else 0
        return pkg.Heat(n, n, n, args.r, dtype=spec["dtype"], flags=flags, stream=stream,
                        tdepth=args.tdepth)

    mode = HEAT_MODES[args.heat_mode]
    heat = make_heat(args.heat_mode)
    if mode["dtype"] == "f32":
        u0_dev = u0_dev.float()
        u0_host = u0_host.float().pin_memory()
        u_out_dev = torch.empty_like(u0_dev)
    cg_mf = pkg.CG(pkg.Operator.stencil(m, m, m), stream=stream)
    cg_csr = pkg.CG(pkg.Operator.csr(*csr_dev), stream=stream)
    torch.cuda.synchronize()

    hsteps = args.heat_steps

    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    step_launches = [0]

    def one_step(timed_interior: bool):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        heat.upload(u0_dev)
        if timed_interior and heat.tdepth > 1:
            # blocked passes: one kernel per pass, timed around the whole step loop
            step_ev[0].record(stream)
            l0 = nat.launch_count()
            heat.step(hsteps)
            step_launches[0] = nat.launch_count() - l0
            step_ev[1].record(stream)
        elif timed_interior:
            # the library brackets each Interior launch with events on this stream
            heat.time_interior(True)
            heat.step(hsteps)
            heat.time_interior(False)
        else:
            heat.step(hsteps)
        heat.read(u_out_dev)
        ev[1].record(stream)
        x_mf.zero_()
        _, info_mf = cg_mf.run(b_dev, x_mf, rtol=args.rtol, max_iter=20000)
        ev[2].record(stream)
        x_csr.zero_()
        _, info_csr = cg_csr.run(b_dev, x_csr, rtol=args.rtol, max_iter=20000)
        ev[3].record(stream)
        return ev, info_mf, info_csr

    for _ in range(args.warmup):
        one_step(False)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    launches0 = nat.launch_count()
    barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    seg = {"heat": [], "cg_mf": [], "cg_csr": []}
    interior_ms = []
    infos = []
    for s in range(args.steps):
        ev, i_mf, i_csr = one_step(True)
        ev[3].synchronize()
        seg["heat"].append(ev[0].elapsed_time(ev[1]))
        seg["cg_mf"].append(ev[1].elapsed_time(ev[2]))
        seg["cg_csr"].append(ev[2].elapsed_time(ev[3]))
        if heat.tdepth > 1:
            interior_ms.append(step_ev[0].elapsed_time(step_ev[1]) / step_launches[0])
        else:
            interior_ms.append(heat.interior_time()[0])
        infos.append((i_mf, i_csr))
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = nat.launch_count() - launches0
    clock_info = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    heat_ms = sum(seg["heat"])
    if world > 1:
        t = torch.tensor([elapsed_ms, heat_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed_ms, heat_ms = float(t[0]), float(t[1])

    lup_step = float(n) ** 3 * hsteps
    value = world * lup_step * args.steps / (heat_ms * 1e-3) / 1e9
    hbm_gbs, peak_kind = measured_peaks()

    # dominant kernel: the Interior kernel of the timed heat mode
    int_ms = statistics.mean(interior_ms)
    roofline = interior_roofline(args.heat_mode, n, int_ms, hbm_gbs, peak_kind, heat.tdepth)

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]

    it_mf = [i[0]["iters"] for i in infos]
    it_csr = [i[1]["iters"] for i in infos]
    nrow = float(m) ** 3
    cg_roof = {
        "matrix_free": hbm_roofline("CG matrix-free (SpMV + updates, whole solve)",
                                    it_mf[-1] * CG_BYTES_PER_ROW * nrow, statistics.median(seg["cg_mf"]),
                                    hbm_gbs, peak_kind, bytes_per_row_per_iter=CG_BYTES_PER_ROW),
        "csr": hbm_roofline("CG CSR (SpMV + updates, whole solve)",
                            it_csr[-1] * (CG_BYTES_PER_ROW * nrow + 12.0 * nnz + 4 * nrow),
                            statistics.median(seg["cg_csr"]), hbm_gbs, peak_kind)}
    line = {
        "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": mode["arith"], "data": "synthetic",
        "config": {"workload": f"heat {n}^3 {args.heat_mode} r={args.r} {hsteps} steps (u0 = 8 sine modes k in "
                               f"[1,16] + 1e-3 U[-1,1]) + CG {m}^3 FP64 7-pt Dirichlet Laplacian, "
                               f"matrix-free and CSR int32 (nnz {nnz}), b ~ N(0,1), rtol {args.rtol}",
                   "arithmetic": "FP64 fields; FP64 pipe (temporal blocking)"
                   if args.heat_mode == "f64" and heat.tdepth > 1 else mode["desc"],
                   "tdepth": heat.tdepth,
                   "value_covers": "heat segment (upload + steps + device readback), device time",
                   "l2": "no flush: every input exceeds L2 (field 1.07 GB, vectors 134 MB)",
                   "parallelism": f"replicas x{world}", "seed": SEED},
        "heat": {"glups": value / world, "ms_per_solve": heat_ms / args.steps,
                 "bytes_per_lup": mode["bytes"],
                 "hbm_frac_one_step_per_pass": value / world * mode["bytes"] / hbm_gbs},
        "cg": {"matrix_free": {"iters": it_mf[-1], "its_per_s": it_mf[-1] / (statistics.median(seg["cg_mf"]) * 1e-3),
                               "ms_per_solve": statistics.median(seg["cg_mf"]),
                               "relres_true": infos[-1][0]["relres_true"],
                               "roofline": cg_roof["matrix_free"]},
               "csr": {"iters": it_csr[-1], "its_per_s": it_csr[-1] / (statistics.median(seg["cg_csr"]) * 1e-3),
                       "ms_per_solve": statistics.median(seg["cg_csr"]),
                       "relres_true": infos[-1][1]["relres_true"], "roofline": cg_roof["csr"]}},
        "latency_ms": {k: {"p50": pct(v, 0.5), "p99": pct(v, 0.99)} for k, v in seg.items()},
        # (max - min) / median of each segment over the timed steps
        "variability": {k: (max(v) - min(v)) / statistics.median(v) for k, v in seg.items()},
        "roofline": roofline,
        "clocks": clock_info,
        "gpu_launches": launches,
    }

    # ---- end to end through the C ABI with host buffers ----------------------
    if not args.no_e2e:
        u_back = torch.empty_like(u0_host).pin_memory()
        x_host = torch.zeros(m ** 3, dtype=torch.float64).pin_memory()
        e2e_heat, e2e_cg = [], []
        barrier()
        for s in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            heat.upload(u0_host)                   # pinned host -> device
            heat.step(hsteps)
            heat.read(u_back)                      # device -> pinned host (synchronises)
            t1 = time.perf_counter()
            x_host.zero_()
            cg_mf.run(b_host.numpy(), x_host.numpy(), rtol=args.rtol, max_iter=20000)
            t2 = time.perf_counter()
            e2e_heat.append(t1 - t0)
            e2e_cg.append(t2 - t1)
        e2e_t = max(sum(e2e_heat), 0.0)
        if world > 1:
            t = torch.tensor([e2e_t], dtype=torch.float64, device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_t = float(t[0])
        line["e2e"] = {"value": world * lup_step * args.steps / e2e_t / 1e9, "unit": "GLUP/s",
                       "h2d_bytes_per_step": int(u0_host.numel() * u0_host.element_size()),
                       "d2h_bytes_per_step": int(u_back.numel() * u_back.element_size()),
                       "covers": "heat: heat_upload from pinned host, heat_step, heat_read to pinned host",
                       "cg_matrix_free_host_buffers_its_per_s": it_mf[-1] / statistics.median(e2e_cg)}

    sides = sides_of(args)

    # ---- the other heat modes, one untimed-region solve each -------------------
    if "modes" in sides:
        def solve_once(h, src):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            h.upload(src)
            if h.tdepth > 1:
                step_ev[0].record(stream)
                l0 = nat.launch_count()
                h.step(hsteps)
                nl = nat.launch_count() - l0
                step_ev[1].record(stream)
            else:
                h.time_interior(True)
                h.step(hsteps)
            out = torch.empty_like(src)
            h.read(out)
            ev1.record(stream)
            ev1.synchronize()
            if h.tdepth > 1:
                ims = step_ev[0].elapsed_time(step_ev[1]) / nl
            else:
                ims = h.interior_time()[0]
            return ev0.elapsed_time(ev1), ims, out

        fields = {args.heat_mode: u_out_dev}
        side = {}
        for name in ["f64"] + [k for k in sorted(HEAT_MODES) if k != "f64"]:
            if name == args.heat_mode:
                continue
            spec = HEAT_MODES[name]
            src = torch.from_numpy(u0_np).cuda()
            if spec["dtype"] == "f32":
                src = src.float()
            h2 = make_heat(name)
            seg_ms, ims, out = solve_once(h2, src)
            side_tdepth = h2.tdepth
            h2.close()
            fields[name] = out
            side[name] = {"glups": lup_step / (seg_ms * 1e-3) / 1e9, "arith": spec["arith"],
                          "tdepth": side_tdepth,
                          "roofline": interior_roofline(name, n, ims, hbm_gbs, peak_kind, side_tdepth)}
            del src
        ref = fields["f64"].double()
        refmax = float(ref.abs().max())
        for name, f in fields.items():
            if name == "f64":
                continue
            err = float((f.double() - ref).abs().max())
            entry = side.setdefault(name, {"glups": value / world, "arith": HEAT_MODES[name]["arith"]})
            entry["max_abs_diff_vs_f64_gpu"] = err
            entry["max_rel_diff_vs_f64_gpu"] = err / refmax
        line["heat_modes"] = side

    # ---- batching: 256 uneven heat grids in one persistent launch, 64 CG solves -
    if "batching" in sides:
        line["batching"] = batching_side(pkg, stream, hbm_gbs, peak_kind)

    # ---- the paper's own problem: variable kappa, N = 512, 500 steps ---------------
    if "paper" in sides:
        line["paper_problem"] = paper_problem_side(pkg, stream, hbm_gbs, peak_kind, args.paper_n,
                                                   args.paper_steps)

    # ---- mixed-precision CG beside the FP64 solves (untimed region) ------------
    if "mixed" in sides:
        mixed = {}
        for kind, op in (("matrix_free", pkg.Operator.stencil(m, m, m)), ("csr", pkg.Operator.csr(*csr_dev))):
            with pkg.CG(op, stream=stream, mixed=True) as cgm:
                xm = torch.zeros_like(x_mf)
                cgm.run(b_dev, xm, rtol=args.rtol, max_iter=200000)   # warm-up
                xm.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, im = cgm.run(b_dev, xm, rtol=args.rtol, max_iter=200000)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                nrow = float(m) ** 3
                csr_inner = (8.0 * nnz + 4 * nrow) if kind == "csr" else 0.0
                csr_ref = (12.0 * nnz + 4 * nrow) if kind == "csr" else 0.0
                nbytes = (im["iters"] * (MIXED_INNER_BYTES_PER_ROW[kind] * nrow + csr_inner)
                          + (im["refinements"] + 1) * (MIXED_REFINE_BYTES_PER_ROW * nrow + csr_ref))
                mixed[kind] = {"ms_per_solve": ms, "inner_iters": im["iters"],
                               "refinements": im["refinements"], "relres_true": im["relres_true"],
                               "speedup_vs_f64": line["cg"][kind]["ms_per_solve"] / ms,
                               "roofline": hbm_roofline(f"mixed CG {kind} (whole solve)", nbytes, ms,
                                                        hbm_gbs, peak_kind)}
        line["cg"]["mixed_f32_krylov"] = mixed

    # ---- precision: heat 1024^3 FP32 against FIXED64, CG 512^3 to 1e-10 ---------
    if "precision" in sides:
        line["precision"] = precision_side(pkg, stream)

    # ---- serving: the Poisson request stream, closed loop and one offered load ----
    if "serving" in sides:
        line["serving"] = serving_side(args, loads=(0.7,))

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, host_cores())

    heat.close()
    cg_mf.close()
    cg_csr.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def precision_side(pkg, stream):
    """The precision workload: heat 1024^3 FP32 (storage and arithmetic, the
    default two steps per pass), r = 0.1, 2000 steps, max error against the
    FIXED64 path (FP64 interface, parity-tested against the FP64 oracle); CG
    on 512^3 to rtol 1e-10 with FP32 Krylov vectors and FP64 refinement,
    beside FP64 CG.  The field is formed on the device (heat_u0_modes_device)."""
    import torch

    from workloads import cg_rhs, heat_u0_modes_device

    n, steps, r = 1024, 2000, 0.1
    res = {}
    fields = {}
    for mode, dtype, flags in (("f32", "f32", 0), ("fixed64", "f64", pkg.HS_FIXED64)):
        src = heat_u0_modes_device(n, n, n, "cuda", seed=SEED)
        if dtype == "f32":
            src = src.float()
        with pkg.Heat(n, n, n, r, dtype=dtype, flags=flags, stream=stream) as h:
            h.upload(src)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.step(steps)
            e1.record(stream)
            out = torch.empty_like(src)
            h.read(out)
            ms = e0.elapsed_time(e1)
            res[mode] = {"glups": float(n) ** 3 * steps / (ms * 1e-3) / 1e9, "ms": ms, "tdepth": h.tdepth}
        fields[mode] = out.double()
        del src, out
    ref = fields["fixed64"]
    err = float((fields["f32"] - ref).abs().max())
    res["f32"]["max_abs_err_vs_fixed64"] = err
    res["f32"]["max_rel_err_vs_fixed64"] = err / float(ref.abs().max())
    del fields, ref
    torch.cuda.empty_cache()
    m = 512
    b = torch.from_numpy(cg_rhs(m ** 3, seed=SEED)).cuda()
    cgres = {}
    for name, kw in (("f64", {}), ("mixed_f32_krylov", {"mixed": True})):
        with pkg.CG(pkg.Operator.stencil(m, m, m), stream=stream, **kw) as cg:
            x = torch.zeros_like(b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info = cg.run(b, x, rtol=1e-10, max_iter=400000)
            e1.record(stream)
            e1.synchronize()
            cgres[name] = {"ms": e0.elapsed_time(e1), "iters": info["iters"],
                           "refinements": info["refinements"], "relres_true": info["relres_true"],
                           "converged": info["converged"]}
    cgres["mixed_speedup"] = cgres["f64"]["ms"] / cgres["mixed_f32_krylov"]["ms"]
    del b
    torch.cuda.empty_cache()
    return {"workload": "precision: heat 1024^3 FP32 r=0.1 2000 steps against FIXED64; "
                        "CG 512^3 matrix-free rtol 1e-10, FP64 and mixed",
            "heat": res, "cg": cgres}


def run_precision(args):
    """--workload precision: the precision workload alone."""
    import torch

    from paper_2608_11882_gb300.build import build
    build()
    import paper_2608_11882_gb300 as pkg
    print(json.dumps(precision_side(pkg, torch.cuda.current_stream())), flush=True)
    return 0


def serving_side(args, loads=(0.5, 0.7, 0.9)):
    """The serving workload: a seeded Poisson stream of heat (75%) and CG (25%)
    requests, edges log-uniform in [32, 384] per axis, steps log-uniform in
    [10, 2000], FP32/FP64 half each, admitted by free HBM with fields resident.
    Capacity is measured closed-loop (every request arriving at once); the
    same trace is then replayed at the given fractions of that request rate."""
    import torch

    from paper_2608_11882_gb300.serve import GpuBackend, Server, poisson_trace, predict_seconds, summarize

    base = poisson_trace(args.requests, rate=1.0, seed=SEED)   # arrivals for rate 1, rescaled below
    unit = [q.arrival for q in base]
    cal = GpuBackend(workers=1)
    kbars = cal.calibrate()   # the paper's k-bar model, fitted on this GPU (heat_step alone)
    cal.close()

    def serve(scale):
        for q, a in zip(base, unit):
            q.arrival = a * scale
        be = GpuBackend(workers=4)
        srv = Server(be, quantum=64, max_slots=32, kbars=kbars)
        res = srv.run(base)
        be.close()
        out = summarize(res, base, srv.makespan)
        out.update({"peak_slots": srv.peak_slots, "peak_gb": srv.peak_bytes / 1e9,
                    "rejected": len(srv.rejected)})
        return out

    closed = serve(0.0)
    capacity = args.requests / closed["makespan_s"]
    line = {"workload": f"serving: {args.requests} Poisson-arrival requests (heat 75% / CG 25%), "
                        "edges log-uniform [32, 384], steps log-uniform [10, 2000], FP32/FP64 50/50, "
                        "CG rtol 1e-8", "seed": SEED,
            "closed_loop": closed, "capacity_req_per_s": capacity, "loads": {},
            "kbar_s_per_point_step": kbars,
            "predicted_heat_device_s": sum(predict_seconds(q, kbars) for q in base if q.kind == "heat")}
    for load in loads:
        line["loads"][str(load)] = serve(1.0 / (load * capacity))
    torch.cuda.synchronize()
    return line


def run_serving(args):
    """--workload serving: the serving workload at offered loads 0.5, 0.7, 0.9."""
    from paper_2608_11882_gb300.build import build
    build()
    print(json.dumps(serving_side(args)), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "serving":
        return run_serving(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
