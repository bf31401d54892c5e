#!/usr/bin/env python3
"""Throughput of the SLDG Strang step on GB300: one JSON line on stdout.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--precision fp64|fp32]
    python bench.py --ingest-ncu REP.ncu-rep --ncu-case NAME [--ncu-targets NAME,...]

A step is one Strang step of the whole hot path (x1, x2 half drifts, rho,
Poisson, v1, v2 kicks, x1, x2 half drifts) over the synthetic initial value
of the workload (default: the two-stream instability, 64^2 x 128^2 cells,
degree 2, 5.4e9 nodal values, FP64 storage swept in double-float
arithmetic; the FP32-storage run and the FP64-FMA run of the same workload
are reported beside it).  ``value`` is dof-updates per second over the
whole job with f resident in HBM; ``e2e`` is the same metric through the C
ABI with f uploaded from pinned host memory and W read back every step.
With torchrun (N > 1) every rank runs an independent replica (the path
needs no exchange on one GPU): value is the sum over ranks, timed by the
slowest rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4D SLDG dof-updates/s & HBM GB/s (FP64 vs FP32); adjoint/forward step ratio"
UNIT = "dof-updates/s"
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
FP64_FMA_PER_CLK_SM = 2   # FP64 FMA units per SM of GB300 (1.25 TFLOP/s nominal)
FP32_LANES_PER_SM = 128   # FP32 operations per clock per SM
DF_OPS_PER_MAC = 12       # FP32 operations per lane of a double-float multiply-accumulate
DEFAULT_WORKLOAD = "two_stream_64x128"


def device_sms():
    """Streaming multiprocessors of the current CUDA device."""
    import torch

    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def arithmetic(cfg):
    """The arithmetic type the sweeps of a configuration compute in."""
    if cfg.precision == "fp32":
        return "f32"
    if cfg.flags & 1 or cfg.flags & 16:  # FP64 FMA sweeps; the spline method sweeps in FP64
        return "f64"
    return "double-float (f32 pair; f64 storage)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--precision", default=None, choices=[None, "fp64", "fp32"])
    p.add_argument("--no-extras", action="store_true", help="skip the fp32 and adjoint lines")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    p.add_argument("--native-fp64", action="store_true",
                   help="FP64 storage swept with FP64 FMA instead of double-float arithmetic")
    p.add_argument("--ingest-ncu", default=None, metavar="REP",
                   help="write profiles/ncu_traffic.json from an ncu report and print its summary")
    p.add_argument("--ncu-case", default="two_stream_64x16",
                   help="workload the ncu report was captured on")
    p.add_argument("--ncu-targets", default=f"{DEFAULT_WORKLOAD},nonlinear_landau_64",
                   help="workloads (same degree and x-grid) the traffic is scaled to")
    p.add_argument("--summarize-launches", default=None, metavar="CSV",
                   help="print the per-kernel table of an ncu launch list (gpu__time_duration)")
    return p.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    """The slowest rank's time (a CUDA tensor under NCCL, a CPU one under gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, steps, world, ms_max):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time."""
    return units_per_rank * steps * world / (ms_max / 1e3)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# measured peaks and committed ncu traffic
# ---------------------------------------------------------------------------
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return p, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


HOST_HEADERS = ("ctx.h", "fields.cuh")  # the host context and launcher declarations


def unit_sha1(unit):
    """SHA-1 of one kernel translation unit of csrc/ and every csrc/ header it
    includes (recursively): the sources of the kernels it instantiates.  The
    host-only headers (the context structure, launcher declarations) are
    followed for their includes but not hashed: they hold no device code."""
    d = os.path.join(ROOT, "paper_1803_02143_gb300", "csrc")
    seen = []

    def visit(name):
        path = os.path.join(d, name)
        if name in seen or not os.path.exists(path):
            return
        seen.append(name)
        with open(path) as fh:
            for inc in re.findall(r'#include "([^"]+)"', fh.read()):
                visit(inc)

    visit(unit)
    h = hashlib.sha1()
    for name in sorted(n for n in seen if n not in HOST_HEADERS):
        with open(os.path.join(d, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()


def committed_traffic(key):
    """DRAM bytes per launch of a kernel from a committed ncu capture, or None
    when the sources of its translation unit changed since that capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    e = t.get(key)
    if not e or "unit" not in e or e.get("csrc_sha1") != unit_sha1(e["unit"]):
        return None
    return e.get("bytes_per_launch")


# ---------------------------------------------------------------------------
# ncu report -> committed DRAM traffic per launch and a summary table
# ---------------------------------------------------------------------------
NCU_METRICS = ("gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum,"
               "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed,"
               "sm__throughput.avg.pct_of_peak_sustained_elapsed,"
               "sm__warps_active.avg.pct_of_peak_sustained_active,"
               "smsp__issue_active.avg.pct_of_peak_sustained_active,"
               "sm__inst_executed.sum,launch__registers_per_thread,"
               "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active,"
               "sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active,"
               "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active")

# (workload, precision, kind) whose launches run another kernel than the
# capture case: FP32 v-sweeps of 384- and 256-value lines exceed the packed
# tile and run the one-lane kernel, while the 48- and 32-value lines of the
# capture cases run the packed one
NCU_NOT_SCALED = {("two_stream_64x128", "fp32", "v1"), ("two_stream_64x128", "fp32", "v2"),
                  ("mixed_landau_128", "fp32", "v1"), ("mixed_landau_128", "fp32", "v2")}

# translation unit of each kernel family (its sources key the traffic entry)
KERNEL_UNITS = (("k_sweep_x12_df", "sweep_df_x12.cu"), ("k_sweep_strided_df3", "sweep_df.cu"),
                ("k_sweep_x1_warp", "sweep_df.cu"), ("k_sweep_x12_f32", "sweep_f32.cu"),
                ("k_sweep_strided_f2", "sweep_f32.cu"), ("k_sweep_x1_f2warp", "sweep_f32.cu"),
                ("k_rho_partial", "fields.cu"), ("k_spline_sweep", "spline.cu"))


def _kernel_kind(name):
    """(kind, precision) of a sweep kernel from its ncu name, or None.  FP64:
    the double-float families (a `_df` in the name, and the four-node x1
    kernel `k_sweep_x1_warp`) and kernels whose first template argument is
    double (`k_rho_partial<T>`, `k_spline_sweep<T>`)."""
    base = name.split("(")[0]  # template arguments only, not the parameter list
    fp64 = "_df" in base or "k_sweep_x1_warp" in base or re.search(r"<\s*double\b", base)
    prec = "fp64" if fp64 else "fp32"
    if "k_sweep_x12" in name:
        return "x12", prec
    if "k_sweep_x1" in name:
        return "x1", prec
    if "k_rho_partial" in name:
        return "rho", prec
    m = re.search(r"k_spline_sweep<\s*\w+,\s*(\w+),\s*(\w+)", name)
    if m:  # <T, CONTIG, KEYCOL, NB, RC>: x1 lines contiguous, v-sweeps keyed by column
        if m.group(1) in ("1", "true"):
            return "x1", prec
        return ("v", prec) if m.group(2) in ("1", "true") else ("x2", prec)
    m = re.search(r"k_sweep_strided_\w+<\s*\d+,\s*(\w+),\s*(\w+)", name)
    if m:
        periodic = m.group(1) in ("1", "true")
        percol = m.group(2) in ("1", "true")
        if percol and not periodic:
            return "v", prec
        if periodic and not percol:
            return "x2", prec
    return None


def summarize_launches(path):
    """Launches, total device time and share per kernel of an ncu launch list
    (--metrics gpu__time_duration.sum --csv), as a markdown table."""
    import csv

    with open(path) as fh:
        rows = [r for r in csv.reader(fh) if len(r) > 5]
    head = rows[0]
    ci, cn, cu, cv = (head.index(k) for k in ("ID", "Kernel Name", "Metric Unit", "Metric Value"))
    scale = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0,
             "msecond": 1.0, "s": 1e3, "second": 1e3}
    tot, cnt = {}, {}
    for r in rows[1:]:
        if not r[ci].strip().isdigit():
            continue
        name = r[cn].split("(")[0].replace("void ", "").replace("sldg::", "").strip()
        ms = float(r[cv].replace(",", "")) * scale.get(r[cu].strip().lower(), 1e-6)
        tot[name] = tot.get(name, 0.0) + ms
        cnt[name] = cnt.get(name, 0) + 1
    allms = sum(tot.values())
    print(f"{sum(cnt.values())} launches, {allms:.2f} ms of device time (serialised, cold caches)\n")
    print("| kernel | launches | total ms | share |")
    print("|---|---|---|---|")
    for name in sorted(tot, key=lambda k: -tot[k]):
        print(f"| `{name}` | {cnt[name]} | {tot[name]:.3f} | {100 * tot[name] / allms:.1f}% |")


def ingest_ncu(args):
    """Per-launch DRAM traffic of the sweep kernels in an ncu report captured on
    args.ncu_case, scaled by the ratio of nodal values to each target workload
    (every byte of these kernels scales with the dof count), written to
    profiles/ncu_traffic.json keyed by the current sources of each kernel's
    translation unit; prints a markdown summary of the captured launches."""
    import csv
    import io

    from paper_1803_02143_gb300 import configs

    out = subprocess.run(["ncu", "-i", args.ingest_ncu, "--page", "raw", "--csv",
                          "--print-units", "base", "--metrics", NCU_METRICS],
                         capture_output=True, text=True, check=True).stdout
    rows = list(csv.reader(io.StringIO(out)))
    head, units = rows[0], rows[1]
    data = [r for r in rows[2:] if len(r) == len(head)]
    col = {h: i for i, h in enumerate(head)}
    # values to bytes and nanoseconds whatever scale the report prints
    scale = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "tbyte": 1e12,
             "ns": 1.0, "nsecond": 1.0, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6,
             "s": 1e9, "second": 1e9}
    case = configs.workload(args.ncu_case)
    by_kind, table = {}, []
    vcount = {}
    for r in data:
        name = r[col["Kernel Name"]]
        kk = _kernel_kind(name)

        def num(metric):
            if metric not in col:
                return float("nan")
            v = r[col[metric]].replace(",", "")
            try:
                return float(v) * scale.get(units[col[metric]].strip().lower(), 1.0)
            except ValueError:
                return float("nan")

        rd, wr = num("dram__bytes_read.sum"), num("dram__bytes_write.sum")
        dur = num("gpu__time_duration.sum")
        table.append((name.split("(")[0].replace("void ", "").replace("sldg::", ""), dur, rd, wr,
                      num("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed"),
                      num("sm__throughput.avg.pct_of_peak_sustained_elapsed"),
                      num("smsp__issue_active.avg.pct_of_peak_sustained_active"),
                      num("sm__warps_active.avg.pct_of_peak_sustained_active"),
                      num("sm__inst_executed.sum"), num("launch__registers_per_thread"),
                      num("sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active"),
                      num("sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active"),
                      num("sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active")))
        if kk is None:
            continue
        kind, prec = kk
        if kind == "v":  # v1 and v2 alternate within a step
            i = vcount.get(prec, 0)
            vcount[prec] = i + 1
            kind = "v1" if i % 2 == 0 else "v2"
        unit = next((u for k, u in KERNEL_UNITS if k in name), None)
        by_kind.setdefault((prec, kind), []).append((rd + wr, unit))
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            traffic = json.load(fh)
    except (OSError, ValueError):
        traffic = {}
    traffic["_note"] = ("DRAM bytes (read + write) per launch, scaled from ncu captures on a "
                        "smaller case with the same x-grid and degree by the ratio of nodal "
                        "values (written by bench.py --ingest-ncu); unit names the translation "
                        "unit that instantiates the kernel and csrc_sha1 the hash of its "
                        "sources when the counters were taken.")
    rep = os.path.basename(args.ingest_ncu)
    for tname in args.ncu_targets.split(","):
        tw = configs.workload(tname)
        scale = tw.cfg.numel / case.cfg.numel
        for (prec, kind), vals in by_kind.items():
            unit = vals[0][1]
            if unit is None or (tname, prec, kind) in NCU_NOT_SCALED:
                traffic.pop(f"{tname}:{prec}:{kind}", None)
                continue
            b = sum(v for v, _ in vals) / len(vals)
            traffic[f"{tname}:{prec}:{kind}"] = {
                "bytes_per_launch": b * scale, "capture": f"{rep} on {case.name}",
                "csrc_sha1": unit_sha1(unit), "unit": unit}
    with open(path, "w") as fh:
        json.dump(traffic, fh, indent=1, sort_keys=True)
    n = case.cfg.numel
    print(f"Captured on {case.name}: {n} nodal values; algorithmic bytes per sweep launch "
          f"2 e N (e = element size; the fused x pass does two sweeps per launch).\n")
    print("| kernel | ms | DRAM read GB | DRAM write GB | DRAM % | SM % | issue active % | "
          "warps active % | warp instr per dof | regs | FMA pipe % | ALU pipe % | FP64 pipe % |")
    print("|---|---|---|---|---|---|---|---|---|---|---|---|---|")
    for t in table:
        print(f"| `{t[0]}` | {t[1] / 1e6:.3f} | {t[2] / 1e9:.3f} | {t[3] / 1e9:.3f} | {t[4]:.1f} "
              f"| {t[5]:.1f} | {t[6]:.1f} | {t[7]:.1f} | {t[8] / n:.2f} | {t[9]:.0f} | "
              f"{t[10]:.1f} | {t[11]:.1f} | {t[12]:.1f} |")


# ---------------------------------------------------------------------------
# CPU oracle baseline on a bounded slab of the workload
# ---------------------------------------------------------------------------
def oracle_slab(w, vcells=32):
    """Same x-grid and degree, v reduced to vcells^2 cells: per-dof work of
    the sweeps is unchanged (same line lengths along x, same degree)."""
    import oracle as orc

    c = w.cfg
    nc = (c.ncell[0], c.ncell[1], min(c.ncell[2], vcells), min(c.ncell[3], vcells))
    return orc.Grid(deg=c.degree, nc=nc, lo=c.lo, hi=c.hi, dt=c.dt, vbc=c.vbc,
                    kmax=c.poisson_kmax)


def time_oracle(w, nsteps, warmup=0):
    import oracle as orc

    g = oracle_slab(w)
    f = orc.init(g, w.kind, w.params)
    if warmup:
        orc.step_inplace(g, f, warmup)
    t0 = time.perf_counter()
    orc.step_inplace(g, f, nsteps)
    dt = time.perf_counter() - t0
    dofs = f.size
    return {"value": dofs * nsteps / dt, "unit": UNIT, "cores": orc.threads(), "kind": "oracle",
            "sample": (f"{nsteps} Strang step(s) of the FP64 oracle on {g.nc[0]}x{g.nc[1]}x"
                       f"{g.nc[2]}x{g.nc[3]} cells, degree {g.deg} ({dofs} dofs; the workload's "
                       f"x-grid, degree and domain with a reduced v-grid), {dt:.1f} s"),
            "extrapolated": (f"per-dof rate of the slab taken for the workload's "
                             f"{w.cfg.numel} dofs (same line lengths along x, same degree)"
                             if dofs != w.cfg.numel else None),
            "seconds": dt, "dofs": dofs}


def cpu_info():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            txt = fh.read()
        for key in ("model name", "CPU part"):
            for line in txt.splitlines():
                if line.startswith(key):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


# ---------------------------------------------------------------------------
# the reference arm: the oracle as it stands, on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_1803_02143_gb300 import configs

    w = configs.workload(args.workload, args.precision)
    import oracle as orc

    orc.build()
    g = oracle_slab(w)
    f = orc.init(g, w.kind, w.params)
    orc.step_inplace(g, f, max(0, min(args.warmup, 1)))
    t0 = time.perf_counter()
    orc.step_inplace(g, f, args.steps)
    dt = time.perf_counter() - t0
    value = f.size * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "oracle_sample": list(g.nc), "degree": g.deg,
                   "storage": "fp64", "arithmetic": "f64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.threads(), "kind": "oracle",
                         "sample": f"{args.steps} steps on {g.nc} cells, degree {g.deg} "
                                   f"({f.size} dofs), host {cpu_info()}",
                         "extrapolated": (f"per-dof rate of the slab taken for the workload's "
                                          f"{w.cfg.numel} dofs" if f.size != w.cfg.numel
                                          else None)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def sweep_roofline(w, timing, steps_timed, pk, peak_src, sms):
    """Dominant kernel class of the timed region, against its roofline."""
    cfg = w.cfg
    n = cfg.n
    esize = 8 if cfg.precision == "fp64" else 4
    # x12: the fused X1 X2 pass of FP32 storage, one read and one write of f
    sweeps = {k: v for k, v in timing.items() if k in ("x1", "x2", "v1", "v2", "x12") and v[1] > 0}
    kind = max(sweeps, key=lambda k: sweeps[k][0])
    ms, cnt = sweeps[kind]
    avg_s = ms / cnt / 1e3
    algo_bytes = 2 * cfg.numel * esize          # read + write of f, matrices not counted
    algo_flops = 2 * 2 * n * cfg.numel          # 2(l+1) FMA per dof
    traffic = committed_traffic(f"{w.name}:{cfg.precision}:{kind}")
    hbm = {"achieved": algo_bytes / avg_s / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
           "frac": algo_bytes / avg_s / 1e9 / pk["hbm_gbs"], "peak_source": peak_src}
    native = cfg.flags & 1
    spline = cfg.flags & 16
    clk = pk.get("sm_max_mhz", 2070.0)
    per_kernel = {k: v[0] / steps_timed for k, v in timing.items() if v[1]}
    if cfg.precision == "fp64" and not native and not spline:
        # double-float sweeps: each lane of a double-float multiply-accumulate
        # is 12 FP32 operations (product, its FMA error, TwoSum, two low-word
        # adds, two cross FMAs); the fused pass does two sweeps per byte.  The
        # bound is the roofline with the longer floor for this launch.
        sweeps_per_launch = 2 if kind == "x12" else 1
        ops = sweeps_per_launch * cfg.numel * (2 * n) * DF_OPS_PER_MAC
        peak_t = sms * FP32_LANES_PER_SM * clk * 1e6 / 1e12
        if ops / (peak_t * 1e12) > algo_bytes / (pk["hbm_gbs"] * 1e9):
            return {"bound": "alu", "achieved": ops / avg_s / 1e12, "peak": peak_t,
                    "unit": "T FP32 ops/s", "frac": ops / avg_s / 1e12 / peak_t,
                    "traffic": traffic, "kernel": f"sweep_{kind}",
                    "peak_source": f"FP32 lanes x max SM clock ({sms} SMs x 128 lanes)",
                    "hbm": hbm, "avg_launch_ms": ms / cnt, "per_kernel_ms_per_step": per_kernel}
    if cfg.precision == "fp64" and spline:
        # cubic-spline sweeps in FP64 arithmetic: per point one FMA in each of
        # the two recurrences of the cyclic solve and four in the evaluation
        algo_flops = 2 * 6 * cfg.numel
        native = True
    if cfg.precision == "fp64" and native:
        peak_tf = sms * FP64_FMA_PER_CLK_SM * 2 * clk * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": algo_flops / avg_s / 1e12, "peak": peak_tf,
                "unit": "TFLOP/s", "frac": algo_flops / avg_s / 1e12 / peak_tf,
                "traffic": traffic, "kernel": f"sweep_{kind}",
                "peak_source": f"FP64 FMA units x max SM clock ({sms} SMs x 2 FMA x 2 flop)",
                "hbm": hbm}
    else:
        roof = {"bound": "hbm", "achieved": hbm["achieved"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": hbm["frac"], "traffic": traffic, "kernel": f"sweep_{kind}",
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}
    roof["avg_launch_ms"] = ms / cnt
    roof["per_kernel_ms_per_step"] = per_kernel
    return roof


def run_forward(w, steps, warmup, world, local, sample_clocks=True):
    import torch

    from paper_1803_02143_gb300 import Sldg

    s = Sldg(w.cfg)
    s.set_initial(w.kind, w.params)
    W0 = s.step(warmup, history=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if sample_clocks else None
    barrier(world)
    torch.cuda.synchronize()
    # CUDA events around every kernel launch on the context's stream, inside
    # the timed region (the steps then run as eager launches)
    s.timing(True)
    n0 = s.launch_count
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    W1 = s.step(steps, history=True)  # W of every step to a device slot, one read at the end
    e1.record(s.stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    timing = s.timing_read()
    launches = s.launch_count - n0
    s.timing(False)
    ck = clocks.stop() if clocks else None
    return s, ms, timing, launches, ck, np.concatenate([W0, W1])


def run_splitting_variants(args, w, flags, local):
    """Step time of the same workload and precision with merged drifts (one x
    pass per step instead of two) and with the order-4 triple jump (three
    Strang sub-steps per step), merged or not (a few steps each)."""
    import torch

    from paper_1803_02143_gb300 import _native as N
    from paper_1803_02143_gb300 import configs

    out = {}
    steps = max(2, min(args.steps, 5))
    for name, fl in (("strang_merged", N.SLDG_FLAG_MERGE_DRIFTS), ("order4", N.SLDG_FLAG_ORDER4),
                     ("order4_merged", N.SLDG_FLAG_ORDER4 | N.SLDG_FLAG_MERGE_DRIFTS)):
        w3 = configs.workload(args.workload, w.cfg.precision, flags | fl)
        s3, ms3, _, _, _, _ = run_forward(w3, steps, 1, 1, local, sample_clocks=False)
        s3.close()
        del s3
        torch.cuda.empty_cache()
        out[name] = {"ms_per_step": ms3 / steps, "steps": steps,
                     "value": w3.cfg.numel * steps / (ms3 / 1e3), "unit": UNIT}
    return out


def w_error(W, Wref, dt, t0_step=1):
    """FP32 against FP64: the largest difference of the electric-energy
    histories relative to the largest |W| of the reference, and the
    relative difference at each step with its time."""
    W, Wref = np.asarray(W), np.asarray(Wref)
    rel = np.abs(W - Wref) / np.maximum(np.abs(Wref), 1e-300)
    return {"W_max_rel": float(np.abs(W - Wref).max() / np.abs(Wref).max()),
            "steps": int(W.size),
            "t": [round(dt * (t0_step + m), 6) for m in range(W.size)],
            "W_rel_per_step": [float(x) for x in rel]}


def run_variant(args, name, prec, flags, local, pk, pk_src, sms, steps=None, warmup=None):
    """One more workload or storage precision, timed like the headline run;
    returns its line entry and its W history."""
    import torch

    from paper_1803_02143_gb300 import configs

    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    w2 = configs.workload(name, prec, flags)
    s2, ms2, t2, _, _, W2 = run_forward(w2, steps, warmup, 1, local, sample_clocks=False)
    s2.close()
    del s2
    torch.cuda.empty_cache()
    entry = {"workload": w2.name, "dtype": arithmetic(w2.cfg), "dofs": w2.cfg.numel,
             "value": w2.cfg.numel * steps / (ms2 / 1e3), "unit": UNIT,
             "ms_per_step": ms2 / steps, "steps": steps,
             "roofline": sweep_roofline(w2, t2, steps, pk, pk_src, sms)}
    return entry, W2


def run_e2e(s, w, steps):
    """Through the C ABI with host buffers: every step uploads its input
    state from pinned host memory and reads its W back
    (sldg_step_host_batches, which overlaps the upload of step k+1 with
    step k)."""
    import torch

    host = torch.empty(s.cfg.shape, dtype=s.cfg.dtype, pin_memory=True)
    s.get_f(host)
    s.step_host_batches(host, 2)  # warm
    torch.cuda.synchronize()
    # the host link's rate right now: one plain upload of the same buffer
    # (f already holds these values); the steps cannot run faster than
    # their uploads
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.f.copy_(host, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    esize = 8 if s.cfg.precision == "fp64" else 4
    up_bytes = s.cfg.numel * esize
    t0 = time.perf_counter()
    W = s.step_host_batches(host, steps)
    t1 = time.perf_counter()
    return {"value": s.cfg.numel * steps / (t1 - t0), "unit": UNIT,
            "h2d_bytes_per_step": up_bytes, "d2h_bytes_per_step": 8,
            "ms_per_step": 1e3 * (t1 - t0) / steps, "steps": steps,
            "h2d_gbps_copy_alone": up_bytes / (e0.elapsed_time(e1) * 1e6),
            "h2d_gbps_in_steps": up_bytes * steps / ((t1 - t0) * 1e9),
            "last_W": float(W[-1])}


def run_adjoint_ratio():
    """Adjoint/forward wall ratio on the adjoint workload (32^4, degree 1, 100
    steps, checkpoint every 10): record+backward vs a plain forward, each
    timed after an untimed pass of all three."""
    import torch

    from paper_1803_02143_gb300 import Sldg, configs

    w = configs.workload("adjoint_landau_32")
    s = Sldg(w.cfg)
    # one untimed pass of each phase: tables, replay graphs and the
    # recording's and backward's buffers exist before the timed passes
    s.set_initial(w.kind, w.params)
    s.step(w.steps)
    s.set_initial(w.kind, w.params)
    s.record(w.steps, w.ckpt)
    s.backward()
    torch.cuda.synchronize()
    s.set_initial(w.kind, w.params)
    t0 = time.perf_counter()
    s.step(w.steps)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    s.set_initial(w.kind, w.params)
    t0 = time.perf_counter()
    s.record(w.steps, w.ckpt)
    t_rec = time.perf_counter() - t0
    t0 = time.perf_counter()
    J, _ = s.backward()
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    s.close()
    return {"workload": w.name, "forward_s": t_fwd, "record_s": t_rec, "backward_s": t_bwd,
            "adjoint_forward_ratio": (t_rec + t_bwd) / t_fwd, "J": J}


def run_ours(args, world, rank, local):
    import torch

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        from paper_1803_02143_gb300 import build as B

        B.build()
    barrier(world)
    from paper_1803_02143_gb300 import configs

    flags = 1 if args.native_fp64 else 0
    w = configs.workload(args.workload, args.precision, flags)
    pk, pk_src = peaks()
    sms = device_sms()
    s, ms, timing, launches, clocks, W = run_forward(w, args.steps, args.warmup, world, local)
    ms_max = max_over_ranks(ms, world)
    value = job_value(w.cfg.numel, args.steps, world, ms_max)
    roof = sweep_roofline(w, timing, args.steps, pk, pk_src, sms)
    e2e = None
    if not args.no_e2e:
        barrier(world)
        try:
            e2e = run_e2e(s, w, max(3, min(args.steps, 10)))
            ms_e2e = max_over_ranks(e2e["ms_per_step"] * e2e["steps"], world)
            e2e["value"] = job_value(w.cfg.numel, e2e["steps"], world, ms_e2e)
            e2e["ms_per_step"] = ms_e2e / e2e["steps"]
        except (RuntimeError, MemoryError) as exc:  # pinned host memory for f not available
            e2e = {"value": None, "unit": UNIT, "error": str(exc).splitlines()[0][:200]}
    s.close()
    del s
    torch.cuda.empty_cache()
    extras = {}
    if not args.no_extras and rank == 0:
        times = {}
        if w.cfg.precision == "fp64" and not flags:
            # FP32 storage of the same workload, with its W history against
            # this run's; FP64 storage swept with FP64 FMA
            e32, W32 = run_variant(args, w.name, "fp32", 0, local, pk, pk_src, sms)
            e32["error_vs_fp64"] = w_error(W32, W, w.cfg.dt)
            extras["fp32"] = e32
            times["fp32"] = e32["ms_per_step"]
            efma, Wfma = run_variant(args, w.name, "fp64", 1, local, pk, pk_src, sms,
                                     steps=max(2, min(args.steps, 10)), warmup=1)
            n = min(len(Wfma), len(W))
            efma["double_float_vs_fp64_fma"] = {
                "W_max_rel": float(np.abs(W[:n] - Wfma[:n]).max() / np.abs(Wfma[:n]).max()),
                "steps": n}
            extras["fp64_fma"] = efma
            extras["fp32_over_fp64_step_time"] = times["fp32"] / (ms / args.steps)
        elif w.cfg.precision == "fp32":
            e64, W64 = run_variant(args, w.name, "fp64", 0, local, pk, pk_src, sms)
            extras["fp64"] = e64
            extras["error_vs_fp64"] = w_error(W, W64, w.cfg.dt)
            extras["fp32_over_fp64_step_time"] = (ms / args.steps) / e64["ms_per_step"]
        # the large mixed-precision workload (128^4 cells, degree 1, FP32
        # storage) and its FP64-storage twin
        if w.name != "mixed_landau_128":
            m32, Wm32 = run_variant(args, "mixed_landau_128", "fp32", 0, local, pk, pk_src, sms)
            m64, Wm64 = run_variant(args, "mixed_landau_128", "fp64", 0, local, pk, pk_src, sms)
            m32["error_vs_fp64"] = w_error(Wm32, Wm64, configs.workload("mixed_landau_128").cfg.dt)
            m32["error_vs_fp64"].pop("W_rel_per_step")
            m32["error_vs_fp64"].pop("t")
            m32["fp64_storage"] = {k: m64[k] for k in ("dtype", "value", "unit", "ms_per_step")}
            m32["fp32_over_fp64_step_time"] = m32["ms_per_step"] / m64["ms_per_step"]
            extras["mixed_landau_128"] = m32
        extras["adjoint"] = run_adjoint_ratio()
        extras["splitting"] = run_splitting_variants(args, w, flags, local)
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle as orc

        orc.build()
        cpu = time_oracle(w, nsteps=5)
        cpu["host"] = cpu_info()
    if rank != 0:
        return
    fb = w.cfg.numel * (8 if w.cfg.precision == "fp64" else 4)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": arithmetic(w.cfg), "data": "synthetic",
        "config": {"workload": w.name, "cells": list(w.cfg.ncell), "degree": w.cfg.degree,
                   "storage": w.cfg.precision, "arithmetic": arithmetic(w.cfg),
                   "dofs": w.cfg.numel, "dt": w.cfg.dt, "initial": list(w.params),
                   "l2": "inputs larger than L2 (f is %.1f GB), no flush" % (fb / 1e9),
                   "parallelism": f"replicas x{world}", "sms": sms},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.ingest_ncu:
        ingest_ncu(args)
        return
    if args.summarize_launches:
        summarize_launches(args.summarize_launches)
        return
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
