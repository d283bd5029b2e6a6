#!/usr/bin/env python
"""Benchmark of the block-hydro packet path; prints one JSON line.

Default workload (one bench step): 3D Sedov blast on 256^3 cells as 4096
blocks of 16^3 interior cells (+2 guard layers), FP64, in packets of
seed-uniform 1..256 blocks, 10 time steps: pack the initial state into the
padded layout, form dt, then one persistent launch per time step over every
packet (halo gather, hydro task, fused dt reduction), and unpack the result.
Metric: zone-updates/s (interior cells x time steps / s). The line also
carries the serving latency (p50/p99 per request) of a Poisson request
stream through the continuous-batching server and through plain
per-request launches; for the FP64 workloads, the same workload's rate in
the task's other arithmetics ('variants': double-word flux, which is held to
the FP64 parity rule, and the two FP32-flux forms) and, beside the CPU
baseline, every cell's parity against the oracle's state after the same
number of steps for the FP64 and double-word tasks ('parity').

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload sedov256_uneven|sedov128|sedov128_f32|sedov128_f32x|sedov128_ff|sedov256_uneven_ff|
                     sedov128_rk2|sedov128_rk2_f32|sedov128_rk2_ff|sedov128_tb2|sedov128_tb2_f32|
                     sedov128_rk2_fused|sedov128_rk2_fused_f32|sedov128_amr]
                    [--no-cpu-baseline] [--no-serving] [--no-variants] [--serve-requests N]

Multi-GPU (torchrun, one rank per GPU): each rank runs an independent replica
of the workload (the path has no exchange step between replicas); `value` is
the sum over ranks of the zone updates divided by the slowest rank's time.
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
sys.path.insert(0, ROOT)

# FP64 operations of the scheme per 3D zone update, counted from its
# definition with each face flux, face difference and primitive conversion
# once per zone (add, sub, mul, div, sqrt each 1): primitives 12, slopes 15,
# predictor 64, face states 45, HLL 3 x 86, update 45, signal speed 23.
FLOPS_PER_ZONE_3D = 462
# A Heun RK2 step: two plain-MUSCL stages (primitives 12, slopes 15, face
# states 45, HLL 3 x 86, update 45 each), the signal speed once (23) and the
# stage combination 0.5 (U + U*) (10).
FLOPS_PER_ZONE_3D_RK2 = 2 * (12 + 15 + 45 + 3 * 86 + 45) + 23 + 10
BYTES_PER_ZONE_3D_RK2_STEP = 200         # stage 1: 40 B in + 40 B out; stage 2: 80 B in + 40 B out
BYTES_PER_ZONE_3D = 80        # read U^n and write U^{n+1}: 5 vars x 8 B x 2
FP64_PEAK_TFLOPS = 148 * 2 * 2.032e9 / 1e12    # 2 FP64 lanes / SM / clock at 2032 MHz, non-FMA ops


# the headers every hydro kernel is compiled from; a summary adds the files of
# its own kernels (fused.cuh, amr.cu) on a `kernel_sources:` line
KERNEL_SOURCES = ["common.cuh", "hydro.cuh", "persistent.cuh", "dword.cuh", "softfp64.cuh"]


def kernel_source_hash(extra=()) -> str:
    """sha256 over the code of KERNEL_SOURCES plus `extra` (file names under
    csrc/): comments and whitespace are removed first, so editing a comment
    does not void a recorded capture."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in list(KERNEL_SOURCES) + list(extra):
        src = open(os.path.join(ROOT, "paper_2507_09337_b300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def profiled_traffic(profile_md: str, kernel: str):
    """DRAM bytes per launch from a committed ncu summary, or None if the
    summary covers no capture of this kernel variant or the kernel code
    changed since the captures (hash mismatch). The summary's indented
    machine-readable lines hold one kernel_source_sha256, optionally one
    `kernel_sources:` line (comma-separated extra files the hash covers),
    and one or more `kernel:` lines, each followed by its
    traffic_bytes_per_launch."""
    path = os.path.join(ROOT, "profiles", profile_md)
    if not os.path.exists(path):
        return None
    sha, extra, traffic, current = None, (), {}, None
    for line in open(path):
        if ":" in line and line.startswith("    "):
            k, v = (t.strip() for t in line.strip().split(":", 1))
            if k == "kernel_source_sha256":
                sha = v
            elif k == "kernel_sources":
                extra = tuple(t.strip() for t in v.split(",") if t.strip())
            elif k == "kernel":
                current = v
            elif k == "traffic_bytes_per_launch" and current is not None:
                traffic[current] = float(v)
    if sha != kernel_source_hash(extra):
        return None
    return traffic.get(kernel)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sedov256_uneven", choices=sorted(WORKLOADS))
    ap.add_argument("--tile", default="", choices=["", "8x8", "16x8", "16x16"],
                    help="column tile of the hydro kernel (default: the autotuner's choice)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-latency leg")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the other arithmetics of the FP64 workload (reported under 'variants')")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rates", default="1000,50000",
                    help="arrival rates (requests/s) of the serving leg: one below and one above saturation")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="host threads of the oracle in the reference arm (0: all)")
    return ap.parse_args()


WORKLOADS = {       # name -> (mesh, task, Heun steps at CFL 0.4)
    "sedov256_uneven": ("256", "fp64", False), "sedov256_uneven_ff": ("256", "ff", False),
    "sedov128": ("128", "fp64", False), "sedov128_f32": ("128", "f32flux", False),
    "sedov128_f32x": ("128", "f32flux_ffsum", False), "sedov128_ff": ("128", "ff", False),
    "sedov128_rk2": ("128", "rk2", True), "sedov128_rk2_f32": ("128", "rk2_f32", True),
    "sedov128_rk2_ff": ("128", "rk2_ff", True),
    "sedov128_tb2": ("128", "tb2", False), "sedov128_tb2_f32": ("128", "tb2_f32", False),
    "sedov128_rk2_fused": ("128", "rk2_fused", True), "sedov128_rk2_fused_f32": ("128", "rk2_fused_f32", True),
    "sedov128_amr": ("128", "amr", False),
}


def workload(name):
    from paper_2507_09337_b300 import workloads as wl
    size, task, rk = WORKLOADS[name]
    if size == "128":
        spec, packets = wl.sedov128_packets(64)
        desc = "3D Sedov 128^3, 512 blocks of 16^3 + 2 guards, packets of 64, 10 steps"
    else:
        spec, packets = wl.sedov256_uneven_packets(0)
        desc = "3D Sedov 256^3, 4096 blocks of 16^3 + 2 guards, packets seed-uniform in [1, 256], 10 steps"
    nt = 10
    if rk:
        import dataclasses
        spec = dataclasses.replace(spec, cfl=0.4)
        desc += "; Heun RK2 steps (two plain-MUSCL stages), CFL 0.4"
    if task.startswith("tb2"):
        desc += "; two Hancock steps per launch at the pair's first dt (5 launches)"
    if "fused" in task:
        desc += "; both Heun stages in one launch"
    return spec, packets, nt, task, desc


DTYPES = {"fp64": "f64", "f32flux": "f32 reconstruction/flux + f64 flux differences, update and signal speed",
          "f32flux_ffsum": "f32 reconstruction/flux + float-float flux sums + f64 update (f32 signal speed)",
          "ff": "double-word f32x2 reconstruction/flux + f64 update", "rk2": "f64",
          "rk2_f32": "f32 reconstruction/flux + f64 flux differences and update (Heun RK2)",
          "rk2_ff": "double-word f32x2 reconstruction/flux + f64 update (Heun RK2)",
          "tb2": "f64", "tb2_f32": "f32 reconstruction/flux + f64 flux differences, update and signal speed",
          "rk2_fused": "f64", "rk2_fused_f32": "f32 reconstruction/flux + f64 flux differences and update (Heun RK2)"}
FTYPES = {"tb2": "rd,false", "tb2_f32": "float,false", "rk2_fused": "rd,true", "rk2_fused_f32": "float,true"}
KTYPES = {"fp64": "rd", "f32flux": "float", "f32flux_ffsum": "float,false,true", "ff": "dw", "rk2": "rd,true", "rk2_f32": "float,true",
          "rk2_ff": "dw,true"}


# ---------------------------------------------------------------- clocks during the timed region

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={','.join(self.FIELDS)}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, p in zip(names, parts[2:]):
                if p.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- replicas: timing over ranks

def max_over_ranks(x: float, device) -> float:
    """The largest x over the ranks of the default process group (x itself
    when there is none): the whole job is as slow as its slowest replica."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units all replicas processed over the slowest
    replica's time."""
    return units_per_rank * world / (ms_max * 1e-3)


# ---------------------------------------------------------------- the oracle on the host cores

def parity_error(G, O, nvar: int) -> float:
    """Largest per-cell difference |g - o| / max(|o|, s_v) over cells and
    variables, s_v the largest |momentum| for the momenta (a plain relative
    error is meaningless where momentum vanishes by symmetry); the FP64 path's
    tolerance is 1e-12."""
    import numpy as np
    mom = float(np.abs(O[:, 1:nvar - 1]).max())
    err = 0.0
    for v in range(nvar):
        scale = np.abs(O[:, v])
        if 0 < v < nvar - 1:
            scale = np.maximum(scale, mom)
        d = np.abs(G[:, v] - O[:, v])
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.where(d == 0, 0.0, d / scale)
        err = max(err, float(np.nanmax(r)))
    return err


def oracle_rate(spec, U0, seconds: float, max_steps: int = 400):
    """Zone-updates/s of the oracle on the full mesh, stepping until `seconds`
    of wall time have passed (at least one step); also returns the state it
    reached."""
    import oracle
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    m = oracle.Mesh(**spec.oracle_kwargs())
    U = U0.copy()
    t0 = time.perf_counter()
    n = 0
    while True:
        U, _, _ = oracle.step(m, U, oracle.dt(m, U))
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or n >= max_steps:
            break
    return spec.zones * n / el, threads, n, el, U


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2507_09337_b300 import workloads as wl
    if args.workload == "sedov128_amr":
        return run_reference_amr(args)
    spec, packets, nt, task, desc = workload(args.workload)
    U0 = wl.sedov_state(spec)
    import oracle
    threads = args.cpu_threads or os.cpu_count() or 1
    oracle.set_threads(threads)
    m = oracle.Mesh(**spec.oracle_kwargs())
    U = U0.copy()
    step = oracle.step_rk2 if task.startswith("rk2") else oracle.step
    for _ in range(args.warmup):
        U, _, _ = step(m, U, oracle.dt(m, U))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, _, _ = step(m, U, oracle.dt(m, U))
    el = time.perf_counter() - t0
    value = spec.zones * args.steps / el
    sample = f"{args.steps} time steps (1 per bench step) of the full {spec.zones}-zone mesh, FP64"
    line = {
        "impl": "reference", "metric": "zone-updates/s", "value": value, "unit": "zone-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc + " (reference arm: one time step per bench step)"},
        "cpu_baseline": {"value": value, "unit": "zone-updates/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- other arithmetics on the same workload

VARIANTS = ("ff", "f32flux", "f32flux_ffsum")


def run_variants(B, mesh, spec, nt, U0_dev, stream, steps, dev):
    """The same workload, device-resident and timed the same way, in the other
    arithmetics of the hydro task: double-word flux (held to the FP64 parity
    rule), FP32 flux in the configured arithmetic, and the FP32-flux shortcut."""
    import torch
    out = {}
    h = mesh.handle
    for name in VARIANTS:
        task = B.TASKS[name]
        tile = B.orcha_autotune(spec.ndim, spec.bs, task, nblocks=spec.nblocks)
        bt = B.orcha_batch_create(mesh.packets, tile[0], tile[1])

        def one():
            B.orcha_mesh_load(h, U0_dev.data_ptr(), False, stream)
            B.orcha_batch_advance(bt, task, 0, True, False, stream)
            for _ in range(nt):
                B.orcha_batch_advance(bt, task, 1, False, False, stream)

        with torch.cuda.stream(stream):
            one()                                   # warm-up
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                one()
            e1.record(stream)
        stream.synchronize()
        assert mesh.poll(stream) == 0
        B.orcha_batch_destroy(bt)
        out[name] = {"value": spec.zones * nt * steps / (e0.elapsed_time(e1) * 1e-3), "unit": "zone-updates/s",
                     "dtype": DTYPES[name], "tile": f"{tile[0]}x{tile[1]}"}
    return out


def gpu_state_after(B, mesh, spec, task_name, U0_dev, stream, nsteps):
    """The state after nsteps of task_name from the initial state (CFL dt from
    it), through the persistent path, copied to the host."""
    import torch
    task = B.TASKS[task_name]
    tile = B.orcha_autotune(spec.ndim, spec.bs, task, nblocks=spec.nblocks)
    bt = B.orcha_batch_create(mesh.packets, tile[0], tile[1])
    out = torch.empty_like(U0_dev)
    with torch.cuda.stream(stream):
        B.orcha_mesh_load(mesh.handle, U0_dev.data_ptr(), False, stream)
        B.orcha_batch_advance(bt, task, nsteps, True, False, stream)
        B.orcha_mesh_store(mesh.handle, out.data_ptr(), False, stream)
    stream.synchronize()
    assert mesh.poll(stream) == 0
    B.orcha_batch_destroy(bt)
    return out.cpu().numpy()


# ---------------------------------------------------------------- serving latency

def serving_latency(args):
    """p50/p99 request latency and zone-updates/s of a Poisson stream of
    serving requests (K ~ U[1, 512] blocks of 8^3/16^3/32^3, one step each,
    FP32 flux, 64 GB pool) at one rate the GPU keeps up with and one above
    saturation, through the continuous-batching server and through plain
    per-request launches (a mesh, a packet and per-step launches each)."""
    from paper_2507_09337_b300 import binding as B
    from paper_2507_09337_b300 import serve
    from paper_2507_09337_b300 import workloads as wl
    task = B.ORCHA_TASK_HYDRO_F32FLUX
    base = wl.serving_stream(args.serve_requests, 1.0)
    out = {"requests": args.serve_requests, "task": "f32flux", "budget_gb": 64,
           "workload": "Poisson arrivals; K ~ U[1, 512] blocks of 8^3, 16^3 or 32^3; Sedov-like or Sod-like; "
                       "1 step each; latency = completion - submission", "rates": []}
    for rate in [float(r) for r in args.serve_rates.split(",")]:
        stream = [(t / rate, req) for t, req in base]
        srv = serve.run_server(stream, task, 64 * 10 ** 9)
        pln = serve.run_plain(stream, task)
        out["rates"].append({
            "rate_per_s": rate,
            "server": {"p50_ms": srv["p50_ms"], "p99_ms": srv["p99_ms"], "zone_updates_per_s": srv["zone_updates_per_s"],
                       "pool_peak_gb": srv["pool_peak_gb"]},
            "plain": {"p50_ms": pln["p50_ms"], "p99_ms": pln["p99_ms"], "zone_updates_per_s": pln["zone_updates_per_s"]},
        })
    return out


# ---------------------------------------------------------------- two-level AMR workload

def amr_workload():
    """Sedov 128^3 coarse (512 blocks of 16^3) with the 32 blocks whose
    centres lie within 0.25 of the blast refined (256 fine blocks of half the
    cell width); the initial state is the blast on the fine grid, averaged
    onto the coarse one."""
    from paper_2507_09337_b300 import workloads as wl
    spec, _ = wl.sedov128_packets(64)
    refined = wl.refined_blocks(spec, "sphere", 0.25)
    U0, U1 = wl.amr_split(spec, refined, wl.sedov_state(wl.fine_spec(spec)))
    nleaf = (spec.nblocks - len(refined) + (len(refined) << 3)) * spec.bs[0] * spec.bs[1] * spec.bs[2]
    desc = ("two-level AMR: 3D Sedov, coarse 128^3 as 512 blocks of 16^3 + 2 guards, the 32 central blocks "
            "refined into 256 fine blocks of half the cell width, 10 steps, one dt for both levels, flux correction")
    return spec, refined, U0, U1, nleaf, desc


def run_amr(args):
    import torch
    from paper_2507_09337_b300 import binding as B
    from paper_2507_09337_b300 import build as pkgbuild
    pkgbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spec, refined, U0, U1, nleaf, desc = amr_workload()
    nt = 10
    amr = B.AmrMesh(spec, refined)
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    events = []

    def step(record):
        amr.load(U0, U1)
        B.orcha_amr_advance(amr.handle, 0, True, stream)
        for _ in range(nt):
            if record:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                B.orcha_amr_advance(amr.handle, 1, False, stream)
                e1.record(stream)
                events.append((e0, e1))
            else:
                B.orcha_amr_advance(amr.handle, 1, False, stream)
        stream.synchronize()

    for _ in range(args.warmup):
        step(False)
    assert amr.poll(stream) == 0
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.steps):
        step(True)
    clk = clocks.stop()
    assert amr.poll(stream) == 0
    ms = sum(a.elapsed_time(b) for a, b in events)
    value = nleaf * len(events) / (ms * 1e-3)
    fp64_peak = B.orcha_measure_fp64_rate(0) / 1e12
    achieved = FLOPS_PER_ZONE_3D * value / 1e12
    # end to end: host state in, nt steps, host state out, per bench step
    t0 = time.perf_counter()
    for _ in range(args.steps):
        amr.load(U0, U1)
        B.orcha_amr_advance(amr.handle, nt, True, stream)
        stream.synchronize()
        amr.store()
    e2e = nleaf * nt * args.steps / (time.perf_counter() - t0)
    line = {
        "metric": "zone-updates/s", "value": value, "unit": "zone-updates/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "leaf_zones_per_step": nleaf, "refined_blocks": int(len(refined)),
                   "timed": "device time of the advance calls (events), per step: coarse and fine guard fill, "
                            "hydro of every leaf, flux correction, restriction, dt"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak, "traffic": None, "ops_per_zone_update": FLOPS_PER_ZONE_3D,
                     "kernel": "whole two-level step (amr_hydro_kernel<3,16,16> dominant)",
                     "peak_source": "measured FP64 FMA throughput probe (orcha_measure_fp64_rate)"},
        "clocks": clk,
        "e2e": {"value": e2e, "unit": "zone-updates/s", "h2d_bytes_per_step": int(U0.nbytes + U1.nbytes),
                "d2h_bytes_per_step": int(U0.nbytes + U1.nbytes),
                "api": "orcha_amr_load(host) + orcha_amr_advance + orcha_amr_store(host), wall clock"},
        # per step: coarse guard fill, fine guard fill, hydro of both levels,
        # flux correction, restriction, two signal-speed launches, dt reduction
        "gpu_launches": len(events) * 8,
    }
    if not args.no_cpu_baseline:
        import oracle
        oracle.set_threads(os.cpu_count() or 1)
        m = oracle.Mesh(**spec.oracle_kwargs())
        t0 = time.perf_counter()
        oracle.amr_run(m, refined, U0, U1, 2)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": nleaf * 2 / el, "unit": "zone-updates/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": f"2 two-level steps of the full mesh in {el:.1f} s"}
    amr.close()
    print(json.dumps(line))
    return 0


def run_reference_amr(args):
    """The oracle's two-level step on the AMR workload, one step per bench step."""
    import oracle
    spec, refined, U0, U1, nleaf, desc = amr_workload()
    threads = args.cpu_threads or os.cpu_count() or 1
    oracle.set_threads(threads)
    m = oracle.Mesh(**spec.oracle_kwargs())
    A0, A1, _ = oracle.amr_run(m, refined, U0, U1, args.warmup)
    t0 = time.perf_counter()
    oracle.amr_run(m, refined, A0, A1, args.steps)
    el = time.perf_counter() - t0
    value = nleaf * args.steps / el
    line = {"impl": "reference", "metric": "zone-updates/s", "value": value, "unit": "zone-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc + " (reference arm: one step per bench step)"},
            "cpu_baseline": {"value": value, "unit": "zone-updates/s", "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} two-level steps of the full mesh"},
            "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- our arm

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "sedov128_amr":
        return run_amr(args)

    import torch
    import torch.distributed as dist
    from paper_2507_09337_b300 import binding as B
    from paper_2507_09337_b300 import build as pkgbuild
    from paper_2507_09337_b300 import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        pkgbuild.build()
    if world > 1:
        dist.barrier()

    spec, packets, nt, task_name, desc = workload(args.workload)
    task = B.TASKS[task_name]
    U0_host = wl.sedov_state(spec)
    dev = torch.device("cuda", local)
    U0_dev = torch.from_numpy(U0_host).to(dev)
    out_dev = torch.empty_like(U0_dev)
    mesh = B.Mesh(spec, device=f"cuda:{local}", packets=packets)
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))   # buffers were set up on the current stream
    npk = len(mesh.packets)
    h = mesh.handle
    # tile shape picked by the autotuner (cached per GPU and geometry; outside
    # the timed region), or the one --tile names
    if args.tile:
        tx, ty = (int(v) for v in args.tile.split("x"))
        tile = (tx, ty, float("nan"))
    else:
        tile = B.orcha_autotune(spec.ndim, spec.bs, task, nblocks=spec.nblocks)
    batch = B.orcha_batch_create(mesh.packets, tile[0], tile[1])
    hydro_events = []
    # time steps per batch call (a two-step task advances a pair per launch)
    per_call = 2 if task_name.startswith("tb2") else 1
    launches_per_call = 2 if task_name in ("rk2", "rk2_f32", "rk2_ff") else 1
    # per bench step: pack, signal speed (one launch), dt reduce, the hydro launches, unpack
    launches_per_step = 1 + 1 + 1 + (nt // per_call) * launches_per_call + 1

    def step(record: bool):
        B.orcha_mesh_load(h, U0_dev.data_ptr(), False, stream)
        B.orcha_batch_advance(batch, task, 0, True, False, stream)          # dt of the initial state
        for _ in range(nt // per_call):
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                B.orcha_batch_advance(batch, task, per_call, False, False, stream)
                e1.record(stream)
                hydro_events.append((e0, e1, spec.nblocks * per_call))
            else:
                B.orcha_batch_advance(batch, task, per_call, False, False, stream)
        B.orcha_mesh_store(h, out_dev.data_ptr(), False, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(False)
    stream.synchronize()
    assert mesh.poll(stream) == 0

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            step(True)
        ev1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, dev)
    assert mesh.poll(stream) == 0

    zone_updates = spec.zones * nt * args.steps * world
    value = job_rate(spec.zones * nt * args.steps, world, ms_max)

    # dominant kernel: the hydro task, timed per launch on its own stream
    durs = [(a.elapsed_time(b) * 1e-3, nblk) for a, b, nblk in hydro_events]
    zones_per_block = spec.bs[0] * spec.bs[1] * spec.bs[2]
    tot_s = sum(d for d, _ in durs)
    tot_zones = sum(n for _, n in durs) * zones_per_block
    avg_launch_s = tot_s / len(durs)
    zones_per_launch = tot_zones / len(durs)
    hydro_share = tot_s / (ms * 1e-3)
    # per zone update: the roof that bounds the task and its algorithmic
    # FP64 operations and HBM bytes (a Heun step in two launches moves 200 B,
    # in one launch 80 B; a two-step launch reads and writes once per pair)
    ops_zu, bytes_zu = {"rk2": (FLOPS_PER_ZONE_3D_RK2, 200), "rk2_fused": (FLOPS_PER_ZONE_3D_RK2, 80),
                        "rk2_f32": (0, 200), "rk2_ff": (0, 200), "rk2_fused_f32": (0, 80),
                        "tb2": (FLOPS_PER_ZONE_3D, 40), "tb2_f32": (0, 40)}.get(task_name, (FLOPS_PER_ZONE_3D, 80))
    fp64_bound = task_name in ("fp64", "rk2", "rk2_fused", "tb2")
    hbm_peak, hbm_src = 6400.0, "fallback 6.4 TB/s (MEASURED_PEAKS.json absent)"
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        hbm_src = "measured copy bandwidth (MEASURED_PEAKS.json)"
    fused = task_name.startswith("tb2") or "fused" in task_name
    kname = (f"fused_kernel<3,{tile[0]},{tile[1]},{FTYPES[task_name]}>" if fused else
             f"persistent_kernel<3,{tile[0]},{tile[1]},{KTYPES[task_name]}>")
    prof = {"sedov128": "persistent_kernel_fp64_sedov128.md",
            "sedov256_uneven": "persistent_kernel_fp64_sedov256.md",
            "sedov128_rk2": "persistent_kernel_rk2_sedov128.md",
            "sedov128_f32": "persistent_kernel_f32flux_sedov128.md",
            "sedov128_ff": "persistent_kernel_ff_sedov128.md",
            "sedov128_tb2_f32": "fused_kernel_sedov128.md", "sedov128_tb2": "fused_kernel_sedov128.md",
            "sedov128_rk2_fused": "fused_kernel_sedov128.md"}.get(args.workload)
    traffic = profiled_traffic(prof, kname) if prof else None
    per_launch = {"rk2": "one time step of all packets (two stage launches)",
                  "rk2_f32": "one time step of all packets (two stage launches)",
                  "rk2_ff": "one time step of all packets (two stage launches)",
                  "tb2": "two time steps of all packets", "tb2_f32": "two time steps of all packets"}.get(
        task_name, "one time step of all packets")
    if fp64_bound:
        # the FP64 pipe bounds this task: its peak is measured here, on this
        # GPU, by the library's FMA throughput probe (lane operations/s)
        fp64_peak = B.orcha_measure_fp64_rate(0) / 1e12
        achieved = ops_zu * zones_per_launch / avg_launch_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": traffic, "kernel": kname, "per_launch": per_launch,
                "ops_per_zone_update": ops_zu,
                "peak_source": "measured: FP64 FMA throughput probe (orcha_measure_fp64_rate) on this GPU, "
                               "lane operations/s; the task's operations are counted in the same unit "
                               f"(nominal 2 lanes/SM/clk x 148 SMs x 2032 MHz = {FP64_PEAK_TFLOPS:.3f} T)"}
    else:
        achieved = bytes_zu * zones_per_launch / avg_launch_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": traffic, "kernel": kname, "peak_source": hbm_src, "per_launch": per_launch,
                "bytes_per_zone_update": bytes_zu}
    hbm_eff = BYTES_PER_ZONE_3D * value / world / 1e9
    spec_state_mb = mesh.state[0].numel() * 8 / 1e6

    # end to end through the public API with host buffers: every step copies its
    # input from pinned host memory and its result back. Three meshes on three
    # streams take turns, so while one computes, another's result copy (D2H)
    # and a third's input copy (H2D) run on the two copy engines at once (the
    # way a caller streams independent problems through the library).
    NLANES = 3
    U0_pin = torch.from_numpy(U0_host).pin_memory()
    out_pin = [torch.empty(U0_host.shape, dtype=torch.float64).pin_memory() for _ in range(NLANES)]
    bytes_io = U0_host.nbytes
    lanes = [(h, batch, stream, out_pin[0])]
    extra = []
    for k in range(1, NLANES):
        mk = B.Mesh(spec, device=f"cuda:{local}", packets=packets)
        bk = B.orcha_batch_create(mk.packets, tile[0], tile[1])
        sk = torch.cuda.Stream(dev)
        sk.wait_stream(torch.cuda.current_stream(dev))
        extra.append((mk, bk))
        lanes.append((mk.handle, bk, sk, out_pin[k]))

    def e2e_step(k):
        hk, bk, sk, ok = lanes[k % NLANES]
        B.orcha_mesh_load(hk, U0_pin.data_ptr(), True, sk)
        B.orcha_batch_advance(bk, task, nt, True, True, sk)
        B.orcha_mesh_store(hk, ok.data_ptr(), True, sk)

    for k in range(NLANES):
        e2e_step(k)
    for lane in lanes:
        lane[2].synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for lane in lanes[1:]:
        lane[2].wait_event(e0)
    for k in range(args.steps):
        e2e_step(k)
    for lane in lanes[1:]:
        done = torch.cuda.Event()
        done.record(lane[2])
        stream.wait_event(done)
    e1.record(stream)
    stream.synchronize()
    e2e_value = job_rate(spec.zones * nt * args.steps, world, max_over_ranks(e0.elapsed_time(e1), dev))
    for (mk, _), lane in zip(extra, lanes[1:]):
        assert mk.poll(lane[2]) == 0
    assert mesh.poll(stream) == 0
    # the e2e runs and the device-resident run computed the same state
    assert all(torch.equal(o, out_dev.cpu()) for o in out_pin)

    line = {
        "metric": "zone-updates/s", "value": value, "unit": "zone-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[task_name], "data": "synthetic",
        "config": {"workload": desc, "task": task_name, "zones_per_step": spec.zones * nt,
                   "tile": (f"{tile[0]}x{tile[1]} (--tile)" if args.tile else
                            f"{tile[0]}x{tile[1]} (autotuned, {tile[2]:.3f} ms/step on the tuning mesh)"),
                   "l2": (f"inputs larger than L2 (two {spec_state_mb:.0f} MB state buffers + "
                          f"{U0_host.nbytes / 1e6:.0f} MB initial state)"),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "hydro_share_of_step": hydro_share,
                   "hbm": {"algorithmic_gbs": hbm_eff, "bytes_per_zone": BYTES_PER_ZONE_3D,
                           "frac_of_measured": hbm_eff / hbm_peak, "measured_gbs": hbm_peak,
                           "frac_of_8tbs": hbm_eff / 8000.0,
                           "target": ">= 0.60 of the 8 TB/s HBM roofline",
                           "target_met": hbm_eff / 8000.0 >= 0.60}},
        "roofline": roof,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "zone-updates/s", "h2d_bytes_per_step": bytes_io,
                "d2h_bytes_per_step": bytes_io, "api": "orcha_mesh_load(host) + orcha_batch_advance(graph) + "
                                                         "orcha_mesh_store(host); three meshes on three streams "
                                                         "take turns so copies overlap compute"},
        "gpu_launches": launches_per_step * args.steps,
    }
    if not args.no_serving:
        line["latency"] = serving_latency(args)
    if task_name == "fp64" and world == 1 and not args.no_variants:
        line["variants"] = run_variants(B, mesh, spec, nt, U0_dev, stream, args.steps, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, n, el, U_oracle = oracle_rate(spec, U0_host, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": "zone-updates/s", "cores": cores, "kind": "oracle",
                                "sample": f"{n} time steps of the full {spec.zones}-zone mesh in {el:.1f} s"}
        if task_name == "fp64":
            # parity at the full size: every cell after the oracle's n steps,
            # against the FP64 task and the double-word one (rule: 1e-12)
            line["parity"] = {"steps": n, "rule": "max over cells |g - o| / max(|o|, largest |momentum| for momenta)",
                              "tolerance": 1e-12}
            for name in ("fp64", "ff"):
                G = gpu_state_after(B, mesh, spec, name, U0_dev, stream, n)
                line["parity"][name] = parity_error(G, U_oracle, spec.nvar)
    B.orcha_batch_destroy(batch)
    for mk, bk in extra:
        B.orcha_batch_destroy(bk)
        mk.close()
    mesh.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
