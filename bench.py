#!/usr/bin/env python
"""EBIT step throughput on GB300: cell-updates/s at 4096^2.

Workload: 4096^2 unit square, Fourier-perturbed interface
y = 0.5 + sum_{k<=16} (0.01/k^2) cos(2 pi k x + phi_k) plus 20000 seeded
circles of radius 3-12 cells, steady cellular flow, dt = 0.5 dx.  The headline
is the FP32-fraction form (FP64 circle fit and area sums); the plain FP64 form
is timed beside it.  A step is one full EBIT step: both split sweeps, volume
fractions and height-function curvature.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With N > 1 (torchrun, one rank per GPU) every rank runs its own replica of the
workload (the single grid is not partitioned: replicas only) and the value is
the cell-updates of all ranks over the slowest rank's time.
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

METRIC = "EBIT cell-updates/s at 4096^2 (batched FP32 vs plain FP64), %HBM roofline; p50/p99 step"
UNIT = "cell-updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_bytes_per_cell(kind: str, esz: int) -> float:
    """Algorithmic HBM bytes per cell and launch (dense arrays, each word read
    or written once); K and Z are 1 bit per vertex / cell."""
    bits = 0.125
    return {
        # reads K, Z, sH, sV, velocity; writes K, sH, sV, two verdict bytes
        "sweep": (2 * bits + 3 * esz) + (bits + 2 * esz + 2.0),
        # reads new K, old Z, verdicts; writes Z
        "centre": 2 * bits + 2.0 + bits,
        # reads K, Z, sH, sV; writes C and kappa
        "fields": 2 * bits + 2 * esz + 2 * esz,
        "area": 0.0,
    }[kind]


def step_bytes_per_cell(esz: int) -> float:
    """The fused-step model: state read and written once, u and v read once,
    C and kappa written once (32.5 B/cell FP32, 64.5 B/cell FP64)."""
    return (2 * esz + 0.25) * 2 + 2 * esz + 2 * esz


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def traffic_record(kernel):
    """ncu DRAM bytes per launch for the kernel, if the committed record was
    taken on the current kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None, None
    h = hashlib.sha256()
    for name in sorted(os.listdir(os.path.join(ROOT, "paper_2309_00338_gb300", "csrc"))):
        with open(os.path.join(ROOT, "paper_2309_00338_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    if rec.get("csrc_sha256") != h.hexdigest():
        return None, rec
    k = rec.get("kernels", {}).get(kernel)
    if not k:
        return None, rec
    return k["dram_bytes_per_cell"], rec


def cpu_baseline(wl, budget_s=20.0):
    """The oracle as it stands (FP32-state form, single thread) on whole
    steps of the same workload from its initial state."""
    import oracle
    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, oracle.FP32)
    t0 = time.perf_counter()
    k = 0
    while True:
        oracle.step(S, wl.field.u, wl.field.v, wl.dt)
        k += 1
        if time.perf_counter() - t0 > budget_s or k >= 8:
            break
    t = time.perf_counter() - t0
    return {"value": wl.n * wl.n * k / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{k} whole steps of the {wl.n}^2 workload (FP32 form) from its initial state"}


def run_reference(args, wl, world, rank):
    """The oracle on the host cores, on the same workload, metric and unit."""
    if rank != 0:
        return
    import oracle
    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, oracle.FP32)
    for _ in range(args.warmup):
        oracle.step(S, wl.field.u, wl.field.v, wl.dt)
    t0 = time.perf_counter()
    done = 0
    lat = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        oracle.step(S, wl.field.u, wl.field.v, wl.dt)
        lat.append(time.perf_counter() - t1)
        done += 1
        if time.perf_counter() - t0 > 150.0:
            break
    t = time.perf_counter() - t0
    value = wl.n * wl.n * done / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": wl.name, "grid": [wl.n, wl.n], "prec": "fp32"},
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{done} whole steps of the {wl.n}^2 workload after {args.warmup} warm-up steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(torch, ebit, ctx, u, v, dt, K, stream):
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    ev[0].record(stream)
    for k in range(K):
        ebit.ebit_step(ctx, u, v, dt)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    total = ev[0].elapsed_time(ev[K])
    lat = [ev[k].elapsed_time(ev[k + 1]) for k in range(K)]
    return total, lat


def run_ours(args, wl, world, rank, local):
    import torch
    import torch.distributed as tdist
    from paper_2309_00338_gb300 import ebit

    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            tdist.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        return float(t.item())

    stream = torch.cuda.current_stream()
    n = wl.n
    cells = n * n
    prec = ebit.EBIT_FP32
    ctx = ebit.ebit_init(n, n, wl.dx, wl.scene, prec, stream=stream)
    u = torch.from_numpy(wl.field.u.astype(np.float32)).cuda()
    v = torch.from_numpy(wl.field.v.astype(np.float32)).cuda()
    for _ in range(args.warmup):
        ebit.ebit_step(ctx, u, v, wl.dt)
    ebit.ebit_sync(ctx)
    torch.cuda.synchronize()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    total_ms, lat = timed_steps(torch, ebit, ctx, u, v, wl.dt, args.steps, stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ebit.ebit_sync(ctx)
    total_ms = max_over_ranks(total_ms)
    ms_per_step = total_ms / args.steps
    value = world * cells * args.steps / (total_ms / 1e3)
    diag = ebit.ebit_diagnostics(ctx)

    # per-kernel durations over a second timed region (events around each of
    # the library's launches, on the launching stream)
    ebit.ebit_set_timing(ctx, True)
    ebit.ebit_timings(ctx)
    for _ in range(args.steps):
        ebit.ebit_step(ctx, u, v, wl.dt)
    kt = ebit.ebit_timings(ctx)
    ebit.ebit_set_timing(ctx, False)
    launches_per_step = sum(nl for _, nl in kt.values()) / args.steps
    hbm, peak_kind = peaks()
    esz = 4
    dom = max(kt, key=lambda k: kt[k][0])
    dom_ms = kt[dom][0] / max(1, kt[dom][1])
    dom_bytes = kernel_bytes_per_cell(dom, esz) * cells
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    traffic_cell, _ = traffic_record(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": f"{peak_kind} hbm_gbs (copy)",
                "traffic": None if traffic_cell is None else traffic_cell * cells,
                "algorithmic_bytes": dom_bytes, "avg_launch_ms": dom_ms,
                "kernels": {k: {"ms_per_launch": (t / max(1, nl)), "launches": nl,
                                "share": t / max(1e-12, sum(tt for tt, _ in kt.values())),
                                "GBps": kernel_bytes_per_cell(k, esz) * cells / (t / max(1, nl) / 1e3) / 1e9
                                if t > 0 and k != "area" else None}
                            for k, (t, nl) in kt.items()}}
    step_model = step_bytes_per_cell(esz) * cells
    step_roof = {"bytes_per_cell": step_bytes_per_cell(esz), "achieved_GBps": step_model / (ms_per_step / 1e3) / 1e9,
                 "frac": step_model / (ms_per_step / 1e3) / 1e9 / hbm}

    # end to end through the C ABI with host buffers: every step copies u, v
    # from pinned host memory and reads the step's area back
    hu = torch.from_numpy(wl.field.u.astype(np.float32)).pin_memory()
    hv = torch.from_numpy(wl.field.v.astype(np.float32)).pin_memory()
    du, dv = torch.empty_like(u), torch.empty_like(v)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        du.copy_(hu, non_blocking=True)
        dv.copy_(hv, non_blocking=True)
        ebit.ebit_step(ctx, du, dv, wl.dt)
        ebit.ebit_fraction(ctx)          # area back to the host (synchronises)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t0)))
    e2e = {"value": world * cells * args.steps / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(hu.numel() * 4 + hv.numel() * 4), "d2h_bytes_per_step": 8}
    ebit.ebit_destroy(ctx)

    fp64 = None
    if not args.no_fp64:
        ctx64 = ebit.ebit_init(n, n, wl.dx, wl.scene, ebit.EBIT_FP64, stream=stream)
        u64 = torch.from_numpy(wl.field.u).cuda()
        v64 = torch.from_numpy(wl.field.v).cuda()
        for _ in range(args.warmup):
            ebit.ebit_step(ctx64, u64, v64, wl.dt)
        torch.cuda.synchronize()
        barrier()
        t64, lat64 = timed_steps(torch, ebit, ctx64, u64, v64, wl.dt, args.steps, stream)
        barrier()
        ebit.ebit_sync(ctx64)
        t64 = max_over_ranks(t64)
        sb = step_bytes_per_cell(8) * cells
        fp64 = {"value": world * cells * args.steps / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64 / args.steps,
                "p50_ms": float(np.percentile(lat64, 50)), "p99_ms": float(np.percentile(lat64, 99)),
                "step_roofline_frac": sb / (t64 / args.steps / 1e3) / 1e9 / hbm}
        ebit.ebit_destroy(ctx64)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "dtype_note": "FP32 state and advection; FP64 circle fit and area sums",
                "data": "synthetic",
                "config": {"workload": wl.name, "grid": [n, n], "circles": wl.meta.get("placed"),
                           "curve_modes": 16, "field": "cellular", "cfl": 0.5, "prec": "fp32",
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "working set (~0.45 GB) larger than L2, no flush"},
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "clocks": clk, "e2e": e2e, "gpu_launches": int(round(launches_per_step * args.steps)),
                "roofline": roofline, "step_roofline": step_roof, "fp64": fp64, "cpu_baseline": cpu,
                "markers": {"nH": int(diag["counters"][0]), "nV": int(diag["counters"][1])}}
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist()
    from paper_2309_00338_gb300 import workloads as W
    wl = W.cellular_curve_workload()
    if args.impl == "reference":
        run_reference(args, wl, world, rank)
        return
    run_ours(args, wl, world, rank, local)


if __name__ == "__main__":
    main()
