#!/usr/bin/env python
"""EBIT step throughput on GB300: cell-updates/s at 4096^2.

Workload: 4096^2 unit square, Fourier-perturbed interface
y = 0.5 + sum_{k<=16} (0.01/k^2) cos(2 pi k x + phi_k) plus 20000 seeded
circles of radius 3-12 cells, steady cellular flow, dt = 0.5 dx.  The headline
is the FP32-fraction form (FP64 circle fit and area sums); the plain FP64 form
is timed beside it.  A step is one full EBIT step: both split sweeps, volume
fractions and height-function curvature.  The same line carries the batched
leg (512 uneven grids of 32^2-512^2 in one batch, FP32 and plain FP64, against
plain FP64 one grid at a time) and the serving leg (Poisson arrivals of grids
of 64^2-2048^2 at --leg-rate per second over 10 s, FP32 and plain FP64).

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
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-ghf", action="store_true", help="skip the generalised height-function leg")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batched", action="store_true",
                   help="skip the batched leg (512 uneven grids) of the headline line")
    p.add_argument("--no-serving", action="store_true",
                   help="skip the serving leg (Poisson arrivals at --leg-rate) of the headline line")
    p.add_argument("--leg-rate", type=float, default=50.0,
                   help="arrivals per second of the headline line's serving leg")
    p.add_argument("--record-traffic", nargs="+", metavar="NCU_CSV",
                   help="write profiles/dram_traffic.json from ncu CSV logs of the headline workload and exit")
    p.add_argument("--late-from", type=int, default=1000,
                   help="time a second window from the state after this many steps (0: skip)")
    p.add_argument("--workload", default="cellular_curve_4096",
                   choices=["cellular_curve_4096", "batched", "serving"],
                   help="batched: 512 uneven grids in one batch; serving: Poisson arrivals")
    p.add_argument("--instances", type=int, default=512, help="batched: number of grids")
    p.add_argument("--schedule", type=int, default=-1,
                   help="batched / serving: a fixed ebit_schedule instead of the autotuner's choice")
    p.add_argument("--rate", type=float, default=200.0, help="serving: arrivals per second")
    p.add_argument("--serve-seconds", type=float, default=10.0, help="serving: arrival window")
    p.add_argument("--serve-fp64", action="store_true",
                   help="serving: also serve the same arrivals in plain FP64")
    p.add_argument("--serve-cap", type=float, default=180.0, help="serving: wall-clock cap (s)")
    p.add_argument("--one-at-a-time", type=int, default=64,
                   help="batched: grids of the random sample run one at a time in plain FP64")
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
        # the tiled sweep: reads K, Z, sH, sV and the velocity component,
        # writes K, Z, sH, sV (20.5 B/cell FP32, 40.5 FP64)
        "sweep": (2 * bits + 3 * esz) + (2 * bits + 2 * esz),
        # reads K, Z, sH, sV; writes C and kappa (the area partials and
        # their sum are a few KB)
        "fields": 2 * bits + 2 * esz + 2 * esz,
        # reads C and kappa; writes rho, mu, fx and fy (the face arrays carry
        # one extra column / row, counted exactly in coupling_bytes)
        "coupling": 6 * esz,
    }[kind]


def coupling_bytes(nx: int, ny: int, esz: int) -> int:
    """Algorithmic bytes of one ebit_coupling launch: C and kappa read,
    rho and mu written (ny*nx each), fx ny*(nx+1) and fy (ny+1)*nx written."""
    return esz * (4 * nx * ny + ny * (nx + 1) + (ny + 1) * nx)


# FP64 operations of one crossing candidate of the sweep (two circle fits and
# their mean), counting add, sub, mul, div and sqrt as one each: the chord's
# end points and offsets (8), per circle the third point (1.5), its offsets
# from both ends (10), the implicit-circle coefficients (9), c0 (3), the
# discriminant (4), sqrt (1), h (2), the near root (1), its side test (3) and
# the shift back to the edge (1), and the mean (2).
FIT_OPS = 8 + 2 * (1.5 + 10 + 9 + 3 + 4 + 1 + 2 + 1 + 3 + 1) + 2
# FP64 rate of a GB300 SM: one warp instruction per 16 cycles (2 lanes/clock,
# 1/64 of the FP32 rate), over 152 SMs.
FP64_OPS_PER_CLOCK = 2 * 152


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
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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


# the sources each kernel is compiled from (its own header and the device
# code it shares); a traffic record is valid while these are unchanged
KERNEL_SOURCES = {
    "sweep": ["ebit_tile.cuh", "ebit_device.cuh"],
    "fields": ["ebit_fields.cuh", "ebit_device.cuh"],
    "coupling": ["ebit_coupling.cuh", "ebit_device.cuh"],
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2309_00338_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def record_traffic(paths, cells, workload, command):
    """Writes profiles/dram_traffic.json from ncu CSV logs (one per kernel,
    taken with --metrics dram__bytes_read.sum,dram__bytes_write.sum on the
    benchmark's workload): per kernel the mean DRAM bytes per launch and per
    cell, keyed to a hash of the kernel's current sources."""
    import csv
    kinds = {"k_sweep_tile": "sweep", "k_fields_tile": "fields", "k_coupling": "coupling"}
    per = {}
    for path in paths:
        with open(path) as f:
            rows = [r for r in csv.reader(l for l in f if l.startswith('"'))]
        head, body = rows[0], rows[1:]
        ik, im, iv = head.index("Kernel Name"), head.index("Metric Name"), head.index("Metric Value")
        iu = head.index("Metric Unit") if "Metric Unit" in head else None
        scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
        for r in body:
            kind = next((v for k, v in kinds.items() if k in r[ik]), None)
            if kind is None or not r[im].startswith("dram__bytes"):
                continue
            val = float(r[iv].replace(",", "")) * (scale.get(r[iu], 1.0) if iu is not None else 1.0)
            e = per.setdefault(kind, {"kernel": r[ik].split("(")[0].strip(), "read": [], "write": [],
                                      "path": path})
            e["read" if "read" in r[im] else "write"].append(val)
    out = {"workload": workload, "kernels": {}}
    for kind, e in per.items():
        rd, wr = float(np.mean(e["read"])), float(np.mean(e["write"]))
        out["kernels"][kind] = {
            "kernel": e["kernel"], "launches_captured": len(e["read"]),
            "dram_bytes_read": rd, "dram_bytes_write": wr, "dram_bytes_per_cell": (rd + wr) / cells,
            "source": command.get(kind, ""), "sources": KERNEL_SOURCES[kind],
            "sources_sha256": kernel_source_hash(kind)}
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
    return out


def traffic_record(kernel):
    """ncu DRAM bytes per cell and launch for the kernel, if the committed
    record was taken on the kernel's current sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None, None
    k = rec.get("kernels", {}).get(kernel)
    if not k or k.get("sources_sha256") != kernel_source_hash(kernel):
        return None, rec
    return k["dram_bytes_per_cell"], rec


def cpu_baseline(wl, budget_s=12.0, state=None):
    """The oracle as it stands (FP32-state form, single thread) on whole
    steps of the same workload: from its initial state, and (state given:
    the GPU's state after step 1000, loaded into the oracle) from there."""
    import oracle

    def timed(S, what):
        t0 = time.perf_counter()
        k = 0
        while True:
            oracle.step(S, wl.field.u, wl.field.v, wl.dt)
            k += 1
            if time.perf_counter() - t0 > budget_s or k >= 8:
                break
        t = time.perf_counter() - t0
        return wl.n * wl.n * k / t, f"{k} whole steps of the {wl.n}^2 workload (FP32 form) from {what}"

    S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, oracle.FP32)
    v0, s0 = timed(S, "its initial state")
    out = {"value": v0, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": s0, "host": host_cores()}
    if state is not None:
        S = oracle.State(wl.n, wl.n, wl.dx, oracle.FP32)
        S.K[...], S.Z[...], S.sH[...], S.sV[...] = state["K"], state["Z"], state["sH"], state["sV"]
        S.step_index = state["step_index"]
        v1, s1 = timed(S, f"the GPU's state after step {state['step_index']}")
        out["late"] = {"value": v1, "sample": s1}
    return out


def host_cores():
    """The host's cores as the process sees them (the oracle runs on one)."""
    try:
        aff = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        aff = None
    return {"nproc": os.cpu_count(), "affinity": aff}


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
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cores(),
                             "sample": f"{done} whole steps of the {wl.n}^2 workload after {args.warmup} warm-up steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x, world, device):
    """The largest x over the ranks of the default process group."""
    if world == 1:
        return x
    import torch
    import torch.distributed as tdist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, cells, steps, max_ms):
    """Whole-job throughput: every rank's cell-updates over the slowest rank's time."""
    return world * cells * steps / (max_ms / 1e3)


COUPLING_FLUIDS = dict(rho1=1000.0, rho2=1.2, mu1=1.0e-3, mu2=1.8e-5, sigma=0.0728)


def time_coupling(torch, ebit, ctx, n, dtype, launches):
    """The hand-off to a flow solver (properties and surface-tension source
    from the step's C and kappa; not part of the step), timed by the
    library's events around each of its launches (timing must be on).
    Returns (total ms, launches)."""
    outs = [torch.empty(sh, dtype=dtype, device="cuda") for sh in ((n, n), (n, n), (n, n + 1), (n + 1, n))]
    for _ in range(3):
        ebit.ebit_coupling(ctx, **COUPLING_FLUIDS, rho=outs[0], mu=outs[1], fx=outs[2], fy=outs[3])
    ebit.ebit_timings(ctx)
    for _ in range(launches):
        ebit.ebit_coupling(ctx, **COUPLING_FLUIDS, rho=outs[0], mu=outs[1], fx=outs[2], fy=outs[3])
    return ebit.ebit_timings(ctx)["coupling"]


def coupling_roofline(kc, n, esz, hbm, peak_kind):
    cb = coupling_bytes(n, n, esz)
    c_ms = kc[0] / max(1, kc[1])
    return {"kernel": "k_coupling", "bound": "hbm", "launches": kc[1], "avg_launch_ms": c_ms,
            "achieved": cb / (c_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": cb / (c_ms / 1e3) / 1e9 / hbm, "peak_source": f"{peak_kind} hbm_gbs (copy)",
            "algorithmic_bytes": cb, "bytes_per_cell": 6 * esz,
            "l2": f"C, kappa and outputs ({cb / 1e9:.2f} GB) larger than L2, no flush"}


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


def e2e_loop(torch, ebit, ctx, stream, hu, hv, u, v, dt, K, cells, world, barrier, fields, nb=3):
    """K steps through the C ABI from host memory: each step's u, v are
    copied from pinned host buffers (on an upload stream, into one of nb
    device buffers, while earlier steps compute), and each step's area comes
    back through ebit_area_async; with fields=True its fractions C come back
    too (ebit_fraction_to_host: straight into pinned host memory on a
    download stream while later steps run, so the two directions overlap
    each other and the steps).
    With nb buffers a copy has nb - 1 steps to finish; the host takes step
    k's results once step k+2 is queued.  Returns the e2e record."""
    n2 = u.shape
    dbuf = [(torch.empty_like(u), torch.empty_like(v)) for _ in range(nb)]
    copy_stream = torch.cuda.Stream()   # host -> device
    down_stream = torch.cuda.Stream()   # device -> host
    copied = [torch.cuda.Event() for _ in range(nb)]
    freed = [torch.cuda.Event() for _ in range(nb)]
    nC = (n2[0] - 1, n2[1] - 1)
    Chost = [torch.empty(nC, dtype=u.dtype).pin_memory() for _ in range(nb)] if fields else None
    c_home = [torch.cuda.Event() for _ in range(nb)]

    def upload(k):
        b = k % nb
        with torch.cuda.stream(copy_stream):
            if k >= nb:
                copy_stream.wait_event(freed[b])  # step k - nb has finished with this buffer
            dbuf[b][0].copy_(hu, non_blocking=True)
            dbuf[b][1].copy_(hv, non_blocking=True)
            copied[b].record(copy_stream)

    areas = torch.zeros(nb, dtype=torch.float64).pin_memory()
    arrived = [torch.cuda.Event() for _ in range(nb)]
    got, csum = [], []

    def take(k):
        b = k % nb
        arrived[b].synchronize()
        got.append(float(areas[b]))
        if fields:
            c_home[b].synchronize()
            csum.append(float(Chost[b][0, 0]) + float(Chost[b][-1, -1]))  # touch the copied values

    lag = min(2, nb - 1)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy_stream.wait_event(e0)
    down_stream.wait_event(e0)
    upload(0)
    for k in range(K):
        if k + 1 < K:
            upload(k + 1)
        b = k % nb
        stream.wait_event(copied[b])
        ebit.ebit_step(ctx, dbuf[b][0], dbuf[b][1], dt)
        freed[b].record(stream)
        ebit.ebit_area_async(ctx, areas[b:b + 1])
        arrived[b].record(stream)
        if fields:
            # C straight into pinned host memory on the download stream; the
            # library makes the next step's fields launch wait for the copy
            ebit.ebit_fraction_to_host(ctx, Chost[b], down_stream)
            c_home[b].record(down_stream)
        if k >= lag:
            take(k - lag)
    for k in range(max(0, K - lag), K):
        take(k)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t0)), world, "cuda")
    ebit.ebit_sync(ctx)  # deferred device errors of the e2e steps
    assert len(got) == K and all(a > 0 for a in got)
    esz = u.element_size()
    d2h = 8 + (nC[0] * nC[1] * esz if fields else 0)
    return {"value": job_value(world, cells, K, ms), "unit": UNIT,
            "h2d_bytes_per_step": int(hu.numel() * esz + hv.numel() * esz), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": ms / K,
            "overlap": f"inputs of step k+1 copied on an upload stream into one of {nb} device buffers while "
                       "earlier steps run; step k's area"
                       + (" and fractions C (on a download stream)" if fields else "")
                       + " read back while later steps run"}


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
    total_ms = max_over_ranks(total_ms, world, "cuda")
    ms_per_step = total_ms / args.steps
    value = job_value(world, cells, args.steps, total_ms)
    diag = ebit.ebit_diagnostics(ctx)

    # per-kernel durations over a second timed region (events around each of
    # the library's launches, on the launching stream)
    ebit.ebit_set_timing(ctx, True)
    ebit.ebit_timings(ctx)
    for _ in range(args.steps):
        ebit.ebit_step(ctx, u, v, wl.dt)
    kt = ebit.ebit_timings(ctx)
    kc = time_coupling(torch, ebit, ctx, n, torch.float32, args.steps)
    ebit.ebit_set_timing(ctx, False)
    kt = {k: t for k, t in kt.items() if t[1] > 0 or k != "coupling"}
    launches_per_step = sum(nl for _, nl in kt.values()) / args.steps
    hbm, peak_kind = peaks()
    esz = 4
    dom = max(kt, key=lambda k: kt[k][0])
    dom_ms = kt[dom][0] / max(1, kt[dom][1])
    dom_bytes = kernel_bytes_per_cell(dom, esz) * cells
    dom_gbps = dom_bytes / (dom_ms / 1e3) / 1e9
    traffic_cell, _ = traffic_record(dom)
    # the sweep is bound by the FP64 pipe (the circle fits), not by HBM: its
    # roofline is the algorithmic FP64 work of its fits against the SMs'
    # FP64 rate at the clock sampled during the timed region
    c = diag["counters"]
    fits_per_launch = float(c[ebit.D_FIT_ONLINE] + c[ebit.D_FIT_LINE] + c[ebit.D_FIT_ONE]
                            + c[ebit.D_FIT_TWO]) / 2.0
    sm_mhz = clk.get("sm_mhz") or 2070.0
    fp64_peak = FP64_OPS_PER_CLOCK * sm_mhz * 1e6 / 1e9  # Gop/s
    fit_ops = fits_per_launch * FIT_OPS
    # the sweep's own views: its dense byte model against HBM, and its
    # circle fits against the FP64 pipe, which is what bounds it
    sweep_view = {"kernel": dom, "avg_launch_ms": dom_ms,
                  "traffic": None if traffic_cell is None else traffic_cell * cells,
                  "hbm": {"achieved": dom_gbps, "peak": hbm, "unit": "GB/s", "frac": dom_gbps / hbm,
                          "algorithmic_bytes": dom_bytes, "bytes_per_cell": kernel_bytes_per_cell(dom, esz),
                          "peak_source": f"{peak_kind} hbm_gbs (copy)"},
                  "fp64_pipe": {"bound": "alu", "achieved": fit_ops / (dom_ms / 1e3) / 1e9, "peak": fp64_peak,
                                "unit": "GFLOP/s (FP64)", "frac": fit_ops / (dom_ms / 1e3) / 1e9 / fp64_peak,
                                "peak_source": f"derived: {FP64_OPS_PER_CLOCK} FP64 ops/clock (152 SMs x 2) x "
                                               f"{sm_mhz:.0f} MHz",
                                "algorithmic_flops": fit_ops, "fits_per_launch": fits_per_launch,
                                "flops_per_fit": FIT_OPS}}
    # the metric's roofline: one EBIT step (both sweeps, fields) with
    # the fused-step byte model (32.5 B/cell FP32) against the measured copy
    # bandwidth; traffic = the ncu DRAM bytes of a step's launches when every
    # record was taken on the current sources
    step_model = step_bytes_per_cell(esz) * cells
    per_step = {k: kt[k][1] / args.steps for k in kt}
    recs = {k: traffic_record(k)[0] for k in ("sweep", "fields") if per_step.get(k)}
    step_traffic = (None if any(v is None for v in recs.values())
                    else sum(recs[k] * per_step[k] * cells for k in recs))
    roofline = {"bound": "hbm", "kernel": "ebit_step (sweep x2, fields with the area sum)",
                "achieved": step_model / (ms_per_step / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": step_model / (ms_per_step / 1e3) / 1e9 / hbm,
                "peak_source": f"{peak_kind} hbm_gbs (copy)", "algorithmic_bytes": step_model,
                "bytes_per_cell": step_bytes_per_cell(esz), "traffic": step_traffic,
                "avg_step_ms": ms_per_step, "dominant": sweep_view,
                "kernels": {k: {"ms_per_launch": (t / max(1, nl)), "launches": nl,
                                "share": t / max(1e-12, sum(tt for tt, _ in kt.values())),
                                "GBps": kernel_bytes_per_cell(k, esz) * cells / (t / max(1, nl) / 1e3) / 1e9
                                if t > 0 else None}
                            for k, (t, nl) in kt.items()}}
    c_traffic, _ = traffic_record("coupling")
    coupling = coupling_roofline(kc, n, esz, hbm, peak_kind)
    coupling["traffic"] = None if c_traffic is None else c_traffic * cells

    # end to end through the C ABI with host buffers: every step copies its
    # u, v from pinned host memory and reads the step's results back.  The
    # copy of step k+1's inputs runs on a second stream into the other half
    # of a double buffer while step k computes (ordered by events), as a
    # caller that streams its velocities would do.
    hu = torch.from_numpy(wl.field.u.astype(np.float32)).pin_memory()
    hv = torch.from_numpy(wl.field.v.astype(np.float32)).pin_memory()
    e2e = e2e_loop(torch, ebit, ctx, stream, hu, hv, u, v, wl.dt, args.steps, cells, world, barrier,
                   fields=True)
    e2e["area_only"] = e2e_loop(torch, ebit, ctx, stream, hu, hv, u, v, wl.dt, args.steps, cells, world,
                                barrier, fields=False)

    # a second timed window from the state after 1000 steps, past the first
    # merges and break-ups of the disks (the steps up to it run untimed)
    late = None
    late_state = None
    done_steps = ebit.ebit_get_state(ctx, n, n)["step_index"]
    long_window = None
    if args.late_from > 0:
        # the steps up to it carry per-step events: p50/p99 of the step over
        # hundreds of steps, whatever --steps is
        nlong = max(0, args.late_from - done_steps)
        if nlong > 0:
            tlong, latlong = timed_steps(torch, ebit, ctx, u, v, wl.dt, nlong, stream)
            long_window = {"steps": [done_steps, done_steps + nlong], "ms_per_step": tlong / nlong,
                           "p50_ms": float(np.percentile(latlong, 50)),
                           "p99_ms": float(np.percentile(latlong, 99)),
                           "max_ms": float(np.max(latlong))}
        ebit.ebit_sync(ctx)
        torch.cuda.synchronize()
        barrier()
        tl, latl = timed_steps(torch, ebit, ctx, u, v, wl.dt, args.steps, stream)
        barrier()
        ebit.ebit_sync(ctx)
        dl = ebit.ebit_diagnostics(ctx)["counters"]
        tl = max_over_ranks(tl, world, "cuda")
        late = {"from_step": max(args.late_from, done_steps), "value": job_value(world, cells, args.steps, tl),
                "unit": UNIT, "ms_per_step": tl / args.steps,
                "p50_ms": float(np.percentile(latl, 50)), "p99_ms": float(np.percentile(latl, 99)),
                "step_roofline_frac": step_model / (tl / args.steps / 1e3) / 1e9 / hbm,
                "last_step": {"cancelled": int(dl[ebit.D_CANCELLED]), "zset": int(dl[ebit.D_ZSET]),
                              "nH": int(dl[ebit.D_NH]), "nV": int(dl[ebit.D_NV])}}
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            late_state = ebit.ebit_get_state(ctx, n, n)
    ebit.ebit_destroy(ctx)

    # the same FP32 steps with the generalised height-function fallbacks on
    ghf = None
    if not args.no_ghf:
        ctxg = ebit.ebit_init(n, n, wl.dx, wl.scene, prec, flags=ebit.EBIT_CURV_GHF, stream=stream)
        for _ in range(args.warmup):
            ebit.ebit_step(ctxg, u, v, wl.dt)
        torch.cuda.synchronize()
        barrier()
        tg, latg = timed_steps(torch, ebit, ctxg, u, v, wl.dt, args.steps, stream)
        barrier()
        ebit.ebit_sync(ctxg)
        tg = max_over_ranks(tg, world, "cuda")
        dg = ebit.ebit_diagnostics(ctxg)["counters"]
        ebit.ebit_set_timing(ctxg, True)
        ebit.ebit_timings(ctxg)
        for _ in range(args.steps):
            ebit.ebit_step(ctxg, u, v, wl.dt)
        ktg = ebit.ebit_timings(ctxg)
        ebit.ebit_set_timing(ctxg, False)
        ebit.ebit_destroy(ctxg)
        ghf = {"value": job_value(world, cells, args.steps, tg), "unit": UNIT, "ms_per_step": tg / args.steps,
               "ghf_ms_per_step": ktg["ghf"][0] / args.steps,
               "hf_invalid": int(dg[ebit.D_HF_INVALID]), "resolved_other": int(dg[ebit.D_HF_OTHER]),
               "resolved_mixed": int(dg[ebit.D_HF_MIXED]), "resolved_markers": int(dg[ebit.D_HF_MARKERS]),
               "note": "list pass over kappa plus compacted fits, per step (last step's counters)"}

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
        ebit.ebit_set_timing(ctx64, True)
        kc64 = time_coupling(torch, ebit, ctx64, n, torch.float64, args.steps)
        ebit.ebit_set_timing(ctx64, False)
        t64 = max_over_ranks(t64, world, "cuda")
        sb = step_bytes_per_cell(8) * cells
        fp64 = {"value": job_value(world, cells, args.steps, t64), "unit": UNIT, "ms_per_step": t64 / args.steps,
                "p50_ms": float(np.percentile(lat64, 50)), "p99_ms": float(np.percentile(lat64, 99)),
                "step_roofline_frac": sb / (t64 / args.steps / 1e3) / 1e9 / hbm,
                "coupling": coupling_roofline(kc64, n, 8, hbm, peak_kind)}
        ebit.ebit_destroy(ctx64)

    # configs 4 and 5 beside the headline: the batched FP32 form against
    # plain FP64 (batched, and one grid at a time), and the served FP32 form
    batched = serving = None
    if rank == 0 and world == 1:
        if not args.no_batched:
            batched = batched_leg(args)
        if not args.no_serving:
            serving = serving_leg(args, args.leg_rate, 1)
            serving["fp64"] = serving_leg(args, args.leg_rate, 0)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, state=late_state)

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
                "roofline": roofline, "late_window": late, "coupling": coupling, "ghf": ghf,
                "fp64": fp64, "step_latency_long_window": long_window,
                "batched": batched, "serving": serving,
                "cpu_baseline": cpu,
                "markers": {"nH": int(diag["counters"][0]), "nV": int(diag["counters"][1])}}
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()


def _batched_workloads(count, seed=230900340):
    """Grids of side log-uniform in [32, 512], 1-64 circles of radius
    U[0.05, 0.15] (at least 3 cells), a coin flip between the time-reversed
    vortex (period = steps * dt) and the cellular flow, 200-1000 steps, CFL 0.5."""
    from paper_2309_00338_gb300 import workloads as W
    rng = W.Rng(seed)
    return [W.random_instance(rng) for _ in range(count)]


def _batched_requests(count, seed=230900340):
    out = []
    for wl in _batched_workloads(count, seed):
        vortex = wl.field.name == "vortex"
        out.append(dict(n=wl.n, circles=wl.scene["circles"], steps=wl.steps, cfl=0.5,
                        field=0 if vortex else 1, period=wl.steps * wl.dt if vortex else 1.0,
                        vortex=vortex))
    return out


def _serve(ebit, specs, prec, budget, max_instances=0, arrivals=None, cap_s=None, schedule=-1):
    """Submit specs (at arrival times if given), wait; returns results + stats.
    schedule >= 0: that ebit_schedule for every batch step (no autotuning)."""
    s = ebit.ebit_server_create(budget, max_instances=max_instances, autotune=schedule < 0,
                                schedule=max(0, schedule))
    keep, tickets = [], []
    t0 = time.perf_counter()
    res = {}
    try:
        for k, sp in enumerate(specs):
            if arrivals is not None:
                delay = arrivals[k] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            r, kk = ebit.make_request(sp["n"], sp["circles"], sp["field"], sp["steps"], sp["cfl"], prec,
                                      period=sp["period"], omega=sp.get("omega", 0.0),
                                      centre=sp.get("centre", (0.5, 0.5)), drift=sp.get("drift", (0.0, 0.0)))
            keep.append(kk)
            tickets.append(ebit.ebit_submit(s, r))
        while len(res) < len(tickets):
            for t in tickets:
                if t not in res:
                    r = ebit.ebit_poll(s, t)
                    if r is not None:
                        res[t] = r
            if cap_s is not None and time.perf_counter() - t0 > cap_s:
                break
            time.sleep(0.002)
        wall = time.perf_counter() - t0
        stats = ebit.ebit_server_stats_get(s)
    finally:
        ebit.ebit_server_destroy(s)
    return [res.get(t) for t in tickets], stats, wall


def batched_roofline(cell_updates, gpu_ms, esz):
    """The step's HBM roofline (the dense byte model of step_bytes_per_cell)
    for cell-updates done in gpu_ms of GPU time, against the measured copy
    bandwidth."""
    hbm, kind = peaks()
    bpc = step_bytes_per_cell(esz)
    gbps = bpc * cell_updates / (gpu_ms / 1e3) / 1e9 if gpu_ms > 0 else 0.0
    return {"bound": "hbm", "achieved": gbps, "peak": hbm, "unit": "GB/s", "frac": gbps / hbm,
            "bytes_per_cell": bpc, "peak_source": f"{kind} hbm_gbs (copy)"}


def batched_cpu_baseline(count, budget_s=10.0, seed=230900343):
    """The plain CPU baseline of the batched workload: the oracle as it
    stands (plain FP64), one instance at a time per host thread on every core
    this process may use.  Each thread takes the next grid of a seeded random
    order of the grids and runs it from its initial state until its steps end
    or the time budget does, then takes the next one.  The oracle's steps are
    single foreign calls that release the interpreter lock, so the threads
    run in parallel."""
    import threading
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    from paper_2309_00338_gb300 import workloads as W
    wls = _batched_workloads(count)
    cores = host_cores()["affinity"] or os.cpu_count() or 1
    pick = W.Rng(seed)
    order = list(range(len(wls)))
    for i in range(len(order) - 1, 0, -1):  # seeded Fisher-Yates shuffle
        j = min(i, int(pick.uniform() * (i + 1)))
        order[i], order[j] = order[j], order[i]
    lock = threading.Lock()
    nxt = [0]
    t0 = time.perf_counter()

    def run(_):
        cells = steps = grids = 0
        while time.perf_counter() - t0 < budget_s:
            with lock:
                if nxt[0] >= len(order):
                    break
                wl = wls[order[nxt[0]]]
                nxt[0] += 1
            S = oracle.init(wl.n, wl.n, wl.dx, wl.scene, oracle.FP64)
            grids += 1
            k = 0
            while k < wl.steps and time.perf_counter() - t0 < budget_s:
                oracle.step(S, wl.field.u, wl.field.v, wl.field.dt_eff(k, wl.dt))
                k += 1
            cells += wl.n * wl.n * k
            steps += k
        return cells, steps, grids

    with ThreadPoolExecutor(cores) as ex:
        done = list(ex.map(run, range(cores)))
    wall = time.perf_counter() - t0
    return {"value": sum(d[0] for d in done) / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "prec": "fp64",
            "sample": f"{sum(d[2] for d in done)} grids of the batched workload in a seeded random order "
                      f"(seed {seed}), one at a time per host thread, {sum(d[1] for d in done)} steps in "
                      f"{wall:.1f} s (initialisation included)",
            "host": host_cores()}


def batched_leg(args):
    """512 uneven grids advanced together (one captured launch sequence per
    batch step) in FP32 and FP64, against one-grid-at-a-time plain FP64 on a
    seeded random sample of the grids.  Values are cell-updates over the GPU
    time of the batch steps (the server's own events)."""
    from paper_2309_00338_gb300 import ebit
    import torch
    torch.cuda.set_device(0)
    specs = _batched_requests(args.instances)
    budget = 200 << 30
    out = {}
    for name, prec in (("fp32", 1), ("fp64", 0)):
        res, st, wall = _serve(ebit, specs, prec, budget, schedule=args.schedule)
        lat = [r["step_p50_ms"] for r in res if r]
        ea = [r["e_area"] for r, sp in zip(res, specs) if r and sp["vortex"]]
        out[name] = {"cell_updates": st["cell_updates"], "gpu_ms": st["busy_ms"], "wall_s": wall,
                     "value": st["cell_updates"] / (st["busy_ms"] / 1e3),
                     "batch_steps": st["batch_steps"],
                     "step_p50_ms": float(np.percentile(lat, 50)), "step_p99_ms": float(np.percentile(lat, 99)),
                     "e_area_reversed_median": float(np.median(ea)) if ea else None,
                     "e_area_reversed_max": float(np.max(ea)) if ea else None,
                     "autotune": {"schedule": st["schedule"], "tuned_sets": st["tuned_sets"],
                                  "tune_ms": st["tune_ms"]},
                     "roofline": batched_roofline(st["cell_updates"], st["busy_ms"], 4 if prec == 1 else 8)}
    # plain FP64 one grid at a time on a seeded random sample of the grids
    from paper_2309_00338_gb300 import workloads as W
    pick = W.Rng(230900342)
    idx = sorted(set(min(len(specs) - 1, int(pick.uniform() * len(specs)))
                     for _ in range(4 * args.one_at_a_time)))[:args.one_at_a_time]
    sub = [specs[i] for i in idx]
    res, st, wall = _serve(ebit, sub, 0, budget, max_instances=1)
    out["fp64_one_at_a_time"] = {"instances": len(sub), "sample": "seeded random sample (seed 230900342)",
                                 "cell_updates": st["cell_updates"], "gpu_ms": st["busy_ms"],
                                 "value": st["cell_updates"] / (st["busy_ms"] / 1e3)}
    total = sum(sp["n"] ** 2 * sp["steps"] for sp in specs)
    out["config"] = {"workload": f"batched_{len(specs)}_grids_32-512", "cell_updates": total,
                     "seed": 230900340}
    out["fp32_over_fp64_one_at_a_time"] = out["fp32"]["value"] / out["fp64_one_at_a_time"]["value"]
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = batched_cpu_baseline(len(specs))
    return out


def run_batched(args):
    out = batched_leg(args)
    line = {"metric": "EBIT cell-updates/s, batched uneven grids", "value": out["fp32"]["value"],
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": out["config"],
            "fp32": out["fp32"], "fp64": out["fp64"], "fp64_one_at_a_time": out["fp64_one_at_a_time"],
            "cpu_baseline": out.get("cpu_baseline")}
    print(json.dumps(line), flush=True)


def serving_leg(args, rate, prec=1):
    """Poisson arrivals: grids of side log-uniform in [64, 2048], 1-500
    circles of radius U[3, 30] cells, 50-2000 steps of the vortex, the
    cellular flow or a solid rotation; every request in precision prec
    (1: FP32 fractions with the FP64 fit, 0: plain FP64)."""
    from paper_2309_00338_gb300 import ebit
    from paper_2309_00338_gb300 import workloads as W
    import torch
    torch.cuda.set_device(0)
    rng = W.Rng(230900341)
    specs, arrivals = [], []
    t = 0.0
    while True:
        t += -math.log(1.0 - rng.uniform()) / rate
        if t > args.serve_seconds:
            break
        n = int(round(math.exp(rng.uniform(math.log(64), math.log(2048)))))
        dx = 1.0 / n
        count = rng.integer(1, 500)
        steps = rng.integer(50, 2000)
        kind = rng.integer(0, 2)
        circles = W.place_circles(rng, count, 3 * dx, 30 * dx, 2 * dx, lambda x, y, r: True, max_tries=20)
        sp = dict(n=n, circles=circles, steps=steps, cfl=0.5, field=kind, period=steps * 0.5 * dx,
                  omega=2 * math.pi, centre=(0.5, 0.5), drift=(0.3, 0.1))
        specs.append(sp)
        arrivals.append(t)
    # a 16 GiB admission budget bounds the batch (and so the step latency)
    res, st, wall = _serve(ebit, specs, prec, 16 << 30, arrivals=arrivals, cap_s=args.serve_cap,
                           schedule=args.schedule)
    done = [r for r in res if r is not None]
    lat50 = [r["step_p50_ms"] for r in done]
    lat99 = [r["step_p99_ms"] for r in done]
    qw = [r["queue_ms"] for r in done]
    offered = sum(sp["n"] ** 2 * sp["steps"] for sp in specs) / args.serve_seconds
    return {"value": st["cell_updates"] / wall, "unit": UNIT, "prec": "fp32" if prec == 1 else "fp64",
            "config": {"workload": "serving_poisson", "rate_per_s": rate, "arrival_window_s": args.serve_seconds,
                       "requests": len(specs), "offered_cell_updates_per_s": offered, "wall_cap_s": args.serve_cap},
            "completed": len(done), "wall_s": wall, "gpu_busy_s": st["busy_ms"] / 1e3,
            "batch_steps": st["batch_steps"],
            "gpu_value": st["cell_updates"] / (st["busy_ms"] / 1e3) if st["busy_ms"] else None,
            "step_p50_ms": float(np.median(lat50)) if lat50 else None,
            "step_p99_ms": float(np.percentile(lat99, 99)) if lat99 else None,
            "queue_ms_p50": float(np.median(qw)) if qw else None,
            "queue_ms_p99": float(np.percentile(qw, 99)) if qw else None,
            "autotune": {"schedule": st["schedule"], "tuned_sets": st["tuned_sets"], "tune_ms": st["tune_ms"]},
            "worker_idle_gpu_ms": {"plans": st["plans"], "plan_ms": st["plan_ms"],
                                   "plan_graph_ms": st["plan_graph_ms"],
                                   "admit_ms": st["admit_idle_ms"], "retire_ms": st["retire_ms"]}}


def run_serving(args):
    leg = serving_leg(args, args.rate, 1)
    line = {"metric": "EBIT served cell-updates/s (continuous batching)", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic", **leg}
    if args.serve_fp64:
        line["fp64"] = serving_leg(args, args.rate, 0)
    print(json.dumps(line), flush=True)


TRAFFIC_COMMAND = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                   "--clock-control none -k regex:{k} -s {s} -c {c} --csv --log-file {log} python bench.py "
                   "--steps 1 --warmup 1 --no-cpu-baseline --no-fp64 --no-ghf --late-from 0")


def main():
    args = parse()
    if args.record_traffic:
        cmds = {"sweep": TRAFFIC_COMMAND.format(k="k_sweep_tile", s=2, c=2, log="dram_sweep.csv"),
                "fields": TRAFFIC_COMMAND.format(k="k_fields_tile", s=2, c=1, log="dram_fields.csv"),
                "coupling": TRAFFIC_COMMAND.format(k="k_coupling", s=3, c=1, log="dram_coupling.csv")}
        print(json.dumps(record_traffic(args.record_traffic, 4096 * 4096,
                                        "cellular_curve_n4096 FP32 form (the bench headline)", cmds), indent=1))
        return
    world, rank, local = dist()
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    from paper_2309_00338_gb300 import workloads as W
    wl = W.cellular_curve_workload()
    if args.impl == "reference":
        run_reference(args, wl, world, rank)
        return
    run_ours(args, wl, world, rank, local)


if __name__ == "__main__":
    main()
