"""Host-side legs of bench.py that need no GPU: the batched workload's plain
CPU baseline (the oracle, one grid at a time per host thread)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_batched_cpu_baseline_keeps_every_thread_on_its_own_grid():
    sys.path.insert(0, ROOT)
    import bench
    out = bench.batched_cpu_baseline(8, budget_s=0.5)
    assert out["kind"] == "oracle" and out["prec"] == "fp64" and out["unit"] == bench.UNIT
    assert out["cores"] >= 1 and out["value"] > 0
    # the sample names how many grids and steps the threads ran
    grids = int(out["sample"].split()[0])
    assert 1 <= grids <= 8


def test_batched_workloads_are_seeded():
    sys.path.insert(0, ROOT)
    import bench
    a = bench._batched_workloads(4)
    b = bench._batched_workloads(4)
    assert [w.n for w in a] == [w.n for w in b]
    assert [w.steps for w in a] == [w.steps for w in b]
    reqs = bench._batched_requests(4)
    assert [r["n"] for r in reqs] == [w.n for w in a]


def test_byte_models_are_the_stated_ones():
    """The roofline byte models the bench reports against: one EBIT step
    32.5 B/cell (FP32) and 64.5 (FP64); a sweep 20.5 / 40.5; the fields
    16.25 / 32.25; the coupling 24 / 48, with its face arrays counted exactly."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.step_bytes_per_cell(4) == 32.5 and bench.step_bytes_per_cell(8) == 64.5
    assert bench.kernel_bytes_per_cell("sweep", 4) == 20.5
    assert bench.kernel_bytes_per_cell("sweep", 8) == 40.5
    assert bench.kernel_bytes_per_cell("fields", 4) == 16.25
    assert bench.kernel_bytes_per_cell("fields", 8) == 32.25
    assert bench.kernel_bytes_per_cell("coupling", 4) == 24
    n = 4096
    assert bench.coupling_bytes(n, n, 4) == 4 * (6 * n * n + 2 * n)
    assert bench.FIT_OPS == 81


def test_batched_roofline_arithmetic():
    """The batched legs' roofline: the step's byte model times the
    cell-updates over the GPU time, against the copy bandwidth."""
    sys.path.insert(0, ROOT)
    import bench
    hbm, _ = bench.peaks()
    r = bench.batched_roofline(10 ** 10, 500.0, 4)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["bytes_per_cell"] == 32.5
    assert abs(r["achieved"] - 650.0) < 1e-9 and abs(r["frac"] - 650.0 / hbm) < 1e-12
    assert bench.batched_roofline(10 ** 10, 500.0, 8)["achieved"] == 2 * 645.0 * 1.0
    assert bench.batched_roofline(0, 0.0, 4)["achieved"] == 0.0
