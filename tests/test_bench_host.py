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
