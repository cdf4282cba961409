"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2).

With N > 1 every rank runs its own replica; the whole-job figure is all
ranks' cell-updates over the slowest rank's time, and only rank 0 runs the
reference arm.  The aggregation runs here on gloo ranks; on the GPU machine the
same code runs on NCCL.
"""
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist

    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [30.0, 50.0][rank]  # rank 1 is the slow one
        m = bench.max_over_ranks(ms, world, "cpu")
        q.put((rank, m, bench.job_value(world, 4096 * 4096, 20, m), bench.dist()))
    finally:
        tdist.destroy_process_group()


def test_slowest_rank_sets_the_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, value, d in out:
        assert m == 50.0
        assert value == pytest.approx(2 * 4096 * 4096 * 20 / 0.050)
        assert d == (2, rank, rank)


def test_reference_arm_runs_on_rank_0_only():
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(steps=1, warmup=0)
    # a rank other than 0 returns before touching the workload or the oracle
    assert bench.run_reference(args, None, 2, 1) is None
