"""The N > 1 path of the benchmark on CPU (gloo, two ranks): replicas with
one max-reduce of the time, as `bench.py --gpus N` runs them under
torchrun.  Every rank times its own system; the job's rate is every rank's
cells over the slowest rank's time, the same on every rank.  Each rank's
workload is its own (seeded by rank), and the reference arm works on rank 0
alone."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 1.0 + rank  # rank 1 is the slow one
        rate, t = bench.job_rate(dist, t_local, 1000, 5, world, "cpu")
        out[rank] = (rate, t)
    finally:
        dist.destroy_process_group()


def test_job_rate_is_all_cells_over_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # 2 ranks x 1000 cells x 5 steps over the slower rank's 2 s
    assert out[0] == out[1] == (2 * 1000 * 5 / 2.0, 2.0)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(None, 0.5, 1000, 4, 1, "cpu") == (8000.0, 0.5)


def test_ranks_get_their_own_systems():
    sys.path.insert(0, ROOT)
    import bench
    a, grid_a, _, _ = bench.workload("radical2m", 0)
    b, grid_b, _, _ = bench.workload("radical2m", 1)
    assert a.n == b.n and grid_a == grid_b
    assert not np.array_equal(a.pos, b.pos)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    bench.run_reference(args, 1, 2)  # a rank other than 0 does no work
    assert capsys.readouterr().out == ""
