"""Multi-rank host logic of bench.py on the CPU (gloo, world size 2): each
rank times its own field; the job's time is the maximum over ranks and its
throughput every rank's bytes over that time; the reference arm runs on
rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from conftest import ROOT  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.0][rank]
        m = bench.max_over_ranks(ms, world)
        v = bench.weak_scaling_value(100_000_000, 10, world, m)
        out[rank] = (m, v)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    m, v = out[0]
    assert m == 20.0
    assert v == pytest.approx(2 * 100_000_000 * 10 / 0.020 / 1e9)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.weak_scaling_value(4, 1, 1, 1.0) == pytest.approx(4e-6)


def _ref_worker(rank, world, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, world

    called = []
    bench.cpu_baseline = lambda *a, **k: called.append(a) or {"value": 1.0}
    bench.run_reference(A)
    out[rank] = len(called)


def test_reference_arm_runs_on_rank_zero_only():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_ref_worker, args=(world, out), nprocs=world, join=True)
    assert out[1] == 0 and out[0] >= 1
