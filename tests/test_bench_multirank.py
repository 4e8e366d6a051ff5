"""The multi-rank host logic of bench.py on two gloo ranks (CPU): the slowest rank's time
decides the whole-job rate, and only rank 0 runs the reference arm."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms_local = 100.0 + 50.0 * rank          # rank 1 is the slower one
    ms = bench.max_over_ranks(ms_local, ws, device="cpu")
    rate = bench.replica_rate(ws, 50, 5, ms)
    out[rank] = (ms, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ws = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    for rank in range(ws):
        ms, rate = out[rank]
        assert ms == 150.0
        assert rate == pytest.approx(2 * 50 * 5 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.replica_rate(1, 50, 5, 1000.0) == pytest.approx(250.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench

    class A:                                   # arguments of a tiny run
        N, n, steps, warmup, gpus = 20, 4, 1, 0, 2
    bench.run_reference(A, 2, 1)               # rank 1: no work, no output
    assert capsys.readouterr().out == ""
