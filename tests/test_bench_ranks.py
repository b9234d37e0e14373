"""Multi-rank logic of bench.py on CPU: two gloo ranks, each with its own bricks, reduce
their points (sum) and times (slowest rank); the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.reduce_over_ranks(1000 * (rank + 1), 10.0 + 5.0 * rank, world, "cpu")
    finally:
        dist.destroy_process_group()


def test_whole_job_totals_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        assert out[0] == (3000, 15.0)
        assert out[1] == (3000, 15.0)


def test_single_rank_totals_are_the_local_ones():
    import bench
    assert bench.reduce_over_ranks(1234, 7.5, 1, "cpu") == (1234, 7.5)


def test_reference_arm_prints_only_on_rank_zero(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0, "cpu_seconds": 0.1, "gpus": 2})()
    bench.run_reference(args, bench.workload_of("dd8"))
    assert capsys.readouterr().out == ""
