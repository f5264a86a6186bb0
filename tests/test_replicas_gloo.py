"""The multi-GPU path of bench.py runs independent replicas (one solve per rank, no
collective on the data path): the whole-job figures are the slowest rank's time and the
work of all ranks summed, and only rank 0 runs the CPU reference arm. Checked here with
world_size 2 over gloo on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, work = bench.replica_totals(10.0 + 5.0 * rank, 100.0 * (rank + 1), device="cpu")
    assert bench.dist_env() == (world, rank, 0)
    out[rank] = (ms, work)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_totals_over_gloo():
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [mp.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        # max of the times (10, 15), sum of the work (100 + 200), the same on both ranks
        assert out[0] == out[1] == (15.0, 300.0)


def test_single_process_totals_are_local():
    import bench

    assert bench.replica_totals(12.5, 7.0, device="cpu") == (12.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the CPU reference runs once (rank 0); other ranks exit at once."""
    import argparse

    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "run_cpu_oracle", lambda *a, **k: called.append(1))
    bench.reference_arm(argparse.Namespace(steps=1, warmup=0, gpus=2, workload="p3_n32"))
    assert called == [] and capsys.readouterr().out == ""
