"""The N-GPU path of bench.py on CPU: two gloo ranks, each a replica, aggregate to the
slowest rank's time and the sum of solved right-hand sides; the reference arm runs on
rank 0 only and the other ranks return without work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, solved = bench.aggregate_ranks(100.0 + 50.0 * rank, 12 - rank, world, "cpu")
    q.put((rank, ms, solved))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_replicas():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, solved in got:
        assert ms == 150.0 and solved == 23.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(argparse.Namespace(steps=1, warmup=0, ref_mvps_per_rhs=8175))
    assert capsys.readouterr().out == ""
