"""The N > 1 benchmark path on CPU: replicas share no data, the job time is
the slowest rank's (max over ranks through torch.distributed, here gloo with
world size 2) and the throughput counts every rank's work."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank          # the second replica is slower
    m = bench.max_over_ranks(local_ms)
    rate = bench.job_throughput(100.0, world, m)
    dist.barrier()
    out[rank] = (m, rate)
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world_2():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0                 # slowest rank's time everywhere
    assert res[0][1] == pytest.approx(2 * 100.0 / 0.015)  # both ranks' work over that time


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(10.0, 1, 2.0) == pytest.approx(5000.0)


def test_reference_arm_runs_on_rank0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        config, steps, warmup = 1, 1, 0

    assert bench.run_reference(Args()) is None
