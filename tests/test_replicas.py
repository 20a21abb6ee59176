"""Replica mode of the benchmark (one independent system per rank, no data-path
collective): whole-job throughput = all ranks' units over the slowest rank's
time. Two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, secs = 1000.0 * (rank + 1), 2.0 + rank        # uneven ranks: the slowest sets the time
    rate, tmax = bench.job_rate(units, secs, dist, device="cpu")
    out[rank] = (rate, tmax)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    # every rank reports the same whole-job figure: world x (its own units) / max time
    assert out[0][1] == out[1][1] == 3.0
    assert out[0][0] == pytest.approx(2 * 1000.0 / 3.0)
    assert out[1][0] == pytest.approx(2 * 2000.0 / 3.0)


def test_job_rate_single():
    import importlib
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    assert bench.job_rate(500.0, 2.0) == (250.0, 2.0)
