"""The multi-rank timing of bench.py on CPU: two gloo ranks with different timings
report the same whole-job rate, set by the slower rank (weak scaling: every rank does
the same work on its own replica)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [2.0, 5.0][rank]
    value, tmax = bench.job_rate(torch, dist, 1e6, elapsed, world, "cpu")
    out[rank] = (value, tmax)
    dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    value, tmax = res[0]
    assert tmax == 5.0
    assert abs(value - world * 1e6 / 5.0 / 1e6) < 1e-12


def test_job_rate_single_rank():
    import bench
    assert bench.job_rate(torch, None, 3e6, 1.5, 1, "cpu") == (2.0, 1.5)
