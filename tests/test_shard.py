"""Batch instances split across ranks by bytes (paper_0704_3444_gb300.shard), on CPU."""
import os
import socket

import numpy as np
import pytest

from paper_0704_3444_gb300 import inputs, shard

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


@pytest.fixture(scope="module")
def probs():
    return inputs.batch(512)


def test_instance_bytes_counts_the_stored_values(probs):
    p = probs[0]
    S = p.nx * p.ny
    assert shard.instance_bytes(p, "fp32") == 72 * p.ncomp * S
    assert shard.instance_bytes(p, "fp64") == 144 * p.ncomp * S
    assert shard.instance_bytes(p, "bf16") == 44 * p.ncomp * S
    line = inputs.flat_interface([0.5, 0.5], chi=2.2 * (1 - np.eye(2)))
    line.lattice = "d1q3"
    assert shard.instance_bytes(line, "fp64") == 2 * 3 * 8 * 2 * line.nx


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_every_instance_once_and_balanced(probs, world):
    parts = shard.partition_by_bytes(probs, world)
    flat = sorted(k for p in parts for k in p)
    assert flat == list(range(len(probs)))
    sizes = [shard.instance_bytes(p) for p in probs]
    loads = [sum(sizes[k] for k in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)
    assert parts == shard.partition_by_bytes(probs, world)   # deterministic
    assert all(shard.share(probs, r, world) == parts[r] for r in range(world))


def test_more_ranks_than_instances(probs):
    parts = shard.partition_by_bytes(probs[:3], 5)
    assert sorted(len(p) for p in parts) == [0, 0, 1, 1, 1]
    with pytest.raises(ValueError):
        shard.share(probs, 5, 5)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.share(inputs.batch(64), rank, world)
        got = [None] * world
        dist.all_gather_object(got, mine)
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_ranks_agree_on_the_split_without_exchanging_it():
    """Each of three gloo ranks computes its share on its own; gathered, the shares are
    disjoint, cover the batch, and every rank saw the same split."""
    world, port = 3, _free_port()
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
    assert res[0] == res[1] == res[2]
    assert sorted(k for part in res[0] for k in part) == list(range(64))
