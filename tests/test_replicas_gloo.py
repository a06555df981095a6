"""The replicas-only multi-GPU bookkeeping on CPU: two gloo ranks agree on the
max step time and the whole-job throughput, and draw different boxes."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2501_10622_gb300 import replicas, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = replicas.env_ranks()
        assert (w, r, lr) == (world, rank, rank)
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        mx = replicas.max_over_ranks(ms)
        pos = synth.clumped_box(2000, 10.0, 3, seed=replicas.replica_seed(9, rank))
        digest = float(pos.double().sum())
        digests = [None] * world
        dist.all_gather_object(digests, digest)
        out[rank] = (mx, replicas.whole_job_throughput(1_000_000, world, mx), digests)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    (m0, v0, d0), (m1, v1, d1) = out[0], out[1]
    assert m0 == m1 == 15.0
    assert v0 == v1 == pytest.approx(2 * 1_000_000 / 0.015 / 1e6)
    assert d0 == d1 and d0[0] != d0[1]  # independent replicas


def test_single_process_identity():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.whole_job_throughput(10 ** 6, 1, 1000.0) == pytest.approx(1.0)
