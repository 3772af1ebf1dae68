"""Multi-process host logic of replica runs, with gloo on the CPU
(world size 2): set assignment covers every set once and balances work, and
timings combine as units of all ranks over the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2511_15269_gb300 import replicas, workloads


def test_shard_sets_single_process():
    sizes = [5, 1, 9, 3, 3, 7]
    assert replicas.shard_sets(sizes, 0, 1) == list(range(6))
    a, b = replicas.shard_sets(sizes, 0, 2), replicas.shard_sets(sizes, 1, 2)
    assert sorted(a + b) == list(range(6)) and not set(a) & set(b)
    assert abs(sum(sizes[i] for i in a) - sum(sizes[i] for i in b)) <= max(sizes)
    assert replicas.max_over_ranks(3.5) == 3.5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [len(q) for _, q in workloads.batched_sets(16, seed=0, n_min=100, n_max=5000)]
        mine = replicas.shard_sets(sizes, rank, world)
        units = sum(sizes[i] for i in mine)
        ms = 10.0 + rank  # rank 1 is the slower one
        value, total, slowest = replicas.aggregate_throughput(units, ms)
        out[rank] = (mine, units, value, total, slowest)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    sizes = [len(q) for _, q in workloads.batched_sets(16, seed=0, n_min=100, n_max=5000)]
    a, b = res[0][0], res[1][0]
    assert sorted(a + b) == list(range(16)) and not set(a) & set(b)
    total = sum(sizes)
    for r in range(2):
        _, units, value, tot, slowest = res[r]
        assert tot == total and slowest == 11.0
        assert value == pytest.approx(total / 11e-3 / 1e6)
    assert abs(res[0][1] - res[1][1]) <= max(sizes)
