"""N>1 host path on CPU: frame sharding and the cross-rank timing reductions,
run as two gloo ranks (the GPU decode itself is per rank and needs no
collective)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1504_00353_gb300 import sharding, synth


def test_frame_range_partitions():
    for n in (0, 1, 7, 4096, 10001):
        for world in (1, 2, 3, 8):
            ranges = [sharding.frame_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.frame_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 37
        lo, hi = sharding.frame_range(n, rank, world)
        mask = synth.frozen_mask(64, 32, 2.0)
        rng = np.random.default_rng(0)
        llr = (rng.standard_normal((n, 64)) * 2).astype(np.float32)
        mine = oracle.decode_batch(mask, llr[lo:hi])
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, mine))
        t_max = sharding.max_over_ranks(1.0 + rank)
        frames = sharding.sum_over_ranks(hi - lo)
        dist.barrier()
        if rank == 0:
            full = np.concatenate([p[2] for p in sorted(parts, key=lambda p: p[0])])
            q.put((np.array_equal(full, oracle.decode_batch(mask, llr)), t_max, frames))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    same, t_max, frames = q.get(timeout=10)
    assert same and t_max == 2.0 and frames == 37
