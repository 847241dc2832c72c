"""The multi-rank path of the benchmark on CPU (gloo, world size 2): shard partition,
per-rank point streams, and the max-time / total-work reduction."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2606_24154_gb300 import inputs as I
    from paper_2606_24154_gb300 import sharding as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = I.cube(n_per_edge=2)
        pts = I.cell_points(g, 100, I.rng(1, S.shard_seed_stream(rank)))
        ms = 10.0 + 5.0 * rank
        units = float(pts.shape[0] * g.n * g.n_images)
        mx, tot = S.reduce_step_time(ms, units)
        lo, hi = S.shard_range(1001, rank, world)
        out[rank] = (mx, tot, float(pts[0, 0]), lo, hi)
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_and_shards():
    world = 2
    port = _free_port()
    # every process (the manager's too) is spawned, never forked from a process that may
    # hold threads or a CUDA context
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 15.0                      # max over ranks
    assert r0[1] == r1[1] == 2 * 100 * 24 * 1          # total evaluations of both ranks
    assert r0[2] != r1[2]                              # ranks draw different points
    assert (r0[3], r0[4], r1[3], r1[4]) == (0, 501, 501, 1001)
