"""The multi-rank paths on CPU (gloo, world size 2): shard partition, per-rank point
streams, the max-time / total-work reduction, and results: a point set evaluated shard by
shard and gathered equals the unsharded evaluation, and the space-charge step's all-gather
of carriers gives every rank the whole set, so that its targets' sums equal the unsharded
ones.  The oracle stands in for each rank's GPU evaluation (test only)."""
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


def _result_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_2606_24154_gb300 import inputs as I
    from paper_2606_24154_gb300 import sharding as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # evaluation: a strong-scaling split of one point set (odd size: unequal shards)
        g = I.cube(n_per_edge=4)
        sig, _, _ = O.solve(g)
        pts = I.cell_points(g, 37, I.rng(1, 40))
        lo, hi = S.shard_range(pts.shape[0], rank, world)
        phi, E = O.eval_points(g, sig, pts[lo:hi])
        full_phi = S.gather_rows(torch.from_numpy(phi), pts.shape[0]).numpy()
        full_E = S.gather_rows(torch.from_numpy(E), pts.shape[0]).numpy()
        # space charge: carriers partitioned; all-gather, then this rank's targets
        pos, q = I.carrier_cloud(I.thgem(I.PlateSpec(n_phi=12, n_r=2, n_zc=1, n_zf=3), n_plane=2), 61,
                                 I.rng(3, 40))
        a, b = S.shard_range(pos.shape[0], rank, world)
        gpos, gq = S.allgather_carriers(torch.from_numpy(pos[a:b]), torch.from_numpy(q[a:b]), pos.shape[0])
        tgt = I.cell_points(g, 23, I.rng(3, 41))
        ta, tb = S.shard_range(tgt.shape[0], rank, world)
        sphi, sE = O.space_charge(gpos.numpy(), gq.numpy(), tgt=tgt[ta:tb], soft=1e-6)
        full_sphi = S.gather_rows(torch.from_numpy(sphi), tgt.shape[0]).numpy()
        full_sE = S.gather_rows(torch.from_numpy(sE), tgt.shape[0]).numpy()
        out[rank] = (full_phi, full_E, gpos.numpy(), gq.numpy(), full_sphi, full_sE)
    finally:
        dist.destroy_process_group()


def test_two_rank_results_equal_the_unsharded_ones():
    from oracle import oracle as O
    from paper_2606_24154_gb300 import inputs as I
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_result_worker, args=(world, port, out), nprocs=world, join=True)
        res = [out[0], out[1]]
    g = I.cube(n_per_edge=4)
    sig, _, _ = O.solve(g)
    pts = I.cell_points(g, 37, I.rng(1, 40))
    phi, E = O.eval_points(g, sig, pts)
    pos, q = I.carrier_cloud(I.thgem(I.PlateSpec(n_phi=12, n_r=2, n_zc=1, n_zf=3), n_plane=2), 61, I.rng(3, 40))
    tgt = I.cell_points(g, 23, I.rng(3, 41))
    sphi, sE = O.space_charge(pos, q, tgt=tgt, soft=1e-6)
    for r in res:
        assert np.array_equal(r[0], phi) and np.array_equal(r[1], E)      # per-point results, any batch
        assert np.array_equal(r[2], pos) and np.array_equal(r[3], q)      # every rank holds every carrier
        assert np.array_equal(r[4], sphi) and np.array_equal(r[5], sE)    # sums over the gathered set
