"""Multi-GPU sharding of the evaluation (one process per GPU).

Evaluation at points shards with no data-path collective: every rank holds the same
geometry and charge densities and evaluates its own points (weak scaling: a fixed number
of points per rank).  The only exchange is the timing reduction of the benchmark: the
maximum step time over ranks and the total number of evaluations, so that the
aggregate rate is (all ranks' evaluations) / (slowest rank's time).

For a strong-scaling split of one point set (shard_range), gather_rows puts the ranks'
result blocks back together in rank order.  The dynamic space-charge step partitions the
carriers as targets; every step all-gathers positions and charges (gather_rows on both),
so that every rank sums over all sources for its own targets.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def rank_world():
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def shard_seed_stream(rank: int) -> int:
    """Seed stream of a rank's points: rank r draws stream r of the workload's seed."""
    return int(rank)


def shard_range(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block of [0, n_total) for `rank` (strong-scaling partition)."""
    base, rem = divmod(n_total, world)
    lo = rank * base + min(rank, rem)
    return lo, lo + base + (1 if rank < rem else 0)


def reduce_step_time(ms: float, units: float, device=None) -> tuple[float, float]:
    """(max over ranks of the step time, sum over ranks of the units processed)."""
    rank, world = rank_world()
    if world == 1:
        return float(ms), float(units)
    dev = device if device is not None else torch.device("cpu")
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def gather_rows(local: torch.Tensor, n_total: int) -> torch.Tensor:
    """All-gather of row blocks: rank r holds rows shard_range(n_total, r, world) of an
    (n_total, ...) array; every rank receives the whole array, rows in rank order."""
    rank, world = rank_world()
    if world == 1:
        return local
    lo, hi = shard_range(n_total, rank, world)
    assert local.shape[0] == hi - lo, "local block does not match the partition"
    width = (n_total + world - 1) // world  # the largest block; shorter ones are padded
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: hi - lo] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    out = []
    for r in range(world):
        a, b = shard_range(n_total, r, world)
        out.append(parts[r][: b - a])
    return torch.cat(out, dim=0)


def allgather_carriers(pos_local: torch.Tensor, q_local: torch.Tensor, n_total: int):
    """Positions (n x 3) and charges (n) of all carriers from every rank's block."""
    return gather_rows(pos_local, n_total), gather_rows(q_local, n_total)
