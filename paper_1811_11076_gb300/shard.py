"""Host side of the multi-GPU run: the query batch is sharded across ranks
(independent problems, one replica of the database per GPU); the only
collectives are host-side (timing, and gathering results for a check).

Nothing here touches the data path of a scan.
"""
from __future__ import annotations

import numpy as np


def query_shard(q_off: np.ndarray, rank: int, world: int, per_rank: int):
    """Queries [rank * per_rank, (rank + 1) * per_rank) of a batch given by its
    point offsets q_off (len >= world * per_rank + 1): returns the point range
    (p0, p1) and the shard's own offsets (starting at 0)."""
    if not (0 <= rank < world) or per_rank < 1:
        raise ValueError("need 0 <= rank < world and per_rank >= 1")
    q_off = np.asarray(q_off, dtype=np.int64)
    if world * per_rank + 1 > q_off.shape[0]:
        raise ValueError("batch has fewer than world * per_rank queries")
    a, b = rank * per_rank, (rank + 1) * per_rank
    p0, p1 = int(q_off[a]), int(q_off[b])
    return (p0, p1), q_off[a:b + 1] - p0


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the slowest rank's time); the value
    itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(ids: np.ndarray, dist_: np.ndarray, device=None):
    """Concatenate every rank's [per_rank, k] results in rank order (on every
    rank); the inputs themselves without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return ids, dist_
    world = dist.get_world_size()
    ti = torch.as_tensor(np.ascontiguousarray(ids), device=device)
    td = torch.as_tensor(np.ascontiguousarray(dist_), device=device)
    gi = [torch.empty_like(ti) for _ in range(world)]
    gd = [torch.empty_like(td) for _ in range(world)]
    dist.all_gather(gi, ti)
    dist.all_gather(gd, td)
    return (torch.cat(gi).cpu().numpy(), torch.cat(gd).cpu().numpy())
