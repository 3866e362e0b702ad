"""Splitting the start vectors of one sweep over several processes.

The moments are averages over independent start vectors (Theorem 3.1's
estimator), so P processes can each sweep a contiguous block of the vectors
-- passing its offset as the start-vector index, so that the union is exactly
the single-process set -- and combine once at the end: every rank contributes
n_l * mu^(l) and the weighted sum is divided by the total count.  No data is
exchanged during the sweep.
"""
from __future__ import annotations

import numpy as np


def vector_shard(n_v_total: int, world: int, rank: int) -> tuple[int, int]:
    """(offset, count) of rank's contiguous block; the first n_v_total % world
    ranks take one extra vector."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(int(n_v_total), int(world))
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def combine_moments(mu_local: np.ndarray, count: int, n_v_total: int, all_reduce) -> np.ndarray:
    """Average of the ranks' moments weighted by their vector counts.

    ``all_reduce`` sums a float64 array in place over all ranks (e.g. a
    torch.distributed all_reduce wrapped to take numpy)."""
    buf = np.ascontiguousarray(mu_local, dtype=np.float64) * float(count)
    buf = all_reduce(buf)
    return buf / float(n_v_total)


def torch_all_reduce(group=None, device=None):
    """An ``all_reduce`` for combine_moments over torch.distributed (gloo or nccl)."""
    import torch
    import torch.distributed as dist

    def _reduce(arr: np.ndarray) -> np.ndarray:
        t = torch.from_numpy(arr.copy())
        if device is not None:
            t = t.to(device)
        dist.all_reduce(t, group=group)
        return t.cpu().numpy()
    return _reduce
