"""Host-side logic for running independent instances on several GPUs.

The update has no exchange between instances (each instance is its own
periodic or walled box), so a multi-GPU job is a set of replicas: the
instances of a sweep or of the training-set generation are split into
contiguous blocks, one block per rank, and only the per-instance results are
gathered at the end (no collective on the data path).  Everything here runs
with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous block of unit indices for `rank`: sizes differ by at most one,
    the larger blocks first, and the blocks of ranks 0..world-1 tile 0..n_units-1."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("shard: need 0 <= rank < world and n_units >= 0")
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def _device(dist):
    import torch
    return torch.device("cuda") if dist.get_backend() == "nccl" else torch.device("cpu")


def gather_units(rows: np.ndarray, n_units: int) -> np.ndarray:
    """All-gather per-unit result rows (shape [len(shard)][...], float64) from
    every rank into one [n_units][...] array in unit order, on every rank."""
    import torch
    import torch.distributed as dist
    world, rank = dist.get_world_size(), dist.get_rank()
    mine = shard(n_units, rank, world)
    rows = np.asarray(rows, dtype=np.float64)
    if rows.shape[0] != len(mine):
        raise ValueError("gather_units: rows do not match this rank's shard")
    tail = rows.shape[1:]
    width = max(len(shard(n_units, r, world)) for r in range(world))
    dev = _device(dist)
    buf = torch.zeros((width,) + tail, dtype=torch.float64, device=dev)
    if len(mine):
        buf[:len(mine)] = torch.from_numpy(rows).to(dev)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    out = np.empty((n_units,) + tail)
    for r in range(world):
        s = shard(n_units, r, world)
        out[s.start:s.stop] = parts[r][:len(s)].cpu().numpy()
    return out


def max_over_ranks(x: float) -> float:
    """Largest value of x over the ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
