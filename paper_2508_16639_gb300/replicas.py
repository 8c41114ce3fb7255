"""Multi-GPU use of the library: replicas only.

The Monte Carlo step of one lattice does not shard across GPUs here; what
scales is independent work -- one lattice per rank, or an ensemble / request
stream split across ranks.  One process per GPU (torchrun), no collective on
the data path: ranks only meet for a barrier around the timed region and a
max-reduction of the elapsed times."""
from __future__ import annotations

import os


def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank: int, world: int):
    """The items this rank runs: a round-robin split (every item exactly
    once across ranks, sizes differing by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return list(items)[rank::world]


def replica_seed(seed: int, rank: int) -> int:
    """Seed of this rank's independent lattice."""
    return (seed + rank) & (2**64 - 1)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of `value` over all ranks (identity without a process group)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
