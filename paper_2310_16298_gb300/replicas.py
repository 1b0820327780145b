"""Multi-GPU runs as independent replicas.

Every unit of work the library runs (one grid solve, one problem of a batch,
one served request) is independent of every other: the sweep of Eq. (final)
reads only its own grid.  So N GPUs run N replicas, each on its own shard of
the units, with no data exchange; the only collective is the max-over-ranks
reduction of the measured time (one float per run).  Throughput is then the
units of all ranks divided by the slowest rank's time (weak scaling: the
units per GPU stay fixed as N grows).
"""
from typing import List, Sequence


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous, balanced block of unit indices owned by ``rank``
    (sizes differ by at most one; every index is owned exactly once)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    if n_units < 0:
        raise ValueError("negative unit count")
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def route(i: int, world: int) -> int:
    """Rank that serves the i-th request of an arrival stream (round robin,
    so that every rank sees the same arrival process thinned by ``world``)."""
    return i % world


def routed(items: Sequence, rank: int, world: int) -> List:
    """The items of a stream that ``route`` sends to ``rank``, in order."""
    return [x for i, x in enumerate(items) if route(i, world) == rank]


def field_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's own replica of a single-grid workload (rank 0 keeps the
    workload's seed, so its results match a one-GPU run)."""
    return base_seed + 1_000_003 * rank


def max_over_ranks(seconds: float, device=None) -> float:
    """Largest value over all ranks (the slowest replica); the identity when
    torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(count: float, device=None) -> float:
    """Total of a per-rank count (units or updates) over all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(count)
    t = torch.tensor([float(count)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
