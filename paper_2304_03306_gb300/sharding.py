"""Layout of independent units (domains) over the ranks of a multi-process run.

The solver's data-parallel axis is the set of independent domains (the radius and shape
sweeps, the corrector's training trajectories): each rank advances its own domains with no
collective on the data path.  The host-side pieces here are the only cross-rank steps: a
deterministic cost-balanced assignment of units to ranks, the max-over-ranks of a timing,
and a gather of per-unit diagnostics.  They use torch.distributed and work with the gloo
backend (CPU tests) as well as NCCL.
"""
from __future__ import annotations


def shard(costs, rank: int, world: int) -> list[int]:
    """Indices of the units rank `rank` of `world` owns: largest cost first onto the least
    loaded rank (ties: lower rank, then lower index), so every rank computes the same
    assignment without communicating."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += costs[i]
    return [i for i in range(len(costs)) if owner[i] == rank]


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def max_over_ranks(x: float, device=None) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    dist = _dist()
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather(rows: list) -> list:
    """Every rank's list of per-unit records, concatenated in rank order, on every rank."""
    dist = _dist()
    if dist is None:
        return list(rows)
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, list(rows))
    return [r for part in out for r in part]


def barrier(device=None):
    dist = _dist()
    if dist is not None:
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()
