"""Host logic of multi-GPU runs: one process per GPU, each reconstructing its own scans.

A single scan does not shard: the subsets of Eq. 7 are applied one after the other and
each touches the whole volume, so splitting a scan over GPUs would need an exchange of
partial ray sums after every subset.  Scans are independent, so N GPUs run N replicas of
the path, each on its own scans (round-robin shards of a batch or of a serving stream),
with no collective on the data path: the ranks meet at the barriers around a timed region,
in one max-reduction of their elapsed times (the whole-job rate is the units of all ranks
over the slowest rank's time), and in one gather of per-scan results to rank 0 after it.
"""
from __future__ import annotations

import os


def dist_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str, device=None) -> None:
    """Join the process group of a multi-rank run (no-op for one process)."""
    import torch.distributed as dist
    _, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        if device is not None and backend == "nccl":
            dist.init_process_group(backend, device_id=device)
        else:
            dist.init_process_group(backend)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def shard(n_items: int, rank: int, world: int) -> list[int]:
    """Round-robin share of n_items scans for `rank`: every scan goes to exactly one rank,
    and shares differ by at most one scan."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(range(rank, n_items, world))


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the value itself for one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Units of all ranks per second of the slowest rank (weak scaling: fixed units per rank)."""
    if max_seconds <= 0.0:
        raise ValueError("max_seconds must be > 0")
    return units_per_rank * world / max_seconds


def gather_ordered(values, n_items: int, rank: int, world: int):
    """All ranks' per-scan results on rank 0, in global scan order: ``values`` are this
    rank's results for its shard(n_items, rank, world), in that order.  Rank 0 receives the
    list of n_items results, other ranks None; one process gets its own list back."""
    import torch.distributed as dist
    values = list(values)
    if len(values) != len(shard(n_items, rank, world)):
        raise ValueError("one result per scan of the rank's shard")
    if world == 1 or not (dist.is_available() and dist.is_initialized()):
        return values
    parts = [None] * world if rank == 0 else None
    dist.gather_object(values, parts, dst=0)
    if rank != 0:
        return None
    out = [None] * n_items
    for r, part in enumerate(parts):
        for i, v in zip(shard(n_items, r, world), part):
            out[i] = v
    return out
