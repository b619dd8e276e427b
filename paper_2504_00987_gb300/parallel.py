"""Host-side logic of running the solver on several GPUs of one node, one
process per GPU.

The work shards with no exchange on the data path: replicas (and batch
instances, and serving requests) are independent, so rank r of W simply owns
a contiguous range of instance numbers (its own Philox streams).  The only
collectives are outside the timed region: a barrier, the max over ranks of
the timed duration (the job is as slow as its slowest rank), and the best
result over all ranks (lowest E, then lowest instance number).  Every
function takes the torch.distributed module (or None for one process).
"""
from __future__ import annotations


def shard(world: int, rank: int, per_rank: int) -> tuple[int, int]:
    """(first_instance, count) of `rank` when every rank runs `per_rank` replicas."""
    if world < 1 or not 0 <= rank < world or per_rank < 0:
        raise ValueError("bad world/rank/per_rank")
    first = rank * per_rank
    if first + per_rank > 1 << 32:
        raise ValueError("instance numbers beyond 2^32")
    return first, per_rank


def split_range(total: int, world: int, rank: int) -> tuple[int, int]:
    """(first, count) of an even split of `total` items over `world` ranks
    (the first total % world ranks get one more)."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad total/world/rank")
    base, extra = divmod(total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def max_over_ranks(dist, values: list[float], device=None) -> list[float]:
    """Element-wise max over ranks (identity for one process)."""
    if dist is None:
        return list(values)
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def sum_over_ranks(dist, values: list[float], device=None) -> list[float]:
    if dist is None:
        return list(values)
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()]


def best_over_ranks(dist, E: int, instance: int, device=None) -> tuple[int, int]:
    """The global best (E, instance): lowest energy, lowest instance on ties."""
    if dist is None:
        return E, instance
    import torch

    key = torch.tensor([E * (1 << 32) + instance], dtype=torch.int64, device=device)
    dist.all_reduce(key, op=dist.ReduceOp.MIN)
    k = int(key.item())
    return k >> 32, k & 0xFFFFFFFF


def any_over_ranks(dist, flag: bool, device=None) -> bool:
    """True on every rank if `flag` is true on any rank (identity for one process)."""
    return max_over_ranks(dist, [1.0 if flag else 0.0], device)[0] > 0.0


def run_until_any(dist, run_slice, max_slices: int, device=None) -> tuple[int, bool]:
    """The global termination flag of Alg. 3 across GPUs.  Within one GPU the
    replicas of a launch share a device flag; across ranks every rank runs its
    replicas in slices (`run_slice(i)` runs slice i, e.g. the next generations
    of resumable replicas, and returns True if one of this rank's replicas
    reached the target), and after every slice the ranks take the OR of their
    flags, so all of them stop after the same slice once any has reached.
    Returns (slices run, reached on some rank)."""
    if max_slices < 0:
        raise ValueError("max_slices < 0")
    for i in range(max_slices):
        if any_over_ranks(dist, bool(run_slice(i)), device):
            return i + 1, True
    return max_slices, False
