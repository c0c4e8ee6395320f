"""Multi-GPU host logic: independent replicas, one process per GPU.

Every (start pixel, velocity) of the search is independent, and so is every
search job, so several GPUs run separate work with no exchange on the data
path: each rank searches its own stack (or its share of a job list) on its own
device.  The only communication is host-side bookkeeping over
torch.distributed: a barrier around the timed region and a max over ranks of
the measured times, so that the whole-job rate is the units all ranks
processed divided by the slowest rank's time.  The backend is NCCL on GPUs and
gloo for the CPU tests of this logic.
"""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple


def dist_info() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str = "nccl") -> None:
    """Join the process group when launched with more than one rank."""
    import torch.distributed as dist
    if dist_info()[1] > 1 and not dist.is_initialized():
        dist.init_process_group(backend)


def finish() -> None:
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_initialized():
        dist.barrier()


def shard(n: int, rank: int, world: int) -> range:
    """This rank's contiguous share of n units: sizes differ by at most one, and the
    shares of ranks 0 .. world-1 cover 0 .. n-1 exactly once, in order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


def max_over_ranks(values: Sequence[float], device=None) -> List[float]:
    """Element-wise maximum of `values` over all ranks (the values themselves with one rank)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def sum_over_ranks(values: Sequence[float], device=None) -> List[float]:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.tolist()


def whole_job_rate(units_this_rank: float, seconds_this_rank: float, device=None) -> Tuple[float, float, float]:
    """(rate, total units, slowest time): the units all ranks processed divided by the
    slowest rank's time."""
    total = sum_over_ranks([units_this_rank], device)[0]
    slowest = max_over_ranks([seconds_this_rank], device)[0]
    return total / slowest, total, slowest
