"""Host-side logic of multi-GPU runs: one process per GPU, independent
reconstructions per rank (no data-path collective), timing aggregated as the
slowest rank's time and the units of all ranks.

Reconstructions of different frames or problems share nothing, so a run on N
GPUs gives every rank its own units (whole problems, or a block of the frames
of a batch) and the only communication is the barrier around the timed region
and two scalar reductions of the result: the maximum of the ranks' times and
the sum of their units.  Works with any torch.distributed backend (NCCL on
GPUs, gloo on CPU for the tests); without an initialised process group it is
the single-process identity.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def _active() -> bool:
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def _device():
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous block of the units owned by `rank` (sizes differ by at most
    one; every unit has exactly one owner)."""
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def barrier() -> None:
    if _active():
        dist.barrier()


def max_over_ranks(x: float) -> float:
    """The largest value of x over all ranks (the slowest rank's time)."""
    if not _active():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    """The sum of x over all ranks (units processed by the whole job)."""
    if not _active():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_local: float, seconds_local: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return sum_over_ranks(units_local) / max_over_ranks(seconds_local)
