"""One reconstruction split across GPUs by trajectory samples.

The forward operator and its adjoint are sums over the trajectory samples
(Eq. core:formula): s_k(t) = sum_x c_x p_k^T J(x, t) w_t and
(A^T s)_x = sum_t ..., so a contiguous split of the samples partitions the
work.  Each process (one GPU) holds its slice of r, v and s; A gives its own
samples with no exchange, A^T a partial image that the processes sum.  The
library's mpi_pnp_solve_sharded calls back for that sum once for A^T of the
data and once per CG step (N = nx * ny FP64 values); everything else runs
replicated on identical vectors.

This module holds the host logic around that call: the balanced sample
partition, the all-reduce callables (torch.distributed for processes, a
host-staged fixed-order sum for threads of one process), and the driver that
slices the inputs of one process.
"""
from __future__ import annotations

import threading

import numpy as np
import torch


def sample_shard(T: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced slice [t0, t1) of T samples for `rank` of
    `world`: the first T % world ranks take one sample more."""
    if world < 1 or not 0 <= rank < world or T < 0:
        raise ValueError(f"bad shard request: T={T}, rank={rank}, world={world}")
    base, extra = divmod(T, world)
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


def shard_inputs(r, v, s, rank: int, world: int):
    """This rank's contiguous slices of r [T, 2], v [T, 2] and s [n_ch, T]."""
    t0, t1 = sample_shard(r.shape[0], rank, world)
    return r[t0:t1].contiguous(), v[t0:t1].contiguous(), s[:, t0:t1].contiguous()


def dist_allreduce(group=None):
    """Sum across the processes of a torch.distributed group (NCCL for CUDA
    tensors, gloo for CPU ones); every process receives the same sum."""
    import torch.distributed as dist

    def fn(t: torch.Tensor) -> None:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return fn


class ThreadAllreduce:
    """Sum across `world` threads of one process (one shard each, on one or
    several GPUs): each thread's call completes its stream's work, stages its
    values on the host, and after a barrier every thread takes the sum of all
    threads' values in rank order -- a fixed order, so every thread gets the
    bit-identical result and repeated runs agree.  No device-side wait is
    involved: the threads meet on the host between launches."""

    def __init__(self, world: int, timeout: float = 120.0):
        self.world = world
        self._slots: list = [None] * world
        self._barrier = threading.Barrier(world, timeout=timeout)

    def for_rank(self, rank: int):
        def fn(t: torch.Tensor) -> None:
            if t.is_cuda:
                torch.cuda.current_stream(t.device).synchronize()
            self._slots[rank] = t.detach().cpu().numpy().astype(np.float64, copy=True)
            self._barrier.wait()
            tot = np.zeros_like(self._slots[rank])
            for k in range(self.world):
                tot += self._slots[k]
            self._barrier.wait()  # every thread has read the slots
            t.copy_(torch.from_numpy(tot).to(t.device, t.dtype))
        return fn

    def abort(self) -> None:
        """Release threads waiting in the barrier (their calls raise)."""
        self._barrier.abort()


def pnp_solve_sharded(model, grid, r, v, s, n_iter: int, n_cg: int, nu0: float, rank: int,
                      world: int, allreduce, clip_pct: float = 5.0, with_info: bool = False):
    """Algorithm 1 with A on this rank's slice of the samples of (r, v, s)
    (full-length device tensors), the partial adjoint images summed by
    `allreduce`; returns the reconstruction (identical on every rank)."""
    from . import api
    rr, vv, ss = shard_inputs(r, v, s, rank, world)
    return api.mpi_pnp_solve_sharded(model, grid, rr, vv, ss, n_iter, n_cg, nu0, allreduce,
                                     clip_pct=clip_pct, with_info=with_info)
