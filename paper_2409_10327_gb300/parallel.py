"""Host-side plumbing for N GPUs (one process per GPU, torch.distributed).

The renderer shards without communication: pixels, views and lights are
independent, the tables and weights are read-only replicas, and pixel_offset
keys the random numbers, so rank r renders the rows shard_range(P, N, r) of a
frame with pixel_offset = the first of them and the gathered frame equals
the whole frame.  Timings are reduced with max_over_ranks.  Training
(rt_backward, rt_distill_backward) is data-parallel: every rank takes an equal
share of the rays, and the gradients are averaged with one all-reduce per
step (allreduce_mean), the only exchange of real data.
"""
from __future__ import annotations

from typing import Iterable, Tuple

import torch
import torch.distributed as dist


def shard_range(n: int, world: int, rank: int) -> Tuple[int, int]:
    """[lo, hi) of rank `rank` among `world` contiguous, disjoint shards covering 0..n."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    return n * rank // world, n * (rank + 1) // world


def _active() -> bool:
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def max_over_ranks(x: float) -> float:
    """The largest x over all ranks (x itself without a process group)."""
    if not _active():
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_mean(tensors: Iterable[torch.Tensor]) -> None:
    """Average each tensor in place over the ranks (no-op without a process group).

    With equal shares of the rays per rank the average of the ranks' mean-loss
    gradients is the gradient of the whole batch's mean loss.
    """
    if not _active():
        return
    w = dist.get_world_size()
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        t.div_(w)
