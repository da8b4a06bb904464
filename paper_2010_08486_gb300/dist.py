"""Replica helpers for running the detector on several GPUs, one process each.

Frames are independent, so the detector shards by frame: every rank detects
its own frames (or camera streams) with its own handle, and nothing crosses
ranks on the data path.  Two collectives exist, both outside it:

* the maximum of a per-rank step time, so that whole-job throughput is the
  units all ranks processed divided by the slowest rank's time;
* an optional sum of volume histograms (per stream or global), the signal a
  steering loop consumes.

Works with any torch.distributed backend (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple, TypeVar

import torch
import torch.distributed as dist

T = TypeVar("T")


def rank_info() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items: Sequence[T], rank: int, world: int) -> List[T]:
    """Round-robin share of `items` for `rank`: every item lands on exactly
    one rank and the shares differ in length by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank %d of %d" % (rank, world))
    return [items[i] for i in range(rank, len(items), world)]


def _active() -> bool:
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks (the value itself when not distributed)."""
    if not _active():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of `value` over all ranks (units processed, blobs found)."""
    if not _active():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def merge_hists(hist: torch.Tensor) -> torch.Tensor:
    """Element-wise sum of every rank's histogram, returned on every rank.

    Counts are summed as int64 (a rank's uint32-range counts cannot overflow
    the sum); float histograms (soft or volume sums) are summed as float64."""
    if hist.dtype.is_floating_point:
        acc = hist.to(torch.float64)
    else:
        acc = hist.to(torch.int64)
    acc = acc.clone()
    if _active():
        dist.all_reduce(acc, op=dist.ReduceOp.SUM)
    return acc


def barrier():
    if _active():
        dist.barrier()
