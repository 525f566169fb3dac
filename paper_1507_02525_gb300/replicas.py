"""Host-side logic of multi-GPU runs: one process per GPU, no data-path exchange.

The MrDFT of a batch is a set of independent problems (every signal, and
every window of a signal, is transformed on its own), so a multi-GPU job
splits the signals across ranks and each rank runs the whole transform of
its share on its own GPU; nothing is communicated while transforming.  The
only collectives are host-side bookkeeping around a timed region: a barrier
before and after it, and the maximum of the per-rank times.

These helpers hold that logic so that it runs unchanged under the ``gloo``
backend on CPU (tests) and ``nccl`` on GPUs (bench).
"""
from __future__ import annotations

import os
from dataclasses import dataclass
from typing import List, Sequence


@dataclass(frozen=True)
class RankInfo:
    rank: int
    world: int
    local: int


def rank_info() -> RankInfo:
    """Rank, world size and local rank from the launcher's environment
    (torchrun sets RANK / WORLD_SIZE / LOCAL_RANK; a plain run is rank 0 of 1)."""
    return RankInfo(int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                    int(os.environ.get("LOCAL_RANK", "0")))


def shard(lengths: Sequence[int], rank: int, world: int) -> List[int]:
    """Indices of the signals rank `rank` transforms: contiguous blocks whose
    sample counts are balanced greedily (every signal goes to exactly one rank;
    a rank may get none when there are fewer signals than ranks)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of size {world}")
    total = sum(int(n) for n in lengths)
    out, acc = [], 0
    for idx, n in enumerate(lengths):
        # the signal belongs to the rank whose share contains its midpoint
        mid = acc + int(n) / 2.0
        owner = min(world - 1, int(mid * world / total)) if total else 0
        if owner == rank:
            out.append(idx)
        acc += int(n)
    return out


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over the default process group (identity
    when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank scalar (samples processed) over the default group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def job_throughput(total_samples: float, max_ms_per_step: float) -> float:
    """Whole-job throughput in samples per second: all ranks' samples of one
    step over the slowest rank's step time."""
    if max_ms_per_step <= 0:
        raise ValueError("step time must be positive")
    return total_samples / (max_ms_per_step * 1e-3)
