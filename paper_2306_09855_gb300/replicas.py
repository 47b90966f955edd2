"""Multi-process replicas (one process per GPU, launched by torchrun).

Building a network has no exchange step between GPUs, so N processes build N
independent replicas of the workload; the only collectives are a barrier
around the timed region and the reduction of the timing: the slowest rank's
time and the sum of all ranks' connections.
"""
from __future__ import annotations

import os


def world():
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str = "nccl") -> None:
    import torch.distributed as dist
    if world()[1] > 1 and not dist.is_initialized():
        dist.init_process_group(backend)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def reduce_timing(ms: float, n_units: float, device="cpu"):
    """(max of ms over ranks, sum of n_units over ranks); identity on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(n_units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(n_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())
