"""Multi-process runs (one process per GPU, launched by torchrun).

Replicas: building a network has no exchange step between GPUs, so N
processes build N independent replicas of the workload; the only collectives
are a barrier around the timed region and the reduction of the timing: the
slowest rank's time and the sum of all ranks' connections.

Target shards (Sec. 4 names target-distributed construction as future work):
rank r builds the connections onto its contiguous range of target nodes
(snc_set_target_shard); every draw is keyed by (projection, node, slot), so
no connection data moves between ranks.  The one collective is an all-gather
of the per-rank counts (8 bytes a rank), which places each rank's
connections in a global numbering.
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


def shard_ranges(n_nodes: int, world_size: int):
    """Balanced contiguous target ranges (first, n), one per rank."""
    base, extra = divmod(int(n_nodes), int(world_size))
    out, first = [], 0
    for r in range(int(world_size)):
        n = base + (1 if r < extra else 0)
        out.append((first, n))
        first += n
    return out


def gather_shard_counts(n_local: int, device="cpu"):
    """Every rank's connection count and the first global position of each
    rank's connections (exclusive prefix over ranks)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [int(n_local)], [0]
    t = torch.tensor([int(n_local)], dtype=torch.int64, device=device)
    parts = [torch.zeros_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, t)
    counts = [int(x.item()) for x in parts]
    firsts, run = [], 0
    for c in counts:
        firsts.append(run)
        run += c
    return counts, firsts
