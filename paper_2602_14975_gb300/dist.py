"""Multi-GPU support: replicas only. Each rank (one process per GPU) runs its
own replicas with no data-path communication; the only collectives are the
barriers around timed regions and the max-reduction of the timings."""
from __future__ import annotations

import os


def world():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str = "nccl", device=None):
    import torch.distributed as dist
    ws, _, _ = world()
    if ws > 1 and not dist.is_initialized():
        if device is not None and backend == "nccl":
            dist.init_process_group(backend, device_id=device)
        else:
            dist.init_process_group(backend)
    return ws


def barrier(device=None):
    import torch
    import torch.distributed as dist
    if device is not None and device.type == "cuda":
        torch.cuda.synchronize(device)
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (timings: the slowest rank sets the pace)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_initialized() and dist.get_world_size() > 1):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_id(rank: int, local_index: int, stride: int = 100000) -> int:
    """Globally unique replica id (it keys the noise stream of the replica)."""
    return rank * stride + local_index


def aggregate(units_per_rank: float, seconds_max: float, n_ranks: int) -> float:
    """Whole-job throughput under weak scaling: every rank processed
    units_per_rank in at most seconds_max."""
    return units_per_rank * n_ranks / seconds_max
