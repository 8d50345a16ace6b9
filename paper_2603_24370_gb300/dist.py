"""Multi-process helpers for the throughput harness (one process per GPU).

The relaxation of one grid does not shard without a halo exchange, so several GPUs
run independent replicas (weak scaling): each rank relaxes its own copy of the
workload, the job's time is the maximum over ranks, and the job's throughput is
the units all ranks processed divided by that time. No collective touches the data
path; the only collectives are the barrier around the timed region and the max /
sum of two scalars after it.
"""
from __future__ import annotations

import os


def env_rank() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (1 process: 0, 0, 1)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def pin_visible_device(local_rank: int, world: int) -> None:
    """Give each rank exactly its own GPU before CUDA initialises (the C library then
    always works on device 0 of the process)."""
    if world <= 1:
        return
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    ids = [v for v in vis.split(",") if v.strip()] if vis else None
    os.environ["CUDA_VISIBLE_DEVICES"] = ids[local_rank] if ids and local_rank < len(ids) else str(local_rank)


def aggregate(local_units: float, local_seconds: float, group=None) -> tuple[float, float]:
    """(job units, job seconds): units summed over ranks, time = max over ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(local_units), float(local_seconds)
    backend = dist.get_backend(group)
    dev = torch.device("cuda") if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(u.item()), float(t.item())


def barrier(group=None) -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier(group=group)
