"""Multi-process helpers (one process per GPU).

The relaxation of one grid does not shard without a halo exchange, so several GPUs
run independent replicas of it (weak scaling): each rank relaxes its own copy of the
workload, the job's time is the maximum over ranks, and the job's throughput is
the units all ranks processed divided by that time. No collective touches the data
path; the only collectives are the barrier around the timed region and the max /
sum of two scalars after it.

A batch of independent relaxations shards: `shard` splits the work list across ranks
by cost, each rank relaxes its share as one batch, and `gather_records` collects the
per-problem results (status and observables) in problem order.
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


# ---------------------------------------------------------------- batch work lists
# A batch of independent relaxations (a parameter or interaction scan) shards across
# ranks with no exchange on the data path: each rank relaxes its share as one batch on
# its own GPU, and only the per-problem results (a few numbers each) are gathered.

RECORD_FIELDS = ("index", "converged", "steps", "arrests", "energy", "grad_max", "charge", "flux")


def shard(costs, world: int) -> list[list[int]]:
    """Partition problems 0..n-1 among `world` ranks, balancing the summed cost
    (e.g. interior sites): longest-processing-time-first, each problem to the rank with
    the least cost so far (ties to the lower rank), then each rank's list in ascending
    problem order. Deterministic, so every rank computes the same partition."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def gather_records(local: "list[dict]", n_total: int, group=None) -> "list[dict]":
    """Every rank's per-problem records (dicts with RECORD_FIELDS, "index" the problem's
    position in the full list) -> the full list in problem order, on every rank. One
    all-gather of a fixed-width float64 block per rank (padded to the largest share)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        out = sorted(local, key=lambda r: r["index"])
        return [dict(r) for r in out]
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda") if backend == "nccl" else torch.device("cpu")
    width = len(RECORD_FIELDS)
    cnt = torch.tensor([len(local)], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(counts, cnt, group=group)
    cap = max(int(c.item()) for c in counts)
    block = torch.full((max(cap, 1), width), -1.0, dtype=torch.float64, device=dev)
    for k, r in enumerate(local):
        block[k] = torch.tensor([float(r[f]) for f in RECORD_FIELDS], dtype=torch.float64)
    blocks = [torch.empty_like(block) for _ in range(world)]
    dist.all_gather(blocks, block, group=group)
    out: list[dict | None] = [None] * n_total
    for rk, (b, c) in enumerate(zip(blocks, counts)):
        for row in b[: int(c.item())].cpu().tolist():
            rec = dict(zip(RECORD_FIELDS, row))
            rec["index"] = int(rec["index"])
            rec["converged"] = bool(rec["converged"])
            rec["steps"] = int(rec["steps"])
            rec["arrests"] = int(rec["arrests"])
            rec["rank"] = rk
            if not 0 <= rec["index"] < n_total or out[rec["index"]] is not None:
                raise RuntimeError(f"problem {rec['index']} gathered twice or out of range")
            out[rec["index"]] = rec
    missing = [i for i, r in enumerate(out) if r is None]
    if missing:
        raise RuntimeError(f"problems {missing[:8]} were not relaxed by any rank")
    return out  # type: ignore[return-value]
