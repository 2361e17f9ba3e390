"""Replica bookkeeping for runs on several GPUs of one node.

Worlds are independent, so a multi-GPU run is N replicas: each rank simulates its own block of
worlds (weak scaling) and nothing is exchanged on the data path.  torch.distributed carries only
the timing barrier and the reductions of per-rank timings and counts; the helpers below take
whatever process group is initialised (NCCL on GPUs, gloo on CPU in tests).
"""
from __future__ import annotations

import os


def env_rank():
    """(rank, world size, local rank) from the torchrun environment (single process: 0, 1, 0)."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def rank_seed(base, rank):
    """Each rank draws its own worlds: distinct, reproducible seeds."""
    return int(base) + 1000 * int(rank)


def world_block(total, rank, world):
    """Contiguous block [lo, hi) of `total` worlds owned by `rank` (strong-scaling split)."""
    per, extra = divmod(int(total), int(world))
    lo = rank * per + min(rank, extra)
    return lo, lo + per + (1 if rank < extra else 0)


def reduce_scalar(x, op="max", device=None):
    """All-reduce one float over the initialised process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = device or ("cuda" if dist.get_backend() == "nccl" else "cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())
