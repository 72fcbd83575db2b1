"""Process-group helpers for the multi-GPU benchmark path.

The patch groups of a step are independent (paper Sec. 2), so N GPUs run N
independent problems of the same size (weak scaling): no collective touches
the data path.  The only collectives are the barrier around the timed region
and the max over ranks of the elapsed time.  Works with the nccl backend on
GPUs and gloo on CPU (tests).
"""
from __future__ import annotations

import os


def env_world():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def init(backend):
    """Initialise the default process group when launched with WORLD_SIZE > 1."""
    import torch.distributed as dist
    rank, world, _ = env_world()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x, device="cpu"):
    """Max of a float over all ranks (identity on one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(n_units, rank, world):
    """Contiguous [lo, hi) slice of n_units for this rank (strong-scaling split;
    the benchmark itself gives every rank a full problem)."""
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def finalize():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
