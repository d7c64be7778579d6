"""Host-side helpers for running independent solves on several GPUs (one process per GPU).

RLOBPCG's solves are independent problems: every rank solves its own matrices on its own GPU and
nothing is exchanged on the data path. The only collectives are the benchmark's barrier around
the timed region and the max over ranks of the elapsed time (weak scaling: total work grows
with the number of ranks).
"""
from __future__ import annotations

import os


def world_from_env():
    """(rank, world_size, local_rank) from the torchrun environment (1 process if unset)."""
    def geti(name, default):
        try:
            return int(os.environ.get(name, default))
        except ValueError:
            return default
    return geti("RANK", 0), geti("WORLD_SIZE", 1), geti("LOCAL_RANK", 0)


def init(world: int, backend: str) -> None:
    """Join the process group (no-op for a single process). MASTER_ADDR/PORT come from torchrun."""
    if world <= 1:
        return
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend)


def barrier(world: int) -> None:
    if world <= 1:
        return
    import torch.distributed as dist
    dist.barrier()


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest value over all ranks (the slowest rank sets a weak-scaling job's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def finish(world: int) -> None:
    if world <= 1:
        return
    import torch.distributed as dist
    if dist.is_initialized():
        dist.barrier()
        dist.destroy_process_group()


def job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank units in (at most) `seconds`."""
    return world * units_per_rank / seconds
