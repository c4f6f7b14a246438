"""Replica runs on several GPUs of one node: one independent copy of the
workload per rank (the operator has no exchange step between problems), only
the timings are combined.  Host logic, usable with the nccl or gloo backend."""
from __future__ import annotations

import torch
import torch.distributed as tdist


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks of the default
    process group (the list itself when no group of more than one rank
    exists)."""
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return t.tolist()


def weak_value(world_size, cells_per_rank, stages_per_step, ms_per_step):
    """Whole-job Mcell-updates/s per RK stage: every rank updates its own
    cells; the job takes as long as the slowest rank."""
    return world_size * cells_per_rank * stages_per_step / (ms_per_step * 1e-3) / 1e6
