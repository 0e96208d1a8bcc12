"""Weak-scaling split of the batched workload over ranks (one process per GPU).

The spectra of different sources are independent (Eqs. 1-2 act on each
source alone), so every rank runs its own batch of M sources on its own GPU
and no data crosses ranks.  The host logic here is what the ranks share: the
seed of each rank's sources, the barrier around the timed region, the
maximum of the ranks' times, and the whole-job rate."""
from __future__ import annotations

from . import synth


def rank_params(M: int, rank: int) -> synth.ModelParams:
    """The sources of one rank: the generator's seed is the rank, so ranks draw
    different sources and rank 0 draws the single-GPU batch."""
    return synth.model_params(M, seed=rank)


def barrier():
    """Barrier of the default process group, or nothing without one."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over the ranks of the default process group (the value
    itself without one); device: where the reduction's tensor lives (a CUDA
    device for NCCL, None for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, M: int, steps: int, ms_max: float) -> float:
    """Whole-job spectra per second: all ranks' spectra over the slowest rank's time."""
    return world * M * steps / (ms_max * 1e-3)
