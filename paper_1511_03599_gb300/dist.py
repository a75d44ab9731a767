"""Host-side logic of running the PFB on several GPUs (one process per GPU).

The transform partitions without any exchange: output spectrum s reads raw
spectra s .. s+T-1 only, so a stream is cut into contiguous output ranges and
each rank reads its range plus a T-1 raw-spectrum read-only halo; outputs are
disjoint and no collective is needed on the data path.  (Whole beams are the
other natural unit.)  The only collectives here are for timing: a barrier and
the maximum of the per-rank step times.
"""
from __future__ import annotations

import os


def env_rank_world():
    """(rank, local_rank, world_size) from the torchrun environment (defaults: single process)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def shard_spectra(n_spectra: int, T: int, rank: int, world: int):
    """Contiguous output range [s0, s1) of `rank` and the raw range [s0, s1 + T - 1) it reads.

    Ranges are balanced to within one spectrum and cover [0, n_spectra) exactly.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    s0 = n_spectra * rank // world
    s1 = n_spectra * (rank + 1) // world
    return s0, s1, s0, s1 + T - 1


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's own synthetic stream (weak scaling: every rank a full workload)."""
    return base + 7919 * rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
