"""Host logic of multi-GPU runs: replicas only.

The MD path does not shard a single system (the paper runs one GPU per simulation); independent
replicas do.  With N processes (one per GPU, torchrun), each rank runs its own ensemble of replicas
with seeds derived from the rank, there is no collective on the data path, and the only
communication is a barrier and the max-over-ranks of the timed duration.
"""
from __future__ import annotations

import synth


def rank_seed(config_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s ensemble (rank 0 keeps the workload's own seed)."""
    return int(config_seed) + 1000 * int(rank)


def rank_ensemble(rank: int, replicas: int | None = None):
    """The KA ensemble workload (512 replicas, N_r ~ U{512..4096}) as run by `rank`.

    Every rank runs the same replica sizes (so per-GPU work is fixed as ranks are added: weak
    scaling) with different initial configurations.
    """
    wl = synth.workload("ka_ensemble512", replicas=replicas)
    if rank:
        sizes = [s.n for s in wl.states]
        seed = rank_seed(1004, rank)
        wl.states = [synth.ka_random_state(n, 1.2, wl.T, synth.replica_seed(seed, r))
                     for r, n in enumerate(sizes)]
    return wl


def max_over_ranks(ms: float, device=None) -> float:
    """Largest of the ranks' timed durations (the job's wall time); identity without a process
    group.  Works with the NCCL (CUDA tensor) and gloo (CPU tensor) backends."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(particles_per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Whole-job particle-steps/s: all ranks' particle-steps over the slowest rank's time."""
    return particles_per_rank * world * steps / (ms_max / 1e3)
